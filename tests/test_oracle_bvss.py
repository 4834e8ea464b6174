"""Pins for the BVSS, U_div, getVI and binary-MMA oracles (CPU only)."""
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _brute_bvss(g, sigma, tau=None):
    """Tiny-input brute force: dictionary of slice sets built arc by arc."""
    theta = 32 // sigma
    tau = tau or 32 * theta
    lanes = tau // theta
    Ns = (g.n + sigma - 1) // sigma
    sets = [dict() for _ in range(Ns)]
    for j in range(g.n):
        for i in g.col[g.row_ptr[j]:g.row_ptr[j + 1]]:
            d = sets[j // sigma]
            d[int(i)] = d.get(int(i), 0) | (1 << (j % sigma))
    rows, masks, real, v2r = [], [], [0], []
    for s in range(Ns):
        items = sorted(sets[s].items())
        nv = (len(items) + tau - 1) // tau
        for v in range(nv):
            chunk = items[v * tau:(v + 1) * tau]
            chunk = chunk + [(0, 0)] * (tau - len(chunk))
            rows += [r for r, _ in chunk]
            for l in range(lanes):
                w = 0
                for c in range(theta):
                    w |= chunk[l * theta + c][1] << (sigma * c)
                masks.append(w)
            v2r.append(s)
        real.append(real[-1] + nv)
    return np.array(rows, np.int64), np.array(masks, np.uint64), np.array(real), np.array(v2r)


@pytest.mark.parametrize("sigma,tau", [(8, None), (16, None), (32, None), (8, 32)])
@pytest.mark.parametrize("maker", [lambda: gg.er(70, 300, seed=1, directed=True),
                                   lambda: gg.rmat(8, seed=2), lambda: gg.star(300),
                                   lambda: gg.path(1)])
def test_bvss_matches_brute_force(sigma, tau, maker):
    g = maker()
    b = oracle.bvss(g, sigma, tau)
    rows, masks, real, v2r = _brute_bvss(g, sigma, tau)
    assert np.array_equal(b["rowIds"], rows)
    assert np.array_equal(b["masks"].astype(np.uint64), masks)
    assert np.array_equal(b["realPtrs"], real)
    assert np.array_equal(b["v2r"], v2r)


@pytest.mark.parametrize("sigma,tau", [(8, None), (16, None), (32, None), (8, 32)])
def test_bvss_invariants(sigma, tau):
    g = gg.rmat(13, seed=5)
    b = oracle.bvss(g, sigma, tau)
    tau, theta, Nv, Ns = b["tau"], b["theta"], b["Nv"], b["Ns"]
    sm = b["slot_masks"].reshape(Nv, tau)
    rows = b["rowIds"].reshape(Nv, tau)
    # every arc j -> i is exactly one mask bit (bit j mod sigma of slice (j // sigma, i))
    nbits = sum(bin(int(x)).count("1") for x in sm.ravel())
    assert nbits == g.nnz
    vss, slot = np.nonzero(sm)
    ss = b["v2r"][vss]
    arcs = set()
    for v, k in zip(vss, slot):
        m = int(sm[v, k])
        s = int(b["v2r"][v])
        for bit in range(sigma):
            if m >> bit & 1:
                arcs.add((s * sigma + bit, int(rows[v, k])))
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    assert arcs == set(zip(src.tolist(), g.col.tolist()))
    # padding: zero masks only after the real slices; at most one padded VSS per slice set
    filled = (sm != 0).sum(1)
    assert np.all(filled >= 1)
    padded = np.flatnonzero(filled < tau)
    assert len(padded) <= Ns
    for v in padded:
        assert np.all(sm[v, filled[v]:] == 0) and np.all(rows[v, filled[v]:] == 0)
    # realPtrs / virtualToReal are inverse maps
    rp = b["realPtrs"]
    for s in range(Ns):
        assert np.all(b["v2r"][rp[s]:rp[s + 1]] == s)
    last_of_set = np.r_[b["v2r"][1:] != b["v2r"][:-1], True]
    assert np.all(filled[~last_of_set] == tau)
    # rows ascending within a slice set
    for s in range(0, Ns, max(1, Ns // 50)):
        r = rows[rp[s]:rp[s + 1]][sm[rp[s]:rp[s + 1]] != 0]
        assert np.all(np.diff(r) > 0)
    assert len(np.unique(ss)) == (np.diff(rp) > 0).sum()


def test_bvss_golden_fig1():
    """Fig. 1: three slice sets split into 3, 1 and 2 VSSs; slice set 2 owns
    VSSs 4 and 5; vertex 3's slice there has mask 01010010 (LSB first); with
    frontier bits 11000000 the popcount is nonzero, vertex 3 lands in slice
    set 0 at its 4th bit, and VSSs 0, 1, 2 are enqueued."""
    gold = json.load(open(os.path.join(GOLD, "fig1_bvss_example.json")))
    u, v = [], []
    # a directed graph whose columns 0..23 realise the caption's counts
    for r in range(100, 400):
        u.append(0); v.append(r)          # slice set 0: 300 slices -> 3 VSSs
    for r in range(100, 150):
        u.append(8); v.append(r)          # slice set 1: 50 slices  -> 1 VSS
    for r in range(100, 300):
        u.append(16); v.append(r)         # slice set 2: 200 + 1 slices -> 2 VSSs
    for c1 in gold["vertex_3_in_neighbour_columns_1_indexed"]:
        u.append(16 + c1 - 1); v.append(3)
    g = gg.from_edges(400, u, v, symmetrize=False)
    b = oracle.bvss(g, gold["sigma"])
    per_set = np.diff(b["realPtrs"])
    assert per_set[:3].tolist() == gold["vss_per_slice_set"]
    assert np.all(per_set[3:] == 0)
    assert list(range(b["realPtrs"][2], b["realPtrs"][3])) == gold["vss_of_slice_set_2"]
    tau = b["tau"]
    sm = b["slot_masks"].reshape(b["Nv"], tau)
    rows = b["rowIds"].reshape(b["Nv"], tau)
    hit = [(v_, k) for v_ in gold["vss_of_slice_set_2"] for k in range(tau)
           if rows[v_, k] == 3 and sm[v_, k] != 0]
    assert len(hit) == 1
    m = int(sm[hit[0]])
    assert "".join(str(m >> i & 1) for i in range(8)) == gold["vertex_3_mask_in_slice_set_2"]
    alpha = int(gold["frontier_bits_of_slice_set_2"][::-1], 2)
    word = np.array([m], np.uint64)
    assert oracle.slice_hits(word, alpha)[0, 0] == gold["vertex_3_hit"]
    assert 3 // 8 == gold["vertex_3_slice_set"] and 3 % 8 + 1 == gold["vertex_3_bit_set_in_F_next_1_indexed"]
    s0 = gold["vertex_3_slice_set"]
    assert list(range(b["realPtrs"][s0], b["realPtrs"][s0 + 1])) == gold["enqueued_vss"]


def test_udiv_arithmetic_progression():
    """Column c of a full VSS whose 128 slices are rows 0..127 holds rows
    c, c+4, ..., c+124: 32 terms with step 4, population std 4*sqrt((32^2-1)/12)."""
    g = gg.from_edges(136, [128] * 128, list(range(128)), symmetrize=False)
    b = oracle.bvss(g, 8)
    assert b["Nv"] == 1
    expect = 4.0 * np.sqrt((32 ** 2 - 1) / 12.0)
    assert abs(oracle.update_divergence(b) - expect) < 1e-12


@pytest.mark.parametrize("sigma,tau", [(8, None), (16, None), (32, None), (8, 32)])
def test_udiv_vs_numpy_std(sigma, tau):
    g = gg.rmat(10, seed=9)
    b = oracle.bvss(g, sigma, tau)
    tau, Nv, theta = b["tau"], b["Nv"], b["theta"]
    tot = 0.0
    for v in range(Nv):
        cols = []
        for c in range(theta):
            idx = [v * tau + l * theta + c for l in range(tau // theta)]
            sel = [i for i in idx if b["slot_masks"][i] != 0]
            if sel:
                cols.append(np.std(b["rowIds"][sel].astype(np.float64)))
        tot += np.mean(cols)
    assert abs(oracle.update_divergence(b) - tot / Nv) <= 1e-9 * max(1.0, tot / Nv)


def test_udiv_narrow_vss_arithmetic_progression():
    """tau = 32: the 128 slices of rows 0..127 fill four VSSs of eight lane
    words; column c of VSS q holds rows 32q + c, 32q + c + 4, ..., 8 terms
    with step 4, population std 4*sqrt((8^2-1)/12)."""
    g = gg.from_edges(136, [128] * 128, list(range(128)), symmetrize=False)
    b = oracle.bvss(g, 8, 32)
    assert b["Nv"] == 4 and b["lanes"] == 8 and b["masks"].size == 32
    expect = 4.0 * np.sqrt((8 ** 2 - 1) / 12.0)
    assert abs(oracle.update_divergence(b) - expect) < 1e-12


def test_udiv_scrambled_rmat_below_threshold():
    """Scattered row ids over [0, n) give a column std of at most about
    n/sqrt(12) (18,900 for n = 65,536), and columns holding a single slice
    contribute 0, so scale-16 RMAT stays under the 25,000 threshold of §7.1
    and the literal rule dispatches it to the eager kernel."""
    g = gg.rmat(16, seed=1)
    u = oracle.update_divergence(oracle.bvss(g, 8))
    assert 1000 < u < 65536 / 12 ** 0.5 < 25000


def test_getvi_golden():
    gold = json.load(open(os.path.join(GOLD, "getvi_n24.json")))
    n, sigma, rho = gold["n"], gold["sigma"], gold["rho"]
    assert rho == -(-n // sigma)
    idx = oracle.get_vi(np.arange(n), rho, sigma)
    order = np.empty(n, np.int64)
    order[idx] = np.arange(n)
    assert order[:6].tolist() == gold["printed_prefix"]
    assert order[-3:].tolist() == gold["printed_suffix"]


@pytest.mark.parametrize("n", [1, 7, 8, 9, 1000, 65537])
def test_getvi_bijection(n):
    rho = -(-n // 8)
    idx = oracle.get_vi(np.arange(rho * 8), rho, 8)
    assert np.array_equal(np.sort(idx), np.arange(rho * 8))


# ------------------------------------------------------------ binary MMA
def test_frag_b_lanes_golden():
    gold = json.load(open(os.path.join(GOLD, "fig3_fragb_lanes.json")))
    b = oracle.paper_frag_b(0xA5)
    assert np.flatnonzero(b).tolist() == gold["nonzero_fragB_lanes"]
    assert all(b[t] == 0xA5 for t in range(32) if t % 9 == 0)
    assert all(b[t] == 0xA5 << 8 for t in range(32) if t % 9 == 4)


def _mma_by_matmul(a, b):
    """Independent check of the emulator: unpack to 0/1 matrices and use a
    plain integer matmul."""
    A = np.zeros((8, 128), np.int64)
    B = np.zeros((128, 8), np.int64)
    for t in range(32):
        for bit in range(32):
            A[t // 4, 32 * (t % 4) + bit] = int(a[t]) >> bit & 1
            B[32 * (t % 4) + bit, t // 4] = int(b[t]) >> bit & 1
    D = A @ B
    return np.array([[D[t // 4, 2 * (t % 4)], D[t // 4, 2 * (t % 4) + 1]] for t in range(32)])


def test_mma_emulator_vs_matmul():
    rs = np.random.RandomState(0)
    for _ in range(10):
        a = rs.randint(0, 2 ** 32, 32, dtype=np.uint64)
        b = rs.randint(0, 2 ** 32, 32, dtype=np.uint64)
        assert np.array_equal(oracle.mma_m8n8k128_b1(a, b), _mma_by_matmul(a, b))


@pytest.mark.parametrize("alpha", [0, 1, 0x80, 0xFF, 0x5A, 0x03])
def test_k3_identity(alpha):
    """With the Fig. 3 layout, lane t's two fragC entries are exactly the
    popcounts of its own two packed masks against alpha (no wasted output,
    no intra-warp exchange), for both rounds of a VSS."""
    rs = np.random.RandomState(alpha)
    words = rs.randint(0, 2 ** 32, 32, dtype=np.uint64)
    words[0] = 0
    words[1] = 0xFFFFFFFF
    words[2] = 0x01020408
    fb = oracle.paper_frag_b(alpha)
    for rnd in range(2):
        a = (words >> np.uint64(16 * rnd)) & np.uint64(0xFFFF)
        d = oracle.mma_m8n8k128_b1(a, fb)
        for t in range(32):
            m0 = int(words[t]) >> (16 * rnd) & 0xFF
            m1 = int(words[t]) >> (16 * rnd + 8) & 0xFF
            assert d[t, 0] == bin(m0 & alpha).count("1")
            assert d[t, 1] == bin(m1 & alpha).count("1")
    hits = oracle.slice_hits(words, alpha)
    for t in range(32):
        for c in range(4):
            assert hits[t, c] == (((int(words[t]) >> (8 * c)) & 0xFF & alpha) != 0)


@pytest.mark.parametrize("alpha", [0, 1, 0x80, 0xFF, 0x5A])
def test_one_slice_per_row_layout_needs_sixteen_mmas(alpha):
    """The layout Fig. 3 improves on (one slice per fragment row, the
    frontier in fragB column 0): MMA i takes slices 8i .. 8i + 7, slice 8i + r
    in the low byte of lane 4r's fragA word; D[r][0] (lane 4r, first entry)
    is its popcount against alpha.  16 MMAs cover a 128-slice VSS (Fig. 3's
    layout: 2), and only column 0 of each fragC is useful."""
    rs = np.random.RandomState(7 + alpha)
    words = rs.randint(0, 2 ** 32, 32, dtype=np.uint64)
    words[3] = 0
    fb = np.zeros(32, np.uint64)
    fb[0] = alpha
    want = oracle.slice_hits(words, alpha)
    used = np.zeros((32, 2), bool)
    for i in range(16):
        a = np.zeros(32, np.uint64)
        for t in range(0, 32, 4):
            r = t // 4
            a[t] = (int(words[2 * i + r // 4]) >> (8 * (r % 4))) & 0xFF
        d = oracle.mma_m8n8k128_b1(a, fb)
        for r in range(8):
            k = 8 * i + r
            assert (d[4 * r, 0] > 0) == want[k // 4, k % 4]
            used[4 * r, 0] = True
        assert not d[~used].any()        # every other fragC entry is zero: wasted
    assert used.sum() == 8               # 8 of the 64 fragC entries per MMA
