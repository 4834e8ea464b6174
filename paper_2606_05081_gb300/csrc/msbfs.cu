// Multi-source BFS (§6.1, Algorithm 5) and exact closeness centrality
// (§6.2, Eq. 6-7).
//
// kappa BFSs run at once as bit lanes: every vertex owns a kappa-bit element
// (KW = kappa/32 words) of the frontier F, visited V_curr and V_next arrays,
// stored at the remapped index getVI(u, rho) = (u mod 8) * rho + u / 8
// (rho = ceil(n/8)).  One persistent cooperative kernel runs all levels:
//   stage 1 (lazy marking): a warp takes one VSS of the queue; its lanes
//     form 32/KW groups of KW lanes, group g handling slices g, g+G, ...;
//     lane w of a group holds word w of the 8 frontier elements of the VSS's
//     slice set, so the hit vector of a slice is the OR of the frontier
//     words its mask selects (Eq. 2 evaluated for kappa lanes at once); a
//     nonzero word is OR-ed into V_next with one fire-and-forget atomic per
//     word (coalesced across the group) and the target's slice set is
//     marked dirty;
//   stage 2 (finalize): only dirty slice sets are visited (a list built in
//     stage 1); per vertex diff = V_curr xor V_next gives the lanes that
//     reached it at this level: F = diff, V_curr = V_next, levels (source-
//     major) and the closeness sums far += level * popc(diff) (Eq. 6),
//     reach += popc(diff); activeSets = OR of the diffs; a set with any
//     active lane enqueues its VSSs.
// Levels (when asked for) are staged as one byte per (vertex, lane) in
// vertex-major rows of kappa bytes, so a word's new lanes land in one 32-byte
// sector; after the last level the grid transposes the rows into the
// source-major int32 output with coalesced stores.  A lane-major int32 store
// per reached (vertex, lane) would touch one sector per store in a k x n
// array far larger than L2.
// The words of lanes that are inactive for a slice set (activeSets word = 0)
// are never loaded.
#include <cstdio>
#include <cstring>
#include <vector>

#include "msbfs.h"
#include "tc.cuh"

struct MsCtl {
    unsigned long long bar;
    int err;
    int nlevels;
    int timeout_where;
    int qlen[2];
    int dlen[2];
};

// Work counters of the multi-source launches of one call (host-visible
// through blest_msbfs_stats): the terms of the kernel's byte model.
struct MsStats {
    unsigned long long launches;    // persistent-kernel launches (batches)
    unsigned long long levels;      // levels run, summed over the launches
    unsigned long long vss;         // VSSs processed in stage 1
    unsigned long long hit_words;   // nonzero kappa-bit words OR-ed into V_next
    unsigned long long dirty_sets;  // slice sets finalised in stage 2
    unsigned long long pull_levels; // levels whose stage 1 pulled (summed over the launches)
    unsigned long long pull_arcs;   // in-neighbour elements read by pulling vertices
};

struct MsbfsWork {
    int kappa = 0;
    int KW = 0;
    unsigned *F = nullptr, *Vc = nullptr, *Vn = nullptr, *active = nullptr;
    int *dirty = nullptr;
    int *dlist[2] = {nullptr, nullptr};
    int *Q[2] = {nullptr, nullptr};
    MsCtl *ctl = nullptr;
    MsCtl *h_ctl = nullptr;
    MsStats *stats = nullptr;      // device counters of the current call
    int *stamp = nullptr;          // per slice set: the level stage 2 last finalised it
    unsigned char *lv8 = nullptr;  // staged levels: rho * 8 rows of kappa bytes (allocated on first use)
    int *d_src = nullptr;
    int grid = 0;
    int grid_tc = -1;              // grid of the tensor-core kernel (-1: not computed yet)
    long long *far = nullptr, *reach = nullptr;   // closeness accumulators (reordered ids)
    // closeness: one batch (source ids from a device cursor, the persistent
    // kernel, cursor advance) captured once in a CUDA graph and replayed
    int *k_dev = nullptr;          // sources in the current batch
    long long *cursor = nullptr;   // [0] next source, [1] end of the range
    int *sticky = nullptr;         // first device error of any replayed batch
    cudaGraph_t cc_graph = nullptr;
    cudaGraphExec_t cc_exec = nullptr;
    cudaStream_t cc_stream = nullptr;
    int cc_engine = -1;            // stage-1 engine the captured batch graph launches
};

namespace {

constexpr int MS_BLOCK = 512;

struct MsParams {
    int n, rho, k;
    int lpv;                      // lane words per VSS: 32 (tau = 128) or 8 (tau = 32)
    const int *__restrict__ rowIds;
    const unsigned *__restrict__ masks;
    const int *__restrict__ realPtrs;
    const int *__restrict__ v2r;
    unsigned *F, *Vc, *Vn, *active;
    int *dirty;
    int *dlist[2];
    int *Q[2];
    MsCtl *ctl;
    const int *srcs;              // k source ids, original numbering
    const int *new_of_old;        // may be null
    const int *old_of_new;        // may be null
    const int *k_dev;             // non-null: the batch size is read here (graph replays)
    int *levels;                  // k*n, source-major, original ids; may be null
    unsigned char *lv8;           // non-null: levels staged as bytes, row u (reordered id) of KW*32
                                  //    lanes; LV8_FAR marks a lane written directly to levels
    long long *far, *reach;       // may be null
    MsStats *stats;               // work counters (added once per CTA and level)
    int Nv;                       // VSSs of the BVSS
    int remap;                    // 1: getVI element order of §6.1; 0: element u at index u (ablation)
    int track;                    // 1: activeSets / dirtySets of Algorithm 5; 0: every VSS and every
                                  //    slice set at every level (ablation)
    int dir;                      // stage-1 direction: 0 push (Algorithm 5), 1 pull for dense levels, 2 pull
    const long long *rp;          // in-neighbour CSR of the (reordered) graph, for pulling
    const int *col;
    int *stamp;                   // per slice set: the level stage 2 last wrote its F elements
    unsigned long long budget_ns;
};

// per-CTA work counts of the current level: VSSs, hit words, dirty sets,
// pulled in-neighbour elements
struct MsAcc {
    unsigned long long vss, hitw, dirty, parcs;
};

// A level pulls (direction 1) when its queue holds more than 1/PULL_DIV of
// the VSSs.
constexpr long long PULL_DIV = 8;

// Staged level bytes: 0 .. LV8_FAR - 1 are levels, LV8_NONE is unreached,
// LV8_FAR a level >= LV8_FAR stored directly in the int32 output.
constexpr unsigned LV8_FAR = 0xFEu, LV8_NONE = 0xFFu;

// 0xFF in byte q of the result where bit q of the 4-bit x is set
__device__ __forceinline__ unsigned byte_mask4(unsigned x) {
    return ((x & 1u) ? 0xFFu : 0u) | ((x & 2u) ? 0xFF00u : 0u) | ((x & 4u) ? 0xFF0000u : 0u) |
           ((x & 8u) ? 0xFF000000u : 0u);
}

// The staged level bytes of the lanes in diff (word w of vertex u, reached
// at level ell); cur holds the lanes reached earlier, whose bytes stay.  A
// 4-lane group with no earlier lane is written as one word (new lanes ell,
// the others still unreached); otherwise byte by byte.
template <int KW>
__device__ __forceinline__ void lv8_store(const MsParams &P, int u, int w, unsigned diff, unsigned cur, int ell) {
    const unsigned val = ell < (int)LV8_FAR ? (unsigned)ell : LV8_FAR;
    const unsigned rep = val * 0x01010101u;
    unsigned char *row = P.lv8 + (size_t)u * (KW * 32) + (size_t)w * 32;
    if (cur == 0u) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            unsigned x[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const unsigned m = byte_mask4((diff >> (16 * h + 4 * j)) & 15u);
                x[j] = (rep & m) | ~m;
            }
            reinterpret_cast<uint4 *>(row)[h] = make_uint4(x[0], x[1], x[2], x[3]);
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const unsigned nb = (diff >> (4 * j)) & 15u;
        if (!nb) continue;
        if (((cur >> (4 * j)) & 15u) == 0u) {
            const unsigned m = byte_mask4(nb);
            reinterpret_cast<unsigned *>(row)[j] = (rep & m) | ~m;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if ((nb >> q) & 1u) row[4 * j + q] = (unsigned char)val;
        }
    }
}

__device__ __forceinline__ bool ms_barrier(MsCtl *ctl, unsigned &epoch, unsigned long long budget) {
    return grid_barrier(reinterpret_cast<Ctl *>(ctl), epoch, budget);
}

__device__ __forceinline__ int get_vi(int u, int rho) { return (u & 7) * rho + (u >> 3); }
// the bit-array element of vertex u: getVI, or u itself without reindexing
__device__ __forceinline__ int elem(const MsParams &P, int u) { return P.remap ? get_vi(u, P.rho) : u; }
// the slice set of an element index
__device__ __forceinline__ int elem_set(const MsParams &P, int e) { return P.remap ? e % P.rho : e >> 3; }

// Appends to the VSS queue and the dirty-set list are staged per warp in
// shared memory and reserved in the global arrays once per MS_STG entries
// (one atomic per warp and slice set on the same counter serialises in one
// L2 slice when a level touches hundreds of thousands of sets).
constexpr int MS_STG = 256;

struct MsStage {
    int *q, *d;   // staging areas of this warp: VSS ids, dirty slice-set ids
    int qn, dn;   // staged counts (warp-uniform)
};

__device__ __forceinline__ void ms_flush_q(const MsParams &P, MsStage &st, int *Q, int slot) {
    const int lane = lane_id();
    __syncwarp();
    if (st.qn) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&P.ctl->qlen[slot], st.qn);
        base = __shfl_sync(FULL_MASK, base, 0);
        for (int k = lane; k < st.qn; k += 32) Q[base + k] = st.q[k];
    }
    __syncwarp();
    st.qn = 0;
}

__device__ __forceinline__ void ms_flush_d(const MsParams &P, MsStage &st, int dl) {
    const int lane = lane_id();
    __syncwarp();
    if (st.dn) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&P.ctl->dlen[dl], st.dn);
        base = __shfl_sync(FULL_MASK, base, 0);
        for (int k = lane; k < st.dn; k += 32) P.dlist[dl][base + k] = st.d[k];
    }
    __syncwarp();
    st.dn = 0;
}

// The last flush of a stage, called by every thread of the CTA: warps add
// their staged counts in shared memory and one thread reserves the CTA's
// space in the global list (one atomic per CTA instead of per warp).
__device__ __forceinline__ void ms_block_flush(int *list, int *ctr, int *staged, int &n, int *s_tot) {
    const int lane = lane_id();
    int off = 0;
    if (lane == 0 && n) off = atomicAdd(&s_tot[0], n);
    off = __shfl_sync(FULL_MASK, off, 0);
    __syncthreads();
    if (threadIdx.x == 0) s_tot[1] = s_tot[0] ? atomicAdd(ctr, s_tot[0]) : 0;
    __syncthreads();
    const int base = s_tot[1] + off;
    for (int k = lane; k < n; k += 32) list[base + k] = staged[k];
    __syncwarp();
    n = 0;
}

// warp-aggregated append of one slice set per lane (its VSS range -> Q)
__device__ __forceinline__ void ms_enqueue(const MsParams &P, MsStage &st, bool want, int ss, int *Q, int slot) {
    const int lane = lane_id();
    if (!__any_sync(FULL_MASK, want)) return;
    int a = 0, len = 0;
    if (want) {
        a = __ldg(&P.realPtrs[ss]);
        len = __ldg(&P.realPtrs[ss + 1]) - a;
    }
    const int incl = warp_incl_scan(len);
    const int T = __shfl_sync(FULL_MASK, incl, 31);
    if (T <= MS_STG && st.qn + T > MS_STG) ms_flush_q(P, st, Q, slot);
    int *dst;
    int base;
    if (T > MS_STG) {      // larger than the staging area: reserve it directly
        int g = 0;
        if (lane == 31) g = atomicAdd(&P.ctl->qlen[slot], T);
        dst = Q + __shfl_sync(FULL_MASK, g, 31);
        base = incl - len;
    } else {
        dst = st.q;
        base = st.qn + incl - len;
        st.qn += T;
    }
    // short ranges by their own lane, long ones (hub slice sets) by the whole warp
    const bool big = len > 8;
    if (!big)
        for (int i = 0; i < len; ++i) dst[base + i] = a + i;
    unsigned lanes = __ballot_sync(FULL_MASK, big);
    while (lanes) {
        const int j = __ffs(lanes) - 1;
        lanes &= lanes - 1u;
        const int aj = __shfl_sync(FULL_MASK, a, j);
        const int lj = __shfl_sync(FULL_MASK, len, j);
        const int bj = __shfl_sync(FULL_MASK, base, j);
        for (int i = lane; i < lj; i += 32) dst[bj + i] = aj + i;
    }
    __syncwarp();
}

// warp-aggregated append of the dirty slice sets the lanes claimed
__device__ __forceinline__ void ms_mark_dirty(const MsParams &P, MsStage &st, bool claimed, int so, int dl) {
    const unsigned m = __ballot_sync(FULL_MASK, claimed);
    if (!m) return;
    const int cnt = __popc(m);
    if (st.dn + cnt > MS_STG) ms_flush_d(P, st, dl);
    if (claimed) st.d[st.dn + __popc(m & ((1u << lane_id()) - 1u))] = so;
    st.dn += cnt;
    __syncwarp();
}

// bit g = OR of the KW-bit field g of x (the 32/KW lane groups of a ballot)
template <int KW>
__device__ __forceinline__ unsigned group_bits(unsigned x) {
    if constexpr (KW == 32) {
        return x != 0u ? 1u : 0u;
    } else if constexpr (KW == 8) {
        x = (x | (x >> 4)) & 0x0F0F0F0Fu;
        x = (x | (x >> 2)) & 0x03030303u;
        x = (x | (x >> 1)) & 0x01010101u;           // bit 8g = any of byte g
        return (x * 0x01020408u) >> 24 & 0xFu;      // gather bits 0, 8, 16, 24 into 0..3
    } else {                                          // KW == 2: 16 pairs
        x = (x | (x >> 1)) & 0x55555555u;            // bit 2g = any of pair g
        x = (x | (x >> 1)) & 0x33333333u;
        x = (x | (x >> 2)) & 0x0F0F0F0Fu;
        x = (x | (x >> 4)) & 0x00FF00FFu;
        x = (x | (x >> 8)) & 0x0000FFFFu;
        return x;
    }
}

// Per-warp table of subset ORs of a slice set's frontier words: entry e < 16
// is the OR of the words of its vertices j < 4 with bit j of e set, entry
// 16 + e the same for vertices 4 + j.  Stored entry-major ([e][lane]), so a
// warp reading one entry per lane hits 32 distinct banks whatever entries
// the lanes pick.  A slot's hit word is then two loads and one OR instead of
// eight mask-selected ORs.
constexpr int MS_TAB = 32;
constexpr size_t MS_TAB_BYTES = (size_t)(MS_BLOCK / 32) * MS_TAB * 32 * sizeof(unsigned);

template <int KW>
__device__ void ms_stage1(const MsParams &P, MsStage &st, int *grab, int *s_tot, int qlen, const int *Qc, int dl,
                          int *s_rows, unsigned char *s_m, unsigned *s_tab, MsAcc *acc) {
    unsigned long long nvss = 0, nhit = 0;
    constexpr int G = 32 / KW;
    const int lane = lane_id();
    const int g = lane / KW, w = lane % KW;
    const int wib = threadIdx.x >> 5;
    int *rows = s_rows + wib * 128;
    unsigned char *m8s = s_m + wib * 128;
    unsigned *tab = s_tab + (size_t)wib * MS_TAB * 32 + lane;   // this lane's column
    // queue entries interleaved over the blocks, claimed by the block's warps
    for (;;) {
        int kc = 0;
        if (lane == 0) kc = atomicAdd(grab, 1);
        kc = __shfl_sync(FULL_MASK, kc, 0);
        const int it = (int)blockIdx.x + kc * (int)gridDim.x;
        if (it >= (P.track ? qlen : P.Nv)) break;
        const int vss = P.track ? Qc[it] : it;
        const int ss = __ldg(&P.v2r[vss]);
        ++nvss;
        const bool own = lane < P.lpv;
        const int4 r = own ? __ldg(reinterpret_cast<const int4 *>(P.rowIds) + (size_t)vss * P.lpv + lane)
                           : make_int4(0, 0, 0, 0);
        const unsigned m = own ? __ldg(&P.masks[(size_t)vss * P.lpv + lane]) : 0u;
        // slots past the last lane word with a slice are padding: the loop stops there
        const unsigned words = __ballot_sync(FULL_MASK, m != 0);
        const int nslots = words ? 4 * (32 - __clz(words)) : 0;
        __syncwarp();
        // slot 4l + i: the bit-array element index of its row (the slice set
        // of the row, for the dirty claims, is that index mod rho) and its
        // 8-bit slice mask (byte i of the lane word, little-endian)
        reinterpret_cast<int4 *>(rows)[lane] =
            make_int4(elem(P, r.x), elem(P, r.y), elem(P, r.z), elem(P, r.w));
        reinterpret_cast<unsigned *>(m8s)[lane] = m;
        const unsigned aw = P.track ? P.active[(size_t)ss * KW + w] : ~0u;
        unsigned f[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) f[j] = aw ? P.F[(size_t)elem(P, ss * 8 + j) * KW + w] : 0u;
        // each lane writes and reads only its own column: no warp sync needed
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            unsigned v[16];
            v[0] = 0u;
#pragma unroll
            for (int e = 1; e < 16; ++e) v[e] = v[e & (e - 1)] | f[4 * h + ((e & 1) ? 0 : (e & 2) ? 1 : (e & 4) ? 2 : 3)];
#pragma unroll
            for (int e = 0; e < 16; ++e) tab[(16 * h + e) * 32] = v[e];
        }
        __syncwarp();
        // slots with a hit (bit s of hm[s / 32]); their slice sets are marked
        // dirty after the loop, 32 slots at a time, so the loop never waits on
        // the dirty flags
        unsigned hm0 = 0, hm1 = 0, hm2 = 0, hm3 = 0;
        const int nt = (nslots + G - 1) / G;
        for (int c0 = 0; c0 < nslots; c0 += 32) {   // chunks of 32 slots (warp-uniform)
            unsigned hm = 0;
            const int t1 = min(nt, (c0 + 32) / G);
#pragma unroll 2
            for (int t = c0 / G; t < t1; ++t) {
                const int kk = t * G + g;
                const unsigned m8 = m8s[kk];
                const unsigned hit = tab[(m8 & 15u) * 32] | tab[(16u + (m8 >> 4)) * 32];
                if (hit) {
                    red_or(&P.Vn[(size_t)rows[kk] * KW + w], hit);
                    ++nhit;
                }
                // one bit per group (any of its KW lanes hit): slots t*G .. t*G+G-1,
                // G divides 32, so they sit in this chunk's word
                hm |= group_bits<KW>(__ballot_sync(FULL_MASK, hit != 0)) << ((t * G) & 31);
            }
            if (c0 == 0) hm0 = hm;
            else if (c0 == 32) hm1 = hm;
            else if (c0 == 64) hm2 = hm;
            else hm3 = hm;
        }
#pragma unroll
        for (int r4 = 0; r4 < 4; ++r4) {
            const unsigned hm = r4 == 0 ? hm0 : (r4 == 1 ? hm1 : (r4 == 2 ? hm2 : hm3));
            if (!hm || !P.track) continue;   // warp-uniform
            bool claimed = false;
            int so = 0;
            if (hm >> lane & 1u) {
                so = elem_set(P, rows[32 * r4 + lane]);
                claimed = ld_volatile_i32(&P.dirty[so]) == 0 && atomicExch(&P.dirty[so], 1) == 0;
            }
            ms_mark_dirty(P, st, claimed, so, dl);
        }
    }
    nhit = warp_sum(nhit);
    if (lane == 0) {
        atomicAdd(&acc->vss, nvss);
        atomicAdd(&acc->hitw, nhit);
    }
    ms_block_flush(P.dlist[dl], &P.ctl->dlen[dl], st.d, st.dn, s_tot);
}

template <int KW>
__device__ void ms_stage2(const MsParams &P, MsStage &st, int *grab, int *s_tot, int ell, int dl, int qn, int dcount,
                          int k, MsAcc *acc) {
    unsigned long long nd = 0, nact = 0;
    constexpr int G = 32 / KW;
    const int lane = lane_id();
    const int g = lane / KW, w = lane % KW;
    const int *dlist = P.dlist[dl];
    const int nchunk = (dcount + G - 1) / G;
    // chunks of G dirty sets interleaved over the blocks, claimed by the block's warps
    for (;;) {
        int kc = 0;
        if (lane == 0) kc = atomicAdd(grab, 1);
        kc = __shfl_sync(FULL_MASK, kc, 0);
        const int chunk = (int)blockIdx.x + kc * (int)gridDim.x;
        if (chunk >= nchunk) break;
        const int i = chunk * G + g;
        const bool valid = i < dcount;
        const int ss = valid ? (P.track ? dlist[i] : i) : 0;
        unsigned A = 0;
        // four vertices at a time: their V_next / V_curr words load together
#pragma unroll 1
        for (int j0 = 0; j0 < 8; j0 += 4) {
          unsigned nx4[4], cu4[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
              const int u = ss * 8 + j0 + q;
              nx4[q] = 0u;
              cu4[q] = 0u;
              if (valid && u < P.n) {
                  const size_t e = (size_t)elem(P, u) * KW + w;
                  nx4[q] = P.Vn[e];
                  cu4[q] = P.Vc[e];
              }
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int j = j0 + q;
            const int u = ss * 8 + j;
            unsigned diff = 0;
            if (valid && u < P.n) {
                const size_t e = (size_t)elem(P, u) * KW + w;
                const unsigned next = nx4[q];
                const unsigned cur = cu4[q];
                diff = next ^ cur;
                P.F[e] = diff;
                if (diff) {
                    P.Vc[e] = next;
                    A |= diff;
                    if (P.lv8) lv8_store<KW>(P, u, w, diff, cur, ell);
                    if (P.levels && (!P.lv8 || ell >= (int)LV8_FAR)) {
                        const int uo = P.old_of_new ? __ldg(&P.old_of_new[u]) : u;
                        unsigned d = diff;
                        while (d) {
                            const int b = __ffs(d) - 1;
                            d &= d - 1;
                            const int c = w * 32 + b;
                            if (c < k) P.levels[(size_t)c * P.n + uo] = ell;
                        }
                    }
                }
            }
            if (P.far) {
                int cnt = __popc(diff);
#pragma unroll
                for (int o = KW / 2; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULL_MASK, cnt, o, KW);
                if (w == 0 && cnt) {
                    P.far[u] += (long long)ell * cnt;
                    P.reach[u] += cnt;
                }
            }
          }
        }
        if (valid) {
            P.active[(size_t)ss * KW + w] = A;
        }
        const unsigned bal = __ballot_sync(FULL_MASK, A != 0);
        const bool any = ((bal >> (g * KW)) & (KW == 32 ? 0xFFFFFFFFu : ((1u << KW) - 1u))) != 0;
        if (valid && w == 0) {
            if (P.track) P.dirty[ss] = 0;
            P.stamp[ss] = ell;   // this set's F elements now hold level ell's frontier
            ++nd;
        }
        if (P.track) ms_enqueue(P, st, valid && w == 0 && any, ss, P.Q[qn], qn);
        else if (valid && w == 0 && any) ++nact;   // without tracking only the count ends the loop
    }
    nact = warp_sum(nact);
    if (lane_id() == 0 && nact) atomicAdd(&P.ctl->qlen[qn], (int)nact);
    nd = warp_sum(nd);
    if (lane_id() == 0 && nd) atomicAdd(&acc->dirty, nd);
    ms_block_flush(P.Q[qn], &P.ctl->qlen[qn], st.q, st.qn, s_tot);
}

// ------------------------------------------------------------------
// Stage 1 by pulling (direction-optimizing, for dense levels).  Pushing
// ORs each slot's hit word into V_next with an atomic; on a level where
// most slice sets are active those atomics bound the kernel.  Pulling
// visits every slice set instead (G = 32 / KW sets per warp, lane = word of
// the kappa-bit elements): each vertex with an unvisited lane ORs the
// frontier elements of its in-neighbours (rows sorted by descending
// neighbour degree, so hubs come first) until every unvisited lane is
// covered or the row ends, and writes its own V_next word without an
// atomic.  F is rewritten only for the slice sets stage 2 finalises, so an
// in-neighbour's element counts only when its set's stamp is the previous
// level.  A set that gained a lane is appended to the dirty list; stage 2
// then runs unchanged.  The lanes reached are exactly those a push would
// add (Eq. 2 over the same slices, read by row instead of by column).
template <int KW>
__device__ void ms_stage1_pull(const MsParams &P, MsStage &st, int *grab, int *s_tot, int ell, int dl, int k,
                               MsAcc *acc) {
    constexpr int G = 32 / KW;
    constexpr unsigned GMASK = KW == 32 ? 0xFFFFFFFFu : ((1u << KW) - 1u);
    const int lane = lane_id();
    const int g = lane / KW, w = lane % KW;
    // lanes of word w that carry a source (bits of lanes >= k never get set)
    const int lo = w * 32;
    const unsigned lanes_w = lo + 32 <= k ? 0xFFFFFFFFu : (lo >= k ? 0u : ((1u << (k - lo)) - 1u));
    unsigned long long nd = 0, arcs = 0;
    const int nchunk = (P.rho + G - 1) / G;
    for (;;) {
        int kc = 0;
        if (lane == 0) kc = atomicAdd(grab, 1);
        kc = __shfl_sync(FULL_MASK, kc, 0);
        const int chunk = (int)blockIdx.x + kc * (int)gridDim.x;
        if (chunk >= nchunk) break;
        const int ss = chunk * G + g;
        const bool valid = ss < P.rho;
        bool changed = false;
#pragma unroll 1
        for (int j = 0; j < 8; ++j) {
            const int u = ss * 8 + j;
            const bool ok = valid && u < P.n;
            const size_t e = ok ? (size_t)elem(P, u) * KW + w : 0;
            const unsigned vis = ok ? P.Vc[e] : 0u;
            const unsigned unv = ok ? (~vis & lanes_w) : 0u;
            long long p = ok ? __ldg(&P.rp[u]) : 0;
            const long long pe = ok ? __ldg(&P.rp[u + 1]) : 0;
            unsigned acc_w = 0;
            // the group keeps pulling while it has an unvisited lane not yet reached
            bool live = ((__ballot_sync(FULL_MASK, unv != 0u) >> (g * KW)) & GMASK) != 0u && p < pe;
            while (__any_sync(FULL_MASK, live)) {
                // four in-neighbours a step, their stamps and elements loaded together
                int v4[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) v4[q] = (live && p + q < pe) ? __ldg(&P.col[p + q]) : -1;
                int t4[4];
                unsigned f4[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    t4[q] = v4[q] >= 0 ? P.stamp[v4[q] >> 3] : -1;
                    f4[q] = v4[q] >= 0 ? P.F[(size_t)elem(P, v4[q]) * KW + w] : 0u;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (t4[q] == ell - 1) acc_w |= f4[q];
                    if (v4[q] >= 0 && w == 0) ++arcs;
                }
                p += 4;
                const unsigned open = __ballot_sync(FULL_MASK, (unv & ~acc_w) != 0u);
                live = live && p < pe && ((open >> (g * KW)) & GMASK) != 0u;
            }
            const unsigned nw = acc_w & unv;
            if (nw) {
                P.Vn[e] = vis | nw;   // V_next = V_curr before this stage: the owner writes it alone
                changed = true;
            }
        }
        // the group's set gained a lane: append it to the dirty list (lane w = 0)
        const bool any = ((__ballot_sync(FULL_MASK, changed) >> (g * KW)) & GMASK) != 0u;
        if (valid && w == 0 && any) P.dirty[ss] = 1;
        ms_mark_dirty(P, st, valid && w == 0 && any, ss, dl);
    }
    arcs = warp_sum(arcs);
    if (lane == 0 && arcs) atomicAdd(&acc->parcs, arcs);
    ms_block_flush(P.dlist[dl], &P.ctl->dlen[dl], st.d, st.dn, s_tot);
    (void)nd;
}

// ------------------------------------------------------------------
// Stage 1 on the tensor cores (tcgen05), for the tau = 128 layout.
// Eq. 2 for kappa lanes at once is a 0/1 product: hits[lane j][slot s] =
// sum over the slice set's columns c of F[c](bit j) * mask[s](bit c), and a
// lane reaches a slot's row iff its sum is nonzero.  Each warpgroup (4
// warps) takes one VSS: B = its 128 slots x K (the 8 mask bits as bf16
// 0/1, K padded to 16 with zeros), and for every 128-lane tile of the
// frontier whose active words are nonzero, A = 128 lanes x K (bit j of the
// 8 frontier elements as bf16 0/1); one kind::f16 MMA per 64 slots writes
// D = A B^T (128 lanes x 64 slots, fp32, exact: sums <= 8) to tensor
// memory.  Warp w of the group reads lanes 32w .. 32w + 31 of D; a ballot
// over its 32 threads of D[.][s] != 0 is the hit word of those lanes for
// slot s, OR-ed into V_next like the CUDA-core path's.  kind::i8 does not
// exist on sm_103a; bf16 0/1 operands with fp32 sums are exact.
constexpr int TC_WG = MS_BLOCK / 128;                 // warpgroups per CTA
constexpr int TC_N = 64;                              // slots per MMA = D columns per warpgroup
constexpr uint32_t TC_COLS = TC_WG * TC_N;            // tensor-memory columns per CTA (2 CTAs / SM: 512)
constexpr size_t TC_TILE_BYTES = 128 * 16 * 2;        // 128 rows x 16 bf16
constexpr size_t TC_SMEM = (size_t)TC_WG * 2 * TC_TILE_BYTES;
// per warpgroup: halves [0, 4), tile activity [4, 12) (double-buffered by
// tile parity: a warp past a tile with no MMA may write the next tile's
// flag before a slower warp has read this one), wait ok [12]
constexpr int TC_FLAGS = 13;

// byte offset of row r (K-group 0) in a no-swizzle K-major tile: 8-row core
// groups 256 bytes apart (SBO), the two K-groups of 8 bf16 128 bytes apart
// (LBO), rows of a core group 16 bytes apart
__device__ __forceinline__ uint32_t tc_row_off(int r) { return (uint32_t)((r >> 3) * 256 + (r & 7) * 16); }

struct TcState {
    uint32_t tmem;          // the CTA's tensor-memory base
    unsigned char *tiles;   // A and B tiles of each warpgroup
    uint64_t *mbar;         // MMA completion barrier of each warpgroup
    int *flags;             // TC_FLAGS ints per warpgroup
    int *claim;             // the claimed queue position of each warpgroup
};

template <int KW>
__device__ void ms_stage1_tc(const MsParams &P, MsStage &st, int *grab, int *s_tot, int qlen, const int *Qc, int dl,
                             int *s_rows, unsigned char *s_m, const TcState &tc, uint32_t &phase, MsAcc *acc) {
    constexpr int NT = (KW + 3) / 4;   // 128-lane tiles of the kappa lanes
    const int lane = lane_id();
    const int wib = threadIdx.x >> 5;
    const int g = wib >> 2, q = wib & 3;
    const int t = threadIdx.x & 127;
    const int bar = 1 + g;             // named barrier of the warpgroup (0 is __syncthreads)
    int *rows = s_rows + g * 128;
    unsigned char *hmk = s_m + g * 128;   // slot s had a hit in some tile
    unsigned char *A = tc.tiles + (size_t)g * 2 * TC_TILE_BYTES;
    unsigned char *B = A + TC_TILE_BYTES;
    uint64_t *mbar = tc.mbar + g;
    int *fl = tc.flags + g * TC_FLAGS;
    const uint32_t dcol = tc.tmem + (uint32_t)(g * TC_N);
    constexpr uint32_t IDESC = idesc_bf16_f32(128, TC_N);
    const uint64_t adesc = smem_desc_kmajor(A, 128, 256);
    unsigned long long nvss = 0, nhit = 0;
    bool bad = false;
    for (;;) {
        if (t == 0) tc.claim[g] = atomicAdd(grab, 1);
        named_barrier(bar, 128);
        const int it = (int)blockIdx.x + tc.claim[g] * (int)gridDim.x;
        if (it >= qlen) break;   // uniform in the warpgroup
        const int vss = Qc[it];
        const int ss = __ldg(&P.v2r[vss]);
        if (t == 0) ++nvss;
        // slot t: its row and mask byte (lane word t / 4 of the VSS, byte t % 4)
        const int r = __ldg(&P.rowIds[(size_t)vss * 128 + t]);
        const unsigned m8 = (__ldg(&P.masks[(size_t)vss * 32 + (t >> 2)]) >> (8 * (t & 3))) & 0xFFu;
        rows[t] = elem(P, r);
        hmk[t] = 0;
        *reinterpret_cast<uint4 *>(B + tc_row_off(t)) = bits_to_bf16x8(m8);
        const unsigned anym = __ballot_sync(FULL_MASK, m8 != 0u);
        if (lane == 0) fl[q] = anym != 0u;
        fence_proxy_async_smem();
        named_barrier(bar, 128);
        const bool half0 = (fl[0] | fl[1]) != 0, half1 = (fl[2] | fl[3]) != 0;   // slots 0-63 / 64-127
        for (int m = 0; m < NT && !bad; ++m) {
            const int w = m * 4 + q;   // this warp's 32-lane word of the tile
            const unsigned aw = w < KW ? P.active[(size_t)ss * KW + w] : 0u;
            unsigned bits = 0;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const unsigned f = aw ? P.F[(size_t)elem(P, ss * 8 + c) * KW + w] : 0u;
                bits |= ((f >> lane) & 1u) << c;
            }
            *reinterpret_cast<uint4 *>(A + tc_row_off(t)) = bits_to_bf16x8(bits);
            int *tf = fl + 4 + 4 * (m & 1);
            if (lane == 0) tf[q] = aw != 0u;
            fence_proxy_async_smem();
            tc_fence_before();
            named_barrier(bar, 128);
            const bool tile_on = (tf[0] | tf[1] | tf[2] | tf[3]) != 0;
            if (!tile_on) continue;   // uniform: no frontier lane of the tile
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                if (!(h ? half1 : half0)) continue;   // uniform: padding slots only
                if (t == 0) {
                    tc_fence_after();
                    mma_bf16_commit(dcol, adesc, smem_desc_kmajor(B + h * 2048, 128, 256), IDESC, mbar);
                    // bounded wait: a wait past the budget records a timeout, then waits
                    // once more (bounded) so no MMA is left writing the tensor memory
                    const uint64_t t0 = global_ns();
                    int ok = 1;
                    unsigned spins = 0;
                    while (!mbar_try_wait(mbar, phase)) {
                        if ((++spins & 255u) == 0 && global_ns() - t0 > P.budget_ns) {
                            ok = 0;
                            const uint64_t t1 = global_ns();
                            while (!mbar_try_wait(mbar, phase) && global_ns() - t1 < P.budget_ns) {
                            }
                            break;
                        }
                    }
                    fl[12] = ok;
                }
                named_barrier(bar, 128);
                phase ^= 1u;
                if (!fl[12]) {
                    if (t == 0) atomicCAS(&P.ctl->err, 0, (int)BLEST_ERR_TIMEOUT);
                    bad = true;
                    break;
                }
                tc_fence_after();
                if (w < KW) {   // warp-uniform: the warp's lanes exist
#pragma unroll 1
                    for (int cc = 0; cc < 2; ++cc) {
                        uint32_t d[32];
                        tmem_ld32(dcol + ((uint32_t)(32 * q) << 16) + (uint32_t)(cc * 32), d);
                        unsigned hw = 0;
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            const unsigned b = __ballot_sync(FULL_MASK, d[i] != 0u);
                            if (lane == i) hw = b;
                        }
                        const int sl = h * 64 + cc * 32 + lane;
                        if (hw) {
                            red_or(&P.Vn[(size_t)rows[sl] * KW + w], hw);
                            ++nhit;
                            hmk[sl] = 1;
                        }
                    }
                }
                tc_fence_before();
                named_barrier(bar, 128);   // D read by every warp before the next MMA
            }
        }
        if (bad) break;
        named_barrier(bar, 128);   // the hit marks of every tile
        bool claimed = false;
        int so = 0;
        if (hmk[t]) {
            so = elem_set(P, rows[t]);
            claimed = ld_volatile_i32(&P.dirty[so]) == 0 && atomicExch(&P.dirty[so], 1) == 0;
        }
        ms_mark_dirty(P, st, claimed, so, dl);
        named_barrier(bar, 128);   // rows, marks and B are rewritten by the next VSS
    }
    nhit = warp_sum(nhit);
    if (lane == 0) {
        atomicAdd(&acc->vss, nvss);
        atomicAdd(&acc->hitw, nhit);
    }
    ms_block_flush(P.dlist[dl], &P.ctl->dlen[dl], st.d, st.dn, s_tot);
}

// Staged levels -> the source-major int32 output: a warp takes 32 lanes x
// 32 vertices (original ids), each thread one vertex's 32 bytes, and writes
// 32 rows of 128 contiguous bytes.  Out of line: it runs once per launch,
// and inlined it would take registers from the level loop.
template <int KW>
__device__ __noinline__ void lv8_transpose(const unsigned char *lv8, int *levels, const int *new_of_old, int n, int k,
                                           size_t tid, size_t nthreads) {
    const int ntc = (k + 31) >> 5;
    const long long tiles = (long long)((n + 31) >> 5) * ntc;
    const int lane = lane_id();
    for (long long t = (long long)(tid >> 5); t < tiles; t += (long long)(nthreads >> 5)) {
        const int tcol = (int)(t % ntc);
        const int uo = (int)(t / ntc) * 32 + lane;
        if (uo >= n) continue;
        const int u = new_of_old ? __ldg(&new_of_old[uo]) : uo;
        const uint4 *src = reinterpret_cast<const uint4 *>(lv8 + (size_t)u * (KW * 32) + (size_t)tcol * 32);
        const uint4 a = __ldcg(src), b = __ldcg(src + 1);
        const unsigned x[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        int *o = levels + (size_t)tcol * 32 * (size_t)n + uo;
        const int cmax = min(32, k - tcol * 32);
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            const unsigned v = (x[c >> 2] >> ((c & 3) * 8)) & 0xFFu;
            if (c < cmax && v != LV8_FAR) o[(size_t)c * n] = v == LV8_NONE ? -1 : (int)v;
        }
    }
}

// The whole multi-source BFS of one launch (every block calls it; a block
// returns early only at a grid barrier that failed, all its threads
// together).  tc: the tensor-core stage 1 (its tensor memory is allocated
// by the caller); else the CUDA-core stage 1 with the subset-OR tables in
// s_tab.
template <int KW, bool TC>
__device__ __forceinline__ void ms_run(MsParams P, unsigned *s_tab, const TcState *tc) {
    __shared__ __align__(16) int s_rows[(MS_BLOCK / 32) * 128];
    __shared__ __align__(16) unsigned char s_m[(MS_BLOCK / 32) * 128];
    __shared__ int s_stg[(MS_BLOCK / 32) * 2 * MS_STG];
    __shared__ int s_grab[2];
    __shared__ int s_tot[2][2];   // per stage: the CTA's staged total and its reserved base
    __shared__ MsAcc s_acc;       // this CTA's work counts of the current level
    MsStage st;
    st.q = s_stg + (threadIdx.x >> 5) * 2 * MS_STG;
    st.d = st.q + MS_STG;
    st.qn = 0;
    st.dn = 0;
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nthreads = (size_t)gridDim.x * blockDim.x;
    MsCtl *ctl = P.ctl;
    unsigned epoch = 0;
    const int k = P.k_dev ? *P.k_dev : P.k;

    // ---- init: zero the bit arrays and flags, -1 levels for the k lanes
    const size_t words = (size_t)P.rho * 8 * KW;
    for (size_t i = tid; i < words; i += nthreads) {
        P.F[i] = 0u;
        P.Vc[i] = 0u;
        P.Vn[i] = 0u;
    }
    for (size_t i = tid; i < (size_t)P.rho * KW; i += nthreads) P.active[i] = 0u;
    for (size_t i = tid; i < (size_t)P.rho; i += nthreads) {
        P.dirty[i] = 0;
        P.stamp[i] = -1;
    }
    if (P.lv8) {
        uint4 *l8 = reinterpret_cast<uint4 *>(P.lv8);
        const uint4 none = make_uint4(~0u, ~0u, ~0u, ~0u);
        for (size_t i = tid; i < (size_t)P.rho * KW * 16; i += nthreads) l8[i] = none;
    } else if (P.levels) {
        for (size_t i = tid; i < (size_t)k * P.n; i += nthreads) P.levels[i] = -1;
    }
    if (!ms_barrier(ctl, epoch, P.budget_ns)) return;
    // ---- sources: lane c starts at srcs[c]
    if (tid < (size_t)k) {
        const int c = (int)tid;
        const int so = __ldg(&P.srcs[c]);
        const int u = P.new_of_old ? __ldg(&P.new_of_old[so]) : so;
        const size_t e = (size_t)elem(P, u) * KW + (c >> 5);
        const unsigned bit = 1u << (c & 31);
        atomicOr(&P.Vc[e], bit);
        atomicOr(&P.Vn[e], bit);
        atomicOr(&P.F[e], bit);
        atomicOr(&P.active[(size_t)(u >> 3) * KW + (c >> 5)], bit);
        if (P.lv8) P.lv8[(size_t)u * (KW * 32) + c] = 0;
        else if (P.levels) P.levels[(size_t)c * P.n + so] = 0;
        if (P.reach) atomicAdd((unsigned long long *)&P.reach[u], 1ull);
        P.stamp[u >> 3] = 0;   // the sources' F elements hold level 0
        if (atomicExch(&P.dirty[u >> 3], 1) == 0) P.dlist[1][atomicAdd(&ctl->dlen[1], 1)] = u >> 3;
    }
    if (!ms_barrier(ctl, epoch, P.budget_ns)) return;
    {
        // enqueue the source slice sets and clear their flags
        __shared__ int s_c0;
        if (threadIdx.x == 0) s_c0 = ld_volatile_i32(&ctl->dlen[1]);
        __syncthreads();
        const int cnt = s_c0;
        const int gwarp = (int)(tid >> 5), nwarps = (int)(nthreads >> 5);
        for (int b = gwarp * 32; b < cnt; b += nwarps * 32) {
            const int i = b + lane_id();
            const bool ok = i < cnt;
            const int ss = ok ? P.dlist[1][i] : 0;
            if (ok) P.dirty[ss] = 0;
            ms_enqueue(P, st, ok, ss, P.Q[0], 0);
        }
        ms_flush_q(P, st, P.Q[0], 0);
    }
    if (!ms_barrier(ctl, epoch, P.budget_ns)) return;
    if (tid == 0) ctl->dlen[1] = 0;
    if (!ms_barrier(ctl, epoch, P.budget_ns)) return;

    int ell = 1;
    uint32_t tc_phase = 0;   // parity of the warpgroup's next MMA completion (tensor-core stage 1)
    __shared__ int s_cnt;
    for (;; ++ell) {
        const int qc = (ell - 1) & 1, qn = ell & 1, dl = ell & 1;
        // one thread per block reads the shared counter (see k_bfs)
        if (threadIdx.x == 0) {
            // the previous level's counts of this CTA (all warps passed two
            // block barriers since they added them)
            if (P.stats && ell > 1 && (s_acc.vss | s_acc.hitw | s_acc.dirty | s_acc.parcs) != 0) {
                red_add_u64(&P.stats->vss, s_acc.vss);
                red_add_u64(&P.stats->hit_words, s_acc.hitw);
                red_add_u64(&P.stats->dirty_sets, s_acc.dirty);
                red_add_u64(&P.stats->pull_arcs, s_acc.parcs);
            }
            s_acc.vss = 0;
            s_acc.hitw = 0;
            s_acc.dirty = 0;
            s_acc.parcs = 0;
            s_cnt = ld_volatile_i32(&ctl->qlen[qc]);
            s_grab[0] = 0;
            s_grab[1] = 0;
            s_tot[0][0] = 0;
            s_tot[1][0] = 0;
        }
        __syncthreads();
        const int qlen = s_cnt;
        __syncthreads();
        if (qlen == 0) break;
        if (tid == 0) ctl->qlen[qn] = 0;
        // the level's direction, the same in every block (qlen is the level's count)
        const bool pull = P.dir == 2 || (P.dir == 1 && (long long)qlen * PULL_DIV > (long long)P.Nv);
        if (pull) {
            if (tid == 0 && P.stats) red_add_u64(&P.stats->pull_levels, 1ull);
            ms_stage1_pull<KW>(P, st, &s_grab[0], s_tot[0], ell, dl, k, &s_acc);
        } else if constexpr (TC) {
            ms_stage1_tc<KW>(P, st, &s_grab[0], s_tot[0], qlen, P.Q[qc], dl, s_rows, s_m, *tc, tc_phase, &s_acc);
        } else {
            ms_stage1<KW>(P, st, &s_grab[0], s_tot[0], qlen, P.Q[qc], dl, s_rows, s_m, s_tab, &s_acc);
        }
        if (!ms_barrier(ctl, epoch, P.budget_ns)) return;
        if (threadIdx.x == 0) s_cnt = P.track ? ld_volatile_i32(&ctl->dlen[dl]) : P.rho;
        __syncthreads();
        const int dcount = s_cnt;
        __syncthreads();
        if (tid == 0) ctl->dlen[dl ^ 1] = 0;
        ms_stage2<KW>(P, st, &s_grab[1], s_tot[1], ell, dl, qn, dcount, k, &s_acc);
        if (!ms_barrier(ctl, epoch, P.budget_ns)) return;
    }
    // ---- staged levels -> source-major int32 (the last level's stage 2
    // ended at a grid barrier, so every byte is in place)
    if (P.lv8) lv8_transpose<KW>(P.lv8, P.levels, P.new_of_old, P.n, k, tid, nthreads);
    if (tid == 0) {
        ctl->nlevels = ell - 1;
        if (P.stats) {
            red_add_u64(&P.stats->launches, 1ull);
            red_add_u64(&P.stats->levels, (unsigned long long)(ell - 1));
        }
    }
}

// two 512-thread CTAs per SM (64 registers a thread)
template <int KW>
__global__ void __launch_bounds__(MS_BLOCK, 2) k_msbfs(MsParams P) {
    extern __shared__ unsigned s_tab[];   // MS_TAB_BYTES: the warps' subset-OR tables
    ms_run<KW, false>(P, s_tab, nullptr);
}

// The tensor-core variant: TC_COLS tensor-memory columns per CTA (two CTAs
// per SM fill the 512 columns), allocated before and freed after the run,
// whichever barrier it ended at.
template <int KW>
__global__ void __launch_bounds__(MS_BLOCK, 2) k_msbfs_tc(MsParams P) {
    extern __shared__ __align__(1024) unsigned char s_tiles[];   // TC_SMEM: A / B tiles
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar[TC_WG];
    __shared__ int s_flags[TC_WG * TC_FLAGS];
    __shared__ int s_claim[TC_WG];
    if (threadIdx.x < 32) tmem_alloc(&s_tmem, TC_COLS);
    if (threadIdx.x == 0) {
        for (int g = 0; g < TC_WG; ++g) mbar_init(&s_mbar[g], 1);
        mbar_init_fence();
    }
    // the K-padding half of every tile row stays zero
    for (size_t i = threadIdx.x; i < TC_SMEM / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(s_tiles)[i] = make_uint4(0u, 0u, 0u, 0u);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    TcState tc;
    tc.tmem = s_tmem;
    tc.tiles = s_tiles;
    tc.mbar = s_mbar;
    tc.flags = s_flags;
    tc.claim = s_claim;
    ms_run<KW, true>(P, nullptr, &tc);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(s_tmem, TC_COLS);
}

__global__ void k_cc(const long long *__restrict__ far, const long long *__restrict__ reach,
                     const int *__restrict__ new_of_old, int n, long long *far_out, double *cc_out,
                     long long *reach_out) {
    const int stride = gridDim.x * blockDim.x;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int u = new_of_old ? new_of_old[v] : v;
        const long long f = far[u], r = reach[u];
        if (far_out) far_out[v] = f;
        if (reach_out) reach_out[v] = r;
        if (cc_out) cc_out[v] = f > 0 ? (double)(r - 1) / (double)f : 0.0;   // Eq. 7, component-normalised
    }
}

// the kernel of a (lane words, engine) pair and its dynamic shared memory
static const void *ms_kernel(int KW, bool tc) {
    if (tc) return KW == 2 ? (const void *)k_msbfs_tc<2> : (KW == 8 ? (const void *)k_msbfs_tc<8> : (const void *)k_msbfs_tc<32>);
    return KW == 2 ? (const void *)k_msbfs<2> : (KW == 8 ? (const void *)k_msbfs<8> : (const void *)k_msbfs<32>);
}
static size_t ms_smem(bool tc) { return tc ? TC_SMEM : MS_TAB_BYTES; }

// Co-resident grid of a kernel; 0 if it cannot be launched.  The
// tensor-core kernel needs at most two CTAs per SM (each holds TC_COLS of
// the SM's 512 tensor-memory columns; a third would wait for columns
// forever), so a larger occupancy refuses it.
static int ms_grid(int KW, bool tc) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void *fn = ms_kernel(KW, tc);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ms_smem(tc)) != cudaSuccess)
        return 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, MS_BLOCK, ms_smem(tc));
    if (tc && per * (int)TC_COLS > 512) return 0;
    return per * sms;
}

}  // namespace

// the next batch of a closeness range: source ids cursor[0] .. up to 1024
__global__ void k_ms_batch_src(int *d_src, int *k_dev, const long long *cursor) {
    const long long b = cursor[0], e = cursor[1];
    const int k = (int)((e - b) < 1024 ? (e - b) : 1024);
    if (threadIdx.x == 0) *k_dev = k;
    for (int c = threadIdx.x; c < k; c += blockDim.x) d_src[c] = (int)(b + c);
}

// after a batch: advance the cursor, keep the first device error
__global__ void k_ms_batch_next(long long *cursor, const MsCtl *ctl, int *sticky) {
    cursor[0] += 1024;
    if (ctl->err && *sticky == 0) *sticky = ctl->err;
}

static void ms_release_graph(MsbfsWork *m) {
    if (m->cc_exec) cudaGraphExecDestroy(m->cc_exec);
    if (m->cc_graph) cudaGraphDestroy(m->cc_graph);
    m->cc_exec = nullptr;
    m->cc_graph = nullptr;
}

void msbfs_release(blest_graph *h) {
    if (h->ms) {
        if (h->ms->h_ctl) cudaFreeHost(h->ms->h_ctl);
        ms_release_graph(h->ms);
        delete h->ms;
        h->ms = nullptr;
    }
}

static blest_status ms_prepare(blest_graph *h, int kappa) {
    if (h->ms && h->ms->kappa >= kappa) return BLEST_OK;
    if (h->ms && h->ms->kappa < kappa) {
        // grow: the old arrays stay owned by the handle (freed at destroy)
        if (h->ms->h_ctl) cudaFreeHost(h->ms->h_ctl);
        ms_release_graph(h->ms);
        delete h->ms;
        h->ms = nullptr;
    }
    MsbfsWork *m = new MsbfsWork();
    m->kappa = kappa;
    m->KW = kappa / 32;
    const size_t rho = (size_t)h->Ns;
    const size_t words = rho * 8 * (size_t)m->KW;
    blest_status st;
    if ((st = dev_alloc_t(h, &m->F, words)) != BLEST_OK) { delete m; return st; }
    if ((st = dev_alloc_t(h, &m->Vc, words)) != BLEST_OK) { delete m; return st; }
    if ((st = dev_alloc_t(h, &m->Vn, words)) != BLEST_OK) { delete m; return st; }
    if ((st = dev_alloc_t(h, &m->active, rho * m->KW)) != BLEST_OK) { delete m; return st; }
    if ((st = dev_alloc_t(h, &m->dirty, rho)) != BLEST_OK) { delete m; return st; }
    for (int i = 0; i < 2; ++i) {
        if ((st = dev_alloc_t(h, &m->dlist[i], rho + 1)) != BLEST_OK) { delete m; return st; }
        if ((st = dev_alloc_t(h, &m->Q[i], (size_t)(h->Nv > 0 ? h->Nv : 1))) != BLEST_OK) { delete m; return st; }
    }
    if ((st = dev_alloc_t(h, &m->ctl, 1)) != BLEST_OK) { delete m; return st; }
    if ((st = dev_alloc_t(h, &m->d_src, 1024)) != BLEST_OK) { delete m; return st; }
    if ((st = dev_alloc_t(h, &m->stats, 1)) != BLEST_OK) { delete m; return st; }
    if ((st = dev_alloc_t(h, &m->stamp, rho + 1)) != BLEST_OK) { delete m; return st; }
    if (cudaMemsetAsync(m->stats, 0, sizeof(MsStats), h->stream) != cudaSuccess) { delete m; return BLEST_ERR_CUDA; }
    if (cudaMallocHost((void **)&m->h_ctl, sizeof(MsCtl)) != cudaSuccess) { delete m; return BLEST_ERR_OOM; }
    m->grid = ms_grid(m->KW, false);
    if (m->grid <= 0) { delete m; return BLEST_ERR_CUDA; }
    h->ms = m;
    return BLEST_OK;
}

// One multi-source launch over k <= kappa sources already on the device
// (k_dev non-null: the batch size is read from the device at launch).
static blest_status ms_launch(blest_graph *h, int k, int *levels_dev, long long *far, long long *reach,
                              const int *k_dev = nullptr) {
    MsbfsWork *m = h->ms;
    MsParams P;
    memset(&P, 0, sizeof P);
    P.n = (int)h->n;
    P.rho = (int)h->Ns;
    P.k = k;
    P.lpv = h->tau / 4;
    P.rowIds = h->g.rowIds;
    P.masks = h->g.masks;
    P.realPtrs = h->g.realPtrs;
    P.v2r = h->g.v2r;
    P.F = m->F;
    P.Vc = m->Vc;
    P.Vn = m->Vn;
    P.active = m->active;
    P.dirty = m->dirty;
    P.dlist[0] = m->dlist[0];
    P.dlist[1] = m->dlist[1];
    P.Q[0] = m->Q[0];
    P.Q[1] = m->Q[1];
    P.ctl = m->ctl;
    P.srcs = m->d_src;
    P.new_of_old = h->g.new_of_old;
    P.old_of_new = h->g.old_of_new;
    P.k_dev = k_dev;
    P.levels = levels_dev;
    P.lv8 = (levels_dev && h->ms_out) ? m->lv8 : nullptr;
    P.far = far;
    P.reach = reach;
    P.stats = m->stats;
    P.Nv = (int)h->Nv;
    P.remap = h->ms_remap;
    P.track = h->ms_track;
    P.dir = h->ms_dir;
    P.rp = h->g.rp;
    P.col = h->g.col;
    P.stamp = m->stamp;
    P.budget_ns = (unsigned long long)h->timeout_ms * 1000000ull;
    if (cudaMemsetAsync(m->ctl, 0, sizeof(MsCtl), h->stream) != cudaSuccess) return BLEST_ERR_CUDA;
    void *args[] = {&P};
    const bool tc = h->ms_engine == 1;
    if (tc && m->grid_tc < 0) m->grid_tc = ms_grid(m->KW, true);
    const int grid = tc ? m->grid_tc : m->grid;
    if (grid <= 0) return BLEST_ERR_UNSUPPORTED;
    cudaError_t e = cudaLaunchCooperativeKernel(ms_kernel(m->KW, tc), dim3(grid), dim3(MS_BLOCK), args, ms_smem(tc),
                                                h->stream);
    if (e != cudaSuccess) {
        blest_internal_record_cuda_error(e, "cudaLaunchCooperativeKernel(k_msbfs)", __FILE__, __LINE__);
        return BLEST_ERR_CUDA;
    }
    return BLEST_OK;
}

static blest_status ms_finish(blest_graph *h, bool sync) {
    MsbfsWork *m = h->ms;
    if (cudaMemcpyAsync(m->h_ctl, m->ctl, sizeof(MsCtl), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return BLEST_ERR_CUDA;
    if (!sync) return BLEST_OK;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return BLEST_ERR_CUDA;
    if (m->h_ctl->err) return (blest_status)m->h_ctl->err;
    return BLEST_OK;
}

static int kappa_for(int k) { return k <= 64 ? 64 : (k <= 256 ? 256 : 1024); }

extern "C" blest_status blest_msbfs(blest_handle h, const int32_t *sources, int32_t k, int32_t *levels) {
    if (!h || h->many || !sources || !levels || k < 1 || k > 1024) return BLEST_ERR_INVALID;
    if (h->sigma != 8) return BLEST_ERR_UNSUPPORTED;   // getVI groups the 8 vertices of a slice set
    std::vector<int32_t> src((size_t)k);
    if (cudaMemcpy(src.data(), sources, (size_t)k * 4, cudaMemcpyDefault) != cudaSuccess) return BLEST_ERR_CUDA;
    for (int32_t s : src)
        if (s < 0 || (int64_t)s >= h->n) return BLEST_ERR_INVALID;
    blest_status st = ms_prepare(h, kappa_for(k));
    if (st != BLEST_OK) return st;
    if (h->ms_out && !h->ms->lv8 &&
        (st = dev_alloc_t(h, &h->ms->lv8, (size_t)h->Ns * 8 * (size_t)h->ms->kappa)) != BLEST_OK)
        return st;
    const bool dev = is_device_ptr(levels);
    int32_t *target = levels;
    if (!dev) {
        void *p = nullptr;
        if (cudaMallocAsync(&p, (size_t)k * (size_t)h->n * 4, h->stream) != cudaSuccess) return BLEST_ERR_OOM;
        target = (int32_t *)p;
    }
    if (cudaMemcpyAsync(h->ms->d_src, src.data(), (size_t)k * 4, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        return BLEST_ERR_CUDA;
    if (cudaMemsetAsync(h->ms->stats, 0, sizeof(MsStats), h->stream) != cudaSuccess) return BLEST_ERR_CUDA;
    st = ms_launch(h, k, target, nullptr, nullptr);
    if (st == BLEST_OK && !dev) {
        if (cudaMemcpyAsync(levels, target, (size_t)k * (size_t)h->n * 4, cudaMemcpyDeviceToHost, h->stream) !=
            cudaSuccess)
            st = BLEST_ERR_CUDA;
        cudaFreeAsync(target, h->stream);
    }
    if (st != BLEST_OK) return st;
    return ms_finish(h, !dev || !h->async);
}

// Distance sums from the sources [first, first + count) (original ids),
// accumulated into the handle's device accumulators.
// Closeness over sources [first, first + count): 1024-source batches, each
// one replay of a CUDA graph holding the source-id kernel, the control-block
// reset, the persistent multi-source kernel and the cursor advance; one
// host synchronisation for the whole range.
static blest_status closeness_batches(blest_graph *h, int64_t first, int64_t count) {
    blest_status st = ms_prepare(h, 1024);
    if (st != BLEST_OK) return st;
    MsbfsWork *m = h->ms;
    if (count <= 0) return BLEST_OK;
    if (!m->k_dev) {
        if ((st = dev_alloc_t(h, &m->k_dev, 1)) != BLEST_OK) return st;
        if ((st = dev_alloc_t(h, &m->cursor, 2)) != BLEST_OK) return st;
        if ((st = dev_alloc_t(h, &m->sticky, 1)) != BLEST_OK) return st;
    }
    cudaStream_t cs = h->stream;
    if (!m->cc_exec || m->cc_stream != cs || m->cc_engine != h->ms_engine) {
        ms_release_graph(m);
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return BLEST_ERR_CUDA;
        k_ms_batch_src<<<1, 1024, 0, cs>>>(m->d_src, m->k_dev, m->cursor);
        st = ms_launch(h, 1024, nullptr, m->far, m->reach, m->k_dev);
        k_ms_batch_next<<<1, 1, 0, cs>>>(m->cursor, m->ctl, m->sticky);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(cs, &g);
        if (st != BLEST_OK || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            blest_internal_record_cuda_error(ec, "capture of the closeness batch", __FILE__, __LINE__);
            return st != BLEST_OK ? st : BLEST_ERR_CUDA;
        }
        m->cc_graph = g;
        if (cudaGraphInstantiate(&m->cc_exec, g, 0) != cudaSuccess) {
            ms_release_graph(m);
            return BLEST_ERR_CUDA;
        }
        m->cc_stream = cs;
        m->cc_engine = h->ms_engine;
    }
    const long long range[2] = {(long long)first, (long long)(first + count)};
    if (cudaMemcpyAsync(m->cursor, range, sizeof range, cudaMemcpyHostToDevice, cs) != cudaSuccess)
        return BLEST_ERR_CUDA;
    if (cudaMemsetAsync(m->sticky, 0, sizeof(int), cs) != cudaSuccess) return BLEST_ERR_CUDA;
    for (int64_t b = first; b < first + count; b += 1024)
        if (cudaGraphLaunch(m->cc_exec, cs) != cudaSuccess) return BLEST_ERR_CUDA;
    int err = 0;
    if (cudaMemcpyAsync(&err, m->sticky, sizeof(int), cudaMemcpyDeviceToHost, cs) != cudaSuccess)
        return BLEST_ERR_CUDA;
    if (cudaStreamSynchronize(cs) != cudaSuccess) return BLEST_ERR_CUDA;
    return err ? (blest_status)err : BLEST_OK;
}

static blest_status closeness_common(blest_graph *h, int64_t first, int64_t count, int64_t *far, double *cc,
                                     int64_t *reach) {
    if (!h || h->many) return BLEST_ERR_INVALID;
    if (h->directed || h->sigma != 8) return BLEST_ERR_UNSUPPORTED;
    if (first < 0 || count < 0 || first + count > h->n) return BLEST_ERR_INVALID;
    blest_status st = ms_prepare(h, 1024);
    if (st != BLEST_OK) return st;
    MsbfsWork *m = h->ms;
    if (!m->far) {
        if ((st = dev_alloc_t(h, &m->far, (size_t)h->n)) != BLEST_OK) return st;
        if ((st = dev_alloc_t(h, &m->reach, (size_t)h->n)) != BLEST_OK) return st;
    }
    if (cudaMemsetAsync(m->far, 0, (size_t)h->n * 8, h->stream) != cudaSuccess) return BLEST_ERR_CUDA;
    if (cudaMemsetAsync(m->reach, 0, (size_t)h->n * 8, h->stream) != cudaSuccess) return BLEST_ERR_CUDA;
    if (cudaMemsetAsync(m->stats, 0, sizeof(MsStats), h->stream) != cudaSuccess) return BLEST_ERR_CUDA;
    st = closeness_batches(h, first, count);
    if (st != BLEST_OK) return st;
    // outputs (original ids); host outputs are staged on the device
    void *dfar = far, *dcc = cc, *dreach = reach;
    std::vector<void *> tmp;
    auto stage = [&](void *user, size_t bytes) -> void * {
        if (!user || is_device_ptr(user)) return user;
        void *p = nullptr;
        if (cudaMallocAsync(&p, bytes, h->stream) != cudaSuccess) return nullptr;
        tmp.push_back(p);
        return p;
    };
    dfar = stage(far, (size_t)h->n * 8);
    dcc = stage(cc, (size_t)h->n * 8);
    dreach = stage(reach, (size_t)h->n * 8);
    if ((far && !dfar) || (cc && !dcc) || (reach && !dreach)) return BLEST_ERR_OOM;
    k_cc<<<(unsigned)((h->n + 255) / 256 < 65535 ? (h->n + 255) / 256 : 65535), 256, 0, h->stream>>>(
        m->far, m->reach, h->g.new_of_old, (int)h->n, (long long *)dfar, (double *)dcc, (long long *)dreach);
    if (far && dfar != far) cudaMemcpyAsync(far, dfar, (size_t)h->n * 8, cudaMemcpyDeviceToHost, h->stream);
    if (cc && dcc != cc) cudaMemcpyAsync(cc, dcc, (size_t)h->n * 8, cudaMemcpyDeviceToHost, h->stream);
    if (reach && dreach != reach) cudaMemcpyAsync(reach, dreach, (size_t)h->n * 8, cudaMemcpyDeviceToHost, h->stream);
    for (void *p : tmp) cudaFreeAsync(p, h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return BLEST_ERR_CUDA;
    return BLEST_OK;
}

extern "C" blest_status blest_closeness(blest_handle h, int64_t *far, double *cc, int64_t *reach) {
    if (!h || !far) return BLEST_ERR_INVALID;
    return closeness_common(h, 0, h->n, far, cc, reach);
}

extern "C" blest_status blest_closeness_range(blest_handle h, int64_t first, int64_t count, int64_t *far,
                                              int64_t *reach) {
    if (!h || !far) return BLEST_ERR_INVALID;
    return closeness_common(h, first, count, far, nullptr, reach);
}

extern "C" blest_status blest_msbfs_stats(blest_handle h, blest_msbfs_counters *out) {
    if (!h || !out) return BLEST_ERR_INVALID;
    memset(out, 0, sizeof *out);
    if (!h->ms) return BLEST_OK;
    MsStats st;
    if (cudaMemcpyAsync(&st, h->ms->stats, sizeof st, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return BLEST_ERR_CUDA;
    out->kappa = h->ms->kappa;
    out->launches = (int64_t)st.launches;
    out->levels = (int64_t)st.levels;
    out->vss = (int64_t)st.vss;
    out->hit_words = (int64_t)st.hit_words;
    out->dirty_sets = (int64_t)st.dirty_sets;
    out->pull_levels = (int64_t)st.pull_levels;
    out->pull_arcs = (int64_t)st.pull_arcs;
    return BLEST_OK;
}

extern "C" blest_status blest_set_msbfs_engine(blest_handle h, int32_t tc) {
    if (!h || h->many || (tc != 0 && tc != 1)) return BLEST_ERR_INVALID;
    if (tc && (h->sigma != 8 || h->tau != 128)) return BLEST_ERR_UNSUPPORTED;
    if (tc && !(h->ms_remap && h->ms_track)) return BLEST_ERR_UNSUPPORTED;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return BLEST_ERR_CUDA;
    h->ms_engine = tc;
    return BLEST_OK;
}

extern "C" blest_status blest_set_msbfs_direction(blest_handle h, int32_t mode) {
    if (!h || h->many || mode < 0 || mode > 2) return BLEST_ERR_INVALID;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return BLEST_ERR_CUDA;
    h->ms_dir = mode;
    if (h->ms) ms_release_graph(h->ms);   // the captured closeness batch bakes the direction in
    return BLEST_OK;
}

extern "C" blest_status blest_set_msbfs_output(blest_handle h, int32_t staged) {
    if (!h || h->many || (staged != 0 && staged != 1)) return BLEST_ERR_INVALID;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return BLEST_ERR_CUDA;
    h->ms_out = staged;
    return BLEST_OK;
}

extern "C" blest_status blest_set_msbfs_variant(blest_handle h, int32_t reindex, int32_t tracking) {
    if (!h || h->many || (reindex != 0 && reindex != 1) || (tracking != 0 && tracking != 1)) return BLEST_ERR_INVALID;
    if (h->ms_engine == 1 && !(reindex && tracking)) return BLEST_ERR_UNSUPPORTED;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return BLEST_ERR_CUDA;
    h->ms_remap = reindex;
    h->ms_track = tracking;
    if (h->ms) ms_release_graph(h->ms);   // the captured closeness batch bakes the variant in
    return BLEST_OK;
}
