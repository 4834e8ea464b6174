// Single-source BFS over BVSS: one persistent cooperative kernel runs every
// level (§5.3 kernel fusion) and picks, per level, one of
//   push eager  (Algorithm 2): visited check, atomic OR on the next frontier,
//                the first setter of a slice-set field enqueues its VSSs;
//   push lazy   (Algorithm 3 stage 1): fire-and-forget OR into V_next, then
//                stage 2 sweeps V_curr xor V_next, sets levels and enqueues;
//   bottom-up   (Algorithm 4 stage 1): each unvisited vertex scans its
//                in-neighbours for a frontier vertex, then stage 2;
// the per-VSS hit test (Eq. 2) runs either on tensor cores with the
// m8n8k128 b1 AND.POPC layout of Fig. 3 or on CUDA cores (AND + field test).
//
// The kernel is instantiated per BVSS layout: slice width SIGMA (8, 16, 32)
// and LPV lane words per VSS (32: the warp-wide VSS of §3.1, tau = 32 *
// theta; 8: a narrow VSS of tau = 32 slices, four per warp pass).
//
// State between levels is the same whatever mode ran (levels L, visited
// bits V_curr = V_next, exact frontier bits F, VSS queue Q, slice-set queue
// SQ), so modes mix freely.  F, Q and SQ rotate over three buffers and the
// per-level counters over four slots; the buffer of level l-2 is cleared
// sparsely (only the slice-set fields it holds) while level l runs, so a
// top-down eager level needs a single grid barrier and no O(n) clearing.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "handle.h"
#include "mlp.h"

namespace {

constexpr int BFS_MAX_THREADS = 1024;

struct BfsParams {
    int n, W;
    const int *__restrict__ rowIds;
    const unsigned *__restrict__ masks;
    const int *__restrict__ realPtrs;
    const int *__restrict__ v2r;
    const long long *__restrict__ rp;
    const int *__restrict__ col;
    const int *__restrict__ deg;
    const unsigned *__restrict__ nz;  // bit u set iff u has an in-neighbour (bottom-up levels)
    const int4 *__restrict__ head;    // first four in-neighbours of each vertex
    int *L;
    unsigned *Vc, *Vn;
    unsigned *F[3];
    int2 *Q[3];             // queue entries {VSS id, its slice set}
    int *SQ[3];
    Ctl *ctl;
    blest_level_log *log;
    int log_cap;
    int src;
    int policy, fixed_mode, lazy, tc, switching;
    int defer_queue;        // lazy and bottom-up levels count their VSS queue and leave it to the next level
    int tc16;               // tensor-core levels use the 16-MMA layout instead of Fig. 3's
    float eta;
    const int *schedule;
    int sched_len;
    const float *mlp;
    int batch;              // VSS passes a warp keeps in flight in top-down levels (1, 2, 4)
    float avg_deg;
    unsigned long long budget_ns;
    const int *new_of_old;  // non-null: out[v] = L[new_of_old[v]]
    int *out;
};

// Compile-time facts of a BVSS layout.
template <int SIGMA, int LPV>
struct Lay {
    static constexpr int THETA = 32 / SIGMA;           // slices per lane word
    static constexpr int TAU = LPV * THETA;            // slices per VSS
    static constexpr int G = 32 / LPV;                 // VSSs per warp pass
    static constexpr int LOGS = SIGMA == 8 ? 3 : (SIGMA == 16 ? 4 : 5);
    static constexpr unsigned FMASK = SIGMA == 32 ? 0xFFFFFFFFu : ((1u << SIGMA) - 1u);
    static constexpr bool TC_OK = SIGMA == 8 && LPV == 32;   // the Fig. 3 fragment layout
};

// CUDA-core hit test: bit c set iff slice c of the lane word shares a bit
// with the slice set's frontier field alpha (popc(mask_c & alpha) > 0).
template <int SIGMA>
__device__ __forceinline__ unsigned hits_cc(unsigned m, unsigned alpha) {
    if constexpr (SIGMA == 8) {
        const unsigned x = m & (alpha * 0x01010101u);
        return (unsigned)((x & 0xFFu) != 0) | ((unsigned)((x & 0xFF00u) != 0) << 1) |
               ((unsigned)((x & 0xFF0000u) != 0) << 2) | ((unsigned)((x >> 24) != 0) << 3);
    } else if constexpr (SIGMA == 16) {
        const unsigned x = m & (alpha * 0x00010001u);
        return (unsigned)((x & 0xFFFFu) != 0) | ((unsigned)((x >> 16) != 0) << 1);
    } else {
        return (unsigned)((m & alpha) != 0);
    }
}

// Fig. 3 layout: fragA = two packed sigma-bit masks in the low 16 bits;
// fragB = alpha on lanes t mod 9 == 0, alpha << 8 on lanes t mod 9 == 4,
// zero elsewhere.  Lane t's fragC pair is popc(mask_c & alpha) for its own
// two slices, so no shuffle is needed.  bsel = 1, 256 or 0 by lane.
__device__ __forceinline__ unsigned hits_tc(unsigned m, unsigned alpha, unsigned bsel) {
    const unsigned fb = alpha * bsel;
    int d0, d1, d2, d3;
    asm volatile(
        "mma.sync.aligned.m8n8k128.row.col.s32.b1.b1.s32.and.popc {%0,%1}, {%2}, {%3}, {%4,%5};\n"
        : "=r"(d0), "=r"(d1)
        : "r"(m & 0xFFFFu), "r"(fb), "r"(0), "r"(0));
    asm volatile(
        "mma.sync.aligned.m8n8k128.row.col.s32.b1.b1.s32.and.popc {%0,%1}, {%2}, {%3}, {%4,%5};\n"
        : "=r"(d2), "=r"(d3)
        : "r"(m >> 16), "r"(fb), "r"(0), "r"(0));
    return (unsigned)(d0 != 0) | ((unsigned)(d1 != 0) << 1) | ((unsigned)(d2 != 0) << 2) |
           ((unsigned)(d3 != 0) << 3);
}

// The layout Fig. 3 improves on: one slice per fragment row, so 16 MMAs per
// 128 slices.  MMA i takes slices 8i .. 8i + 7 (lane 2i + r/4, byte r % 4 of
// the VSS's mask words): row r of fragA holds slice 8i + r in the low byte
// of thread 4r, column 0 of fragB holds alpha in thread 0's low byte, and
// D[r][0] = popc(slice & alpha) lands in thread 4r's first accumulator; a
// ballot returns each slice's hit to the lane that owns it.  Used by the
// ablation that measures the optimal layout against it.
__device__ __forceinline__ unsigned hits_tc16(unsigned m, unsigned alpha) {
    const int lane = lane_id();
    const int r = lane >> 2;
    const bool head = (lane & 3) == 0;
    const unsigned fb = lane == 0 ? alpha : 0u;
    unsigned hits = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const unsigned w = __shfl_sync(FULL_MASK, m, 2 * i + (r >> 2));
        const unsigned fa = head ? ((w >> (8 * (r & 3))) & 0xFFu) : 0u;
        int d0, d1;
        asm volatile(
            "mma.sync.aligned.m8n8k128.row.col.s32.b1.b1.s32.and.popc {%0,%1}, {%2}, {%3}, {%4,%5};\n"
            : "=r"(d0), "=r"(d1)
            : "r"(fa), "r"(fb), "r"(0), "r"(0));
        const unsigned hb = __ballot_sync(FULL_MASK, head && d0 != 0);   // bit 4r: slice 8i + r
        if ((lane >> 1) == i) {
            const unsigned x = hb >> (16 * (lane & 1));                   // rows 4h .. 4h + 3
            hits = (x & 1u) | ((x >> 3) & 2u) | ((x >> 6) & 4u) | ((x >> 9) & 8u);
        }
    }
    return hits;
}

// the theta row ids of lane word `word` (one 4-, 8- or 16-byte load)
template <int THETA>
__device__ __forceinline__ void load_rows(const int *__restrict__ rowIds, size_t word, int (&r)[4]) {
    if constexpr (THETA == 4) {
        const int4 v = __ldg(reinterpret_cast<const int4 *>(rowIds) + word);
        r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
    } else if constexpr (THETA == 2) {
        const int2 v = __ldg(reinterpret_cast<const int2 *>(rowIds) + word);
        r[0] = v.x; r[1] = v.y; r[2] = 0; r[3] = 0;
    } else {
        r[0] = __ldg(rowIds + word); r[1] = 0; r[2] = 0; r[3] = 0;
    }
}

__device__ __forceinline__ int pick(const int4 &r, int c) {
    return c == 0 ? r.x : (c == 1 ? r.y : (c == 2 ? r.z : r.w));
}

// the SIGMA frontier bits of slice set ss (its field of the bitvector)
template <int SIGMA>
__device__ __forceinline__ unsigned ld_field(const unsigned *F, int ss) {
    if constexpr (SIGMA == 8) return (unsigned)reinterpret_cast<const unsigned char *>(F)[ss];
    else if constexpr (SIGMA == 16) return (unsigned)reinterpret_cast<const unsigned short *>(F)[ss];
    else return F[ss];
}

template <int SIGMA>
__device__ __forceinline__ void clear_field(unsigned *F, int ss) {
    if constexpr (SIGMA == 8) reinterpret_cast<unsigned char *>(F)[ss] = 0;
    else if constexpr (SIGMA == 16) reinterpret_cast<unsigned short *>(F)[ss] = 0;
    else F[ss] = 0u;
}

// position of the k-th (0-based) set bit of x
__device__ __forceinline__ int nth_set_bit(unsigned x, int k) {
    int pos = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const unsigned lo = x & ((1u << step) - 1u);
        const int c = __popc(lo);
        if (k >= c) { k -= c; x >>= step; pos += step; }
        else x = lo;
    }
    return pos;
}

// Queue appends are staged per warp in shared memory and reserved in the
// global queues once per STG_Q entries: every warp reserving its own few
// entries with one atomic on the same two counters serialises tens of
// thousands of same-address atomics per level in one L2 slice.
constexpr int STG_Q = 256;   // staged VSS entries per warp
constexpr int STG_S = 128;   // staged slice-set ids per warp (>= 32 lanes x 4 sets)
constexpr int STG_BYTES = STG_Q * 8 + STG_S * 4;

// Per-CTA totals of a level's appends and counters (shared memory, zeroed at
// the level start): the level's last flush reserves queue space and adds
// the counters once per CTA instead of once per warp, so the control block
// sees a few hundred atomics per level rather than thousands.
struct BlkAcc {
    int q, s;                       // staged queue entries / slice-set ids of the CTA
    int qbase, sbase;               // the CTA's reserved offsets
    unsigned long long nv, fe;      // newly visited vertices and their out-arcs
    unsigned long long sv, sa;      // bottom-up: probed vertices and extra arcs read
};

struct Stage {
    int2 *q;     // this warp's staging area in shared memory
    int *sq;
    int qn, sqn; // staged counts (warp-uniform)
    int defer;   // the level's VSS queue is counted, not written (warp-uniform)
    int qdef;    // VSS entries counted but not written by this warp
};

__device__ __forceinline__ void stage_flush(const BfsParams &P, Stage &st, int2 *Q, int *SQ, int slot) {
    const int lane = lane_id();
    __syncwarp();
    // both reservations are issued before either is used: one round trip
    int qb = 0, sb = 0;
    if (lane == 0) {
        if (st.qn) qb = atomicAdd(&P.ctl->qlen[slot], st.qn);
        if (st.sqn) sb = atomicAdd(&P.ctl->sqlen[slot], st.sqn);
    }
    qb = __shfl_sync(FULL_MASK, qb, 0);
    sb = __shfl_sync(FULL_MASK, sb, 0);
    for (int k = lane; k < st.qn; k += 32) Q[qb + k] = st.q[k];
    for (int k = lane; k < st.sqn; k += 32) SQ[sb + k] = st.sq[k];
    __syncwarp();
    st.qn = 0;
    st.sqn = 0;
}

// Warp-aggregated enqueue of up to 4 slice sets per lane (bit c of `want`
// set => slice set ss[c], whose VSSs are [a[c], a[c] + len[c])): the VSS
// ranges go to Q, the set ids to SQ, both through the warp's staging area.
// Short ranges are written by their own lane; a long range (the slice set
// of a hub vertex spans thousands of VSSs) by the whole warp, so no lane
// issues a long serial run of stores; a batch larger than the staging area
// reserves its own space in Q.
constexpr int ENQ_LANE_MAX = 8;

__device__ __forceinline__ void enqueue_ranges(const BfsParams &P, Stage &st, unsigned want, const int ss[4],
                                               const int a[4], const int len[4], int2 *Q, int *SQ, int slot) {
    const int lane = lane_id();
    if (!__any_sync(FULL_MASK, want != 0)) return;
    int tot = 0, nset = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (want >> c & 1u) { tot += len[c]; ++nset; }
    const int incl = warp_incl_scan(tot);
    const int sincl = warp_incl_scan(nset);
    const int T = __shfl_sync(FULL_MASK, incl, 31);
    const int S = __shfl_sync(FULL_MASK, sincl, 31);
    if (st.defer) {
        // deferred queue: the slice sets are staged, their VSSs only counted
        // (the next level expands them from the slice-set queue if it pushes)
        if (st.sqn + S > STG_S) stage_flush(P, st, Q, SQ, slot);
        int sb = st.sqn + sincl - nset;
        st.sqn += S;
        st.qdef += T;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (want >> c & 1u) st.sq[sb++] = ss[c];
        __syncwarp();
        return;
    }
    if ((T <= STG_Q && st.qn + T > STG_Q) || st.sqn + S > STG_S) stage_flush(P, st, Q, SQ, slot);
    int2 *dst;
    int qbase;
    if (T > STG_Q) {
        int g = 0;
        if (lane == 31) g = atomicAdd(&P.ctl->qlen[slot], T);
        dst = Q + __shfl_sync(FULL_MASK, g, 31);
        qbase = incl - tot;
    } else {
        dst = st.q;
        qbase = st.qn + incl - tot;
        st.qn += T;
    }
    int sbase = st.sqn + sincl - nset;
    st.sqn += S;
    int pos[4];
    unsigned big = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        pos[c] = qbase;
        if (want >> c & 1u) {
            st.sq[sbase++] = ss[c];
            if (len[c] <= ENQ_LANE_MAX) {
                for (int k = 0; k < len[c]; ++k) dst[qbase + k] = make_int2(a[c] + k, ss[c]);
            } else {
                big |= 1u << c;
            }
            qbase += len[c];
        }
    }
    unsigned lanes = __ballot_sync(FULL_MASK, big != 0);
    while (lanes) {
        const int j = __ffs(lanes) - 1;
        lanes &= lanes - 1u;
        const unsigned bj = __shfl_sync(FULL_MASK, big, j);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int aj = __shfl_sync(FULL_MASK, a[c], j);
            const int lj = __shfl_sync(FULL_MASK, len[c], j);
            const int pj = __shfl_sync(FULL_MASK, pos[c], j);
            const int sj = __shfl_sync(FULL_MASK, ss[c], j);
            if (bj >> c & 1u)   // warp-uniform
                for (int k = lane; k < lj; k += 32) dst[pj + k] = make_int2(aj + k, sj);
        }
    }
    __syncwarp();
}

// Called by every thread of the CTA at the end of a level's last phase.
__device__ __forceinline__ void block_flush(const BfsParams &P, Stage &st, BlkAcc *acc, int2 *Q, int *SQ, int slot,
                                            unsigned long long nv, unsigned long long fe) {
    const int lane = lane_id();
    nv = warp_sum(nv);
    fe = warp_sum(fe);
    int wq = 0, ws = 0;
    if (lane == 0) {
        if (st.qn + st.qdef) wq = atomicAdd(&acc->q, st.qn + st.qdef);   // deferred entries follow the staged ones
        if (st.sqn) ws = atomicAdd(&acc->s, st.sqn);
        if (nv) {
            atomicAdd(&acc->nv, nv);
            atomicAdd(&acc->fe, fe);
        }
    }
    wq = __shfl_sync(FULL_MASK, wq, 0);
    ws = __shfl_sync(FULL_MASK, ws, 0);
    __syncthreads();
    if (threadIdx.x == 0) {
        acc->qbase = acc->q ? atomicAdd(&P.ctl->qlen[slot], acc->q) : 0;
        acc->sbase = acc->s ? atomicAdd(&P.ctl->sqlen[slot], acc->s) : 0;
        if (acc->nv) {
            red_add_u64(&P.ctl->newv[slot], acc->nv);
            red_add_u64(&P.ctl->fedges[slot], acc->fe);
        }
        if (acc->sv) {
            red_add_u64(&P.ctl->scan_v[slot], acc->sv);
            red_add_u64(&P.ctl->scan_a[slot], acc->sa);
        }
    }
    __syncthreads();
    const int qb = acc->qbase + wq, sb = acc->sbase + ws;
    for (int k = lane; k < st.qn; k += 32) Q[qb + k] = st.q[k];
    for (int k = lane; k < st.sqn; k += 32) SQ[sb + k] = st.sq[k];
    __syncwarp();
    st.qn = 0;
    st.sqn = 0;
    st.qdef = 0;
}

// Writes a deferred VSS queue: the VSS ranges of the nsq slice sets in SQ.
// Each CTA takes a contiguous share of the slice sets, blockDim.x at a time:
// a block-wide scan of the range lengths, one reservation in Q per round,
// then every thread writes entries k, k + blockDim.x, ... of the round,
// finding each entry's slice set by binary search over the scan, so a hub's
// range of thousands of VSSs is spread over the whole CTA.  Called by every
// thread of the grid; a grid barrier follows.  (Push levels take their
// entries in any order.)
__device__ void expand_queue(const BfsParams &P, int bc, int sc, int nsq) {
    __shared__ int s_incl[BFS_MAX_THREADS], s_a[BFS_MAX_THREADS], s_ss[BFS_MAX_THREADS];
    __shared__ int s_wsum[32];
    __shared__ int s_tot, s_base;
    const int lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int *SQc = P.SQ[bc];
    int2 *Qc = P.Q[bc];
    const int per = (nsq + (int)gridDim.x - 1) / (int)gridDim.x;
    const int lo = (int)blockIdx.x * per, hi = min(nsq, lo + per);
    for (int r0 = lo; r0 < hi; r0 += blockDim.x) {   // CTA-uniform
        const int j = r0 + (int)threadIdx.x;
        int ss = 0, a = 0, len = 0;
        if (j < hi) {
            ss = SQc[j];
            a = __ldg(&P.realPtrs[ss]);
            len = __ldg(&P.realPtrs[ss + 1]) - a;
        }
        int incl = warp_incl_scan(len);
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int x = lane < nwarps ? s_wsum[lane] : 0;
            const int xi = warp_incl_scan(x);
            s_wsum[lane] = xi - x;
            if (lane == 31) s_tot = xi;
        }
        __syncthreads();
        incl += s_wsum[warp];
        s_incl[threadIdx.x] = incl;
        s_a[threadIdx.x] = a;
        s_ss[threadIdx.x] = ss;
        if (threadIdx.x == 0) s_base = s_tot ? atomicAdd(&P.ctl->xq[sc], s_tot) : 0;
        __syncthreads();
        const int tot = s_tot, base = s_base;
        const int nent = min((int)blockDim.x, hi - r0);
        for (int k = threadIdx.x; k < tot; k += blockDim.x) {
            int l = 0, h = nent - 1;   // the first entry whose inclusive end exceeds k
            while (l < h) {
                const int mid = (l + h) >> 1;
                if (s_incl[mid] > k) h = mid;
                else l = mid + 1;
            }
            const int ex = l ? s_incl[l - 1] : 0;
            Qc[base + k] = make_int2(s_a[l] + (k - ex), s_ss[l]);
        }
        __syncthreads();   // the arrays are rewritten by the next round
    }
}

// ---------------------------------------------------------------- push
// Eager (Algorithm 2) or lazy (Algorithm 3 stage 1) top-down level.  A warp
// pass covers G VSSs (one per lane group of LPV lanes); a warp keeps B passes
// in flight: it loads the B*G queue entries, then their slices and masks,
// then their frontier fields, before using any of them, so the
// dependent-load chain is paid once per B*G VSSs.
// The VSS entries of one warp pass: lane j < B*G holds entry j ({VSS, slice
// set}, VSS -1 = none), nent of them valid; lane group g of LPV lanes
// handles entries g, g + G, ... (B of them, loaded before any is used).
template <bool EAGER, int HIT, int B, int SIGMA, int LPV>
__device__ __forceinline__ void push_entries(const BfsParams &P, Stage &st, BlkAcc *acc, int ell, int bc, int bn,
                                             int slot, unsigned bsel, int2 mine, int nent, unsigned long long &nv,
                                             unsigned long long &fe) {
    using LY = Lay<SIGMA, LPV>;
    constexpr int THETA = LY::THETA, G = LY::G;
    const int lane = lane_id();
    const int grp = lane / LPV, sl = lane % LPV;
    const unsigned *Fc = P.F[bc];
    unsigned *Fn = P.F[bn];
    int vss[B], ss[B];
    int r[B][4];
    unsigned m[B], alpha[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        vss[b] = __shfl_sync(FULL_MASK, mine.x, b * G + grp);
        ss[b] = __shfl_sync(FULL_MASK, mine.y, b * G + grp);
    }
    // slices, masks and frontier fields of the VSSs are independent loads
#pragma unroll
    for (int b = 0; b < B; ++b) {
        if (vss[b] >= 0) {
            load_rows<THETA>(P.rowIds, (size_t)vss[b] * LPV + sl, r[b]);
            m[b] = __ldg(&P.masks[(size_t)vss[b] * LPV + sl]);
            alpha[b] = ld_field<SIGMA>(Fc, ss[b]);
        } else {
            r[b][0] = r[b][1] = r[b][2] = r[b][3] = 0;
            m[b] = 0u;
            alpha[b] = 0u;
        }
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
        if (b * G >= nent) continue;   // warp-uniform: no group has an entry
        unsigned hits;
        if constexpr (HIT == 1) hits = hits_tc(m[b], alpha[b], bsel);
        else if constexpr (HIT == 2) hits = hits_tc16(m[b], alpha[b]);
        else hits = hits_cc<SIGMA>(m[b], alpha[b]);
        if (EAGER) {
            // phase 1: visited words of the hit rows (independent loads)
            int u[4];
            unsigned vw[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                u[c] = r[b][c];
                vw[c] = (c < THETA && (hits >> c & 1u)) ? P.Vc[u[c] >> 5] : 0xFFFFFFFFu;
            }
            // phase 2: claim the unvisited ones, one atomic per candidate row (the
            // lanes' atomics on a word are serialised by the memory system, so
            // exactly one lane sees each bit and each slice-set field clear;
            // combining them across the warp first costs more than it saves).
            // All of a lane's atomics and its degree and VSS-range loads are
            // issued before any result is used: one round trip together.
            unsigned old[4];
            int dg[4], a[4], len[4], sso[4];
            unsigned cand = 0;
#pragma unroll
            for (int c = 0; c < THETA; ++c) {
                const bool cd = !(vw[c] >> (u[c] & 31) & 1u);
                old[c] = 0xFFFFFFFFu;
                if (cd) {
                    old[c] = atomicOr(&Fn[u[c] >> 5], 1u << (u[c] & 31));
                    cand |= 1u << c;
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                sso[c] = c < THETA ? (u[c] >> LY::LOGS) : 0;
                dg[c] = 0;
                a[c] = 0;
                len[c] = 0;
                if (cand >> c & 1u) {
                    dg[c] = __ldg(&P.deg[u[c]]);
                    a[c] = __ldg(&P.realPtrs[sso[c]]);
                    len[c] = __ldg(&P.realPtrs[sso[c] + 1]);
                }
            }
            // phase 3: winners set their level and visited bits (one OR per word
            // among the lane's own rows, which ascend); the first claim of a
            // slice-set field enqueues its VSSs (once per set)
            unsigned want = 0, wbits = 0;
            int wword = -1;
#pragma unroll
            for (int c = 0; c < THETA; ++c) {
                const bool win = (cand >> c & 1u) && !(old[c] >> (u[c] & 31) & 1u);
                if (win) {
                    const int wd = u[c] >> 5;
                    if (wd != wword) {
                        if (wword >= 0) {
                            red_or(&P.Vc[wword], wbits);
                            red_or(&P.Vn[wword], wbits);
                        }
                        wword = wd;
                        wbits = 0;
                    }
                    wbits |= 1u << (u[c] & 31);
                    P.L[u[c]] = ell;
                    nv += 1;
                    fe += (unsigned long long)dg[c];
                    const int fo = u[c] & (31 & ~(SIGMA - 1));   // the set's field in the word
                    if (((old[c] >> fo) & LY::FMASK) == 0) want |= 1u << c;
                }
                len[c] -= a[c];
            }
            if (wword >= 0) {
                red_or(&P.Vc[wword], wbits);
                red_or(&P.Vn[wword], wbits);
            }
            enqueue_ranges(P, st, want, sso, a, len, P.Q[bn], P.SQ[bn], slot);
        } else {
            // lazy marking: fire-and-forget ORs into V_next, one per distinct word
            // among the lane's own rows (they ascend, so equal words are adjacent)
            unsigned mbits = 0;
            int mword = -1;
#pragma unroll
            for (int c = 0; c < THETA; ++c) {
                if (hits >> c & 1u) {
                    const int u = r[b][c];
                    if ((u >> 5) != mword) {
                        if (mword >= 0) red_or(&P.Vn[mword], mbits);
                        mword = u >> 5;
                        mbits = 0;
                    }
                    mbits |= 1u << (u & 31);
                }
            }
            if (mword >= 0) red_or(&P.Vn[mword], mbits);
        }
    }
}

// Eager (Algorithm 2) or lazy (Algorithm 3 stage 1) top-down level.  A warp
// pass covers G VSSs (one per lane group of LPV lanes); a warp keeps B passes
// in flight: it loads the B*G queue entries, then their slices and masks,
// then their frontier fields, before using any of them, so the
// dependent-load chain is paid once per B*G VSSs.  Passes are interleaved
// over the blocks; the warps of a block claim their block's next pass from
// a shared counter, so a warp whose passes hit many rows does not hold up
// the level.
template <bool EAGER, int HIT, int B, int SIGMA, int LPV>
__device__ void push_level(const BfsParams &P, Stage &st, int *grab, BlkAcc *acc, int ell, int bc, int bn, int slot,
                           int qlen, unsigned bsel) {
    using LY = Lay<SIGMA, LPV>;
    constexpr int G = LY::G;
    const int lane = lane_id();
    const int2 *Qc = P.Q[bc];
    unsigned long long nv = 0, fe = 0;
    const int npass = (qlen + B * G - 1) / (B * G);
    for (;;) {
        int k = 0;
        if (lane == 0) k = atomicAdd(grab, 1);
        k = __shfl_sync(FULL_MASK, k, 0);
        const int pass = (int)blockIdx.x + k * (int)gridDim.x;
        if (pass >= npass) break;
        const int w0 = pass * B * G;
        // lane j < B*G fetches queue entry w0 + j (VSS and slice set)
        const int2 mine = (lane < B * G && w0 + lane < qlen) ? Qc[w0 + lane] : make_int2(-1, 0);
        push_entries<EAGER, HIT, B, SIGMA, LPV>(P, st, acc, ell, bc, bn, slot, bsel, mine, qlen - w0, nv, fe);
    }
    if (EAGER) {
        block_flush(P, st, acc, P.Q[bn], P.SQ[bn], slot, nv, fe);
    }
}

// ------------------------------------------------------------ bottom-up
// Algorithm 4 stage 1.  A warp loads 32 visited words at once (lane = word),
// keeps only unvisited vertices that have in-neighbours (nz mask), and then
// walks the compacted list 32 vertices at a time (lane = vertex).  Each lane
// probes its in-neighbours four at a time: four column loads, then four
// frontier-bit loads, then the test.  Found bits collect in shared memory
// and each word's V_next is written once by the warp that owns it.

// Algorithm 4's test for one unvisited vertex u (act): is any in-neighbour
// in the frontier?  The first four in-neighbours (rows sorted by descending
// degree) come from the 16-byte head hd; the highest-degree one is probed
// alone first (the likeliest frontier member), the other three only where
// it missed, which keeps the random frontier-word reads through L2 to about
// one a vertex; longer rows then read four ids per step.
__device__ __forceinline__ bool bu_probe_head(const BfsParams &P, const unsigned *Fc, int u, bool act, const int4 &hd,
                                              unsigned long long &sa) {
    const int v0 = hd.x;
    const unsigned f0 = v0 >= 0 ? Fc[v0 >> 5] : 0u;
    bool hit = (v0 >= 0) && ((f0 >> (v0 & 31)) & 1u);
    unsigned fw[3];
#pragma unroll
    for (int q = 1; q < 4; ++q) {
        const int vq = pick(hd, q);
        fw[q - 1] = (!hit && vq >= 0) ? Fc[vq >> 5] : 0u;
    }
#pragma unroll
    for (int q = 1; q < 4; ++q) {
        const int vq = pick(hd, q);
        hit |= (vq >= 0) && ((fw[q - 1] >> (vq & 31)) & 1u);
    }
    if (act && !hit && hd.w >= 0) {
        long long p = __ldg(&P.rp[u]) + 4;
        const long long e = __ldg(&P.rp[u + 1]);
        while (!hit && p < e) {
            sa += (unsigned long long)((e - p) < 4 ? (e - p) : 4);
            int w4[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) w4[q] = (p + q < e) ? __ldg(&P.col[p + q]) : -1;
            unsigned f4[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) f4[q] = w4[q] >= 0 ? Fc[w4[q] >> 5] : 0u;
#pragma unroll
            for (int q = 0; q < 4; ++q) hit |= (w4[q] >= 0) && ((f4[q] >> (w4[q] & 31)) & 1u);
            p += 4;
        }
    }
    return act && hit;
}

// Probes of one 32-word group, compacted: the unvisited vertices (with an
// in-neighbour) of the group are numbered and handled two per lane per
// round.  Returns the lane's word of found bits (word base + lane).
__device__ __forceinline__ unsigned bu_probe_compact(const BfsParams &P, const unsigned *Fc, int base, unsigned unv,
                                                     unsigned *found, unsigned long long &sv,
                                                     unsigned long long &sa) {
    const int lane = lane_id();
    found[lane] = 0u;
    const int cnt = __popc(unv);
    const int incl = warp_incl_scan(cnt);
    const int total = __shfl_sync(FULL_MASK, incl, 31);
    const int excl = incl - cnt;
    __syncwarp();
    // two compacted vertices per lane per round: idx = b + lane and b + 32 + lane
    for (int b = 0; b < total; b += 64) {
        int u[2];
        bool act[2], hit[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int idx = b + 32 * k + lane;
            act[k] = idx < total;
            hit[k] = false;
            // owner lane: the largest lane whose exclusive prefix is <= idx (a lane with
            // cnt == 0 shares its prefix with the next lane, so the largest one owns idx)
            int j = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int ex = __shfl_sync(FULL_MASK, excl, j + step);
                if (idx >= ex) j += step;
            }
            const unsigned uj = __shfl_sync(FULL_MASK, unv, j);
            const int ej = __shfl_sync(FULL_MASK, excl, j);
            u[k] = act[k] ? ((base + j) << 5) + nth_set_bit(uj, idx - ej) : 0;
        }
        int4 hd[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            hd[k] = act[k] ? __ldg(&P.head[u[k]]) : make_int4(-1, -1, -1, -1);
            if (act[k]) sv += 1;
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) hit[k] = bu_probe_head(P, Fc, u[k], act[k], hd[k], sa);
#pragma unroll
        for (int k = 0; k < 2; ++k)
            if (act[k] && hit[k]) atomicOr(&found[(u[k] >> 5) - base], 1u << (u[k] & 31));
    }
    __syncwarp();
    const unsigned f = found[lane];
    __syncwarp();
    return f;
}

// Probes of one 32-word group, direct: lane b handles vertex 32 w + b of
// each word w that holds a candidate, four words at a time, so a lane keeps
// four head loads in flight and the head loads of a word are one coalesced
// 512-byte access.  For levels where most vertices are unvisited.
constexpr int BU_K = 4;
__device__ __forceinline__ unsigned bu_probe_direct(const BfsParams &P, const unsigned *Fc, int base, unsigned unv,
                                                    unsigned long long &sv, unsigned long long &sa) {
    const int lane = lane_id();
    unsigned mine = 0u;
    unsigned todo = __ballot_sync(FULL_MASK, unv != 0u);   // words with a candidate
    while (todo) {   // warp-uniform
        int wj[BU_K];
        unsigned uw[BU_K];
#pragma unroll
        for (int k = 0; k < BU_K; ++k) {
            wj[k] = todo ? __ffs(todo) - 1 : -1;
            todo &= todo ? todo - 1u : 0u;
            uw[k] = __shfl_sync(FULL_MASK, unv, wj[k] >= 0 ? wj[k] : 0);
            if (wj[k] < 0) uw[k] = 0u;
        }
        int v[BU_K];
        bool act[BU_K], hit[BU_K];
        int4 hd[BU_K];
#pragma unroll
        for (int k = 0; k < BU_K; ++k) {
            act[k] = (uw[k] >> lane) & 1u;
            v[k] = ((base + (wj[k] >= 0 ? wj[k] : 0)) << 5) + lane;
            hd[k] = act[k] ? __ldg(&P.head[v[k]]) : make_int4(-1, -1, -1, -1);
            if (act[k]) sv += 1;
        }
#pragma unroll
        for (int k = 0; k < BU_K; ++k) hit[k] = bu_probe_head(P, Fc, v[k], act[k], hd[k], sa);
#pragma unroll
        for (int k = 0; k < BU_K; ++k) {
            const unsigned fb = __ballot_sync(FULL_MASK, act[k] && hit[k]);
            if (lane == wj[k]) mine = fb;
        }
    }
    return mine;
}

// --------------------------------------------------- stage 2 (finalize)
// Algorithm 3 stage 2 for one group of 32 bitvector words (lane = word):
// nx / cu are the lane's V_next / V_curr words; diff = nx ^ cu are the
// vertices reached at this level.  F and V_curr take the new values (and
// V_next too when write_vn: the fused bottom-up level computes nx in
// registers); a word with at most four new vertices stores their levels and
// loads their out-degrees from its own lane, a denser word is stored lane =
// vertex, eight words per round, so those stores coalesce.  A word holds
// theta = 32/SIGMA slice-set fields; a changed field enqueues its set.
template <int SIGMA>
__device__ __forceinline__ void finalize_group(const BfsParams &P, Stage &st, BlkAcc *acc, int base, unsigned nx,
                                               unsigned cu,
                                               bool write_vn, int ell, int bn, int slot, unsigned long long &nv,
                                               unsigned long long &fe) {
    constexpr int THETA = 32 / SIGMA;
    constexpr unsigned FMASK = SIGMA == 32 ? 0xFFFFFFFFu : ((1u << SIGMA) - 1u);
    const int lane = lane_id();
    unsigned *Fn = P.F[bn];
    const int t = base + lane;
    unsigned diff = 0;
    if (t < P.W) {
        diff = nx ^ cu;
        if (diff) {
            P.Vc[t] = nx;
            if (write_vn) P.Vn[t] = nx;
            Fn[t] = diff;
            nv += (unsigned long long)__popc(diff);
        }
    }
    // the VSS ranges of the changed slice-set fields load together with the
    // degrees below
    unsigned want = 0;
    int sso[4] = {0, 0, 0, 0}, ra[4] = {0, 0, 0, 0}, rl[4] = {0, 0, 0, 0};
#pragma unroll
    for (int c = 0; c < THETA; ++c) {
        sso[c] = t * THETA + c;
        if ((diff >> (SIGMA * c)) & FMASK) {
            want |= 1u << c;
            ra[c] = __ldg(&P.realPtrs[sso[c]]);
            rl[c] = __ldg(&P.realPtrs[sso[c] + 1]);
        }
    }
    // a sparse word (at most four new vertices): level stores and degree
    // loads from its own lane, the degrees summed only after the enqueue
    // below, so their latency overlaps it
    const int pc = __popc(diff);
    int dv[4] = {0, 0, 0, 0};
    if (pc > 0 && pc <= 4) {
        unsigned d = diff;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (d) {
                const int v = t * 32 + __ffs(d) - 1;
                d &= d - 1u;
                dv[q] = __ldg(&P.deg[v]);
                P.L[v] = ell;
            }
        }
    }
    // a dense word: one 16-byte degree load per group of four vertices
    // holding a new one, all in flight together
    if (pc > 4) {
        const int4 *dq = reinterpret_cast<const int4 *>(P.deg) + (size_t)t * 8;
        unsigned long long dsum = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const unsigned nib = (diff >> (4 * q)) & 0xFu;
            if (nib) {
                const int v0 = t * 32 + 4 * q;
                int4 dd;
                if (v0 + 4 <= P.n) {
                    dd = __ldg(dq + q);
                } else {   // the last, partial word: no load past vertex n - 1
                    dd.x = __ldg(&P.deg[v0]);
                    dd.y = v0 + 1 < P.n ? __ldg(&P.deg[v0 + 1]) : 0;
                    dd.z = v0 + 2 < P.n ? __ldg(&P.deg[v0 + 2]) : 0;
                    dd.w = v0 + 3 < P.n ? __ldg(&P.deg[v0 + 3]) : 0;
                }
                dsum += (unsigned long long)((nib & 1u ? dd.x : 0) + (nib & 2u ? dd.y : 0) +
                                             (nib & 4u ? dd.z : 0) + (nib & 8u ? dd.w : 0));
            }
        }
        fe += dsum;
    }
    const unsigned dense = __ballot_sync(FULL_MASK, pc > 4);
    if (dense) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (!((dense >> (8 * r)) & 0xFFu)) continue;   // warp-uniform
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int j = 8 * r + k;
                const unsigned dj = __shfl_sync(FULL_MASK, diff, j);
                if ((dense >> j & 1u) && (dj >> lane & 1u)) P.L[((base + j) << 5) + lane] = ell;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) rl[c] -= ra[c];
    enqueue_ranges(P, st, want, sso, ra, rl, P.Q[bn], P.SQ[bn], slot);
    fe += (unsigned long long)(dv[0] + dv[1]) + (unsigned long long)(dv[2] + dv[3]);
}

// Stage 2 over all words: a claim covers one 32-word group; claims are
// interleaved over the blocks and taken by the block's warps from a shared
// counter (the changed words cluster, so a fixed split leaves a few warps
// with most of the work).
template <int SIGMA>
__device__ void finalize_level(const BfsParams &P, Stage &st, int *grab, BlkAcc *acc, int ell, int bn, int slot) {
    const int lane = lane_id();
    unsigned long long nv = 0, fe = 0;
    const int ngroups = (P.W + 31) / 32;
    // one group per claim; the next group's words load while the current
    // one is finalised
    auto claim = [&](int &i, unsigned &nx, unsigned &cu) {
        int k = 0;
        if (lane == 0) k = atomicAdd(grab, 1);
        k = __shfl_sync(FULL_MASK, k, 0);
        i = (int)blockIdx.x + k * (int)gridDim.x;
        const int tt = i * 32 + lane;
        const bool ok = i < ngroups && tt < P.W;
        nx = ok ? P.Vn[tt] : 0u;
        cu = ok ? P.Vc[tt] : 0u;
    };
    int i;
    unsigned nx, cu;
    claim(i, nx, cu);
    while (i < ngroups) {
        int i1;
        unsigned nx1, cu1;
        claim(i1, nx1, cu1);
        finalize_group<SIGMA>(P, st, acc, i * 32, nx, cu, false, ell, bn, slot, nv, fe);
        i = i1;
        nx = nx1;
        cu = cu1;
    }
    block_flush(P, st, acc, P.Q[bn], P.SQ[bn], slot, nv, fe);
}

// ------------------------------------------------------------ bottom-up
// Algorithm 4 stage 1 fused with stage 2.  A warp claims a group of 32
// bitvector words (lane = word), keeps the unvisited vertices that have
// in-neighbours (nz mask) and probes them (direct when most vertices are
// unvisited, compacted otherwise).  Each word is owned by the warp that
// claimed it and the probes read only the previous frontier F[bc], so the
// warp finalises its own words at once (V_curr = V_next = visited | found,
// F = found, levels, queue): one grid barrier per bottom-up level.
template <int SIGMA>
__device__ void bottom_up_level(const BfsParams &P, Stage &st, int *grab, BlkAcc *acc, int ell, int bc, int bn,
                                int slot, unsigned *s_found, bool direct) {
    const int lane = lane_id();
    unsigned *found = s_found + (threadIdx.x >> 5) * 32;
    const unsigned *Fc = P.F[bc];
    const int tail = P.n & 31;
    unsigned long long sv = 0, sa = 0, nv = 0, fe = 0;
    // 32-word groups interleaved over the blocks, claimed by the block's warps
    const int ngroups = (P.W + 31) / 32;
    for (;;) {
        int k = 0;
        if (lane == 0) k = atomicAdd(grab, 1);
        k = __shfl_sync(FULL_MASK, k, 0);
        const int grp = (int)blockIdx.x + k * (int)gridDim.x;
        if (grp >= ngroups) break;
        const int base = grp * 32;
        const int w = base + lane;
        unsigned vis = 0u, unv = 0u;
        if (w < P.W) {
            vis = P.Vc[w];
            unv = ~vis & __ldg(&P.nz[w]);
            if (w == P.W - 1 && tail) unv &= (1u << tail) - 1u;
        }
        const unsigned f = direct ? bu_probe_direct(P, Fc, base, unv, sv, sa)
                                  : bu_probe_compact(P, Fc, base, unv, found, sv, sa);
        finalize_group<SIGMA>(P, st, acc, base, vis | f, vis, true, ell, bn, slot, nv, fe);
    }
    sv = warp_sum(sv);
    sa = warp_sum(sa);
    if (lane == 0 && sv) {
        atomicAdd(&acc->sv, sv);
        atomicAdd(&acc->sa, sa);
    }
    block_flush(P, st, acc, P.Q[bn], P.SQ[bn], slot, nv, fe);
}

// -------------------------------------------------------- mode decision
// Called by a full warp; all lanes return the same choice (a mode, or for the
// learned policy one of its BLEST_NUM_CHOICES mode / VSS-batch choices).
// Every block evaluates it on the same inputs, so every block picks the same.
template <bool TC_OK>
__device__ __forceinline__ int decide_mode(const BfsParams &P, int ell, long long frontier, long long fedges,
                                           long long unvisited, long long slots, int qlen) {
    int mode;
    if (P.policy == BLEST_POLICY_LEARNED && P.mlp) {
        int c = mlp_choose_warp(P.mlp, frontier, fedges, unvisited, slots, ell, P.avg_deg);
        if (c < 0 || c >= MLP_OUT) c = BLEST_MODE_PUSH_EAGER_CC;
        // layouts without the Fig. 3 fragment run the CUDA-core twin of a tensor-core choice
        if (!TC_OK) c = (c == 1) ? 0 : (c == 3) ? 2 : (c == 7) ? 5 : (c == 8) ? 6 : c;
        return c;
    }
    if (P.policy == BLEST_POLICY_FIXED) {
        mode = P.fixed_mode;
    } else if (P.policy == BLEST_POLICY_SCHEDULE && P.sched_len > 0) {
        mode = P.schedule[(ell - 1) % P.sched_len];
    } else {
        // §5.2/§7.1: lazy updates when U_div exceeds the threshold; Eq. 5
        // switches to bottom-up when #unvisited < eta * |Q_curr|.
        mode = P.lazy ? (P.tc ? BLEST_MODE_PUSH_LAZY_TC : BLEST_MODE_PUSH_LAZY_CC)
                      : (P.tc ? BLEST_MODE_PUSH_EAGER_TC : BLEST_MODE_PUSH_EAGER_CC);
        if (P.switching && (double)unvisited < (double)P.eta * (double)qlen) mode = BLEST_MODE_BOTTOM_UP;
    }
    if (mode < 0 || mode >= BLEST_NUM_MODES) mode = BLEST_MODE_PUSH_EAGER_CC;
    // layouts without the Fig. 3 fragment run the CUDA-core twin of a tensor-core mode
    if (!TC_OK && mode == BLEST_MODE_PUSH_EAGER_TC) mode = BLEST_MODE_PUSH_EAGER_CC;
    if (!TC_OK && mode == BLEST_MODE_PUSH_LAZY_TC) mode = BLEST_MODE_PUSH_LAZY_CC;
    return mode;
}

// Buffers of level ell-2 are cleared sparsely and the counters of level
// ell+1 zeroed.  Runs after the level's stage-1 work, on the grid's last
// threads, so it stays off the path of the warps that own queue entries.
template <int SIGMA>
__device__ __forceinline__ void housekeeping(const BfsParams &P, int ell, int bo, int sql, int sz, int tid,
                                             int nthreads) {
    Ctl *ctl = P.ctl;
    const int rt = nthreads - 1 - tid;
    if (ell >= 2) {
        unsigned *Fo = P.F[bo];
        const int *SQo = P.SQ[bo];
        for (int k = rt; k < sql; k += nthreads) clear_field<SIGMA>(Fo, SQo[k]);
    }
    if (rt == 0) {
        ctl->qlen[sz] = 0;
        ctl->sqlen[sz] = 0;
        ctl->xq[sz] = 0;
        ctl->newv[sz] = 0;
        ctl->fedges[sz] = 0;
        ctl->scan_v[sz] = 0;
        ctl->scan_a[sz] = 0;
    }
}

template <bool EAGER, int SIGMA, int LPV>
__device__ __forceinline__ void push_dispatch(const BfsParams &P, Stage &st, int *grab, BlkAcc *acc, bool tc, int ell,
                                              int bc, int bn, int sn, int qlen, unsigned bsel, int batch = 1) {
    // eager levels run one pass at a time (their atomics and loads already
    // overlap within a pass, and a second pass's state would not fit the
    // 64-register budget of a 1024-thread CTA); lazy levels keep 1, 2 or 4.
    // A tensor-core level runs the Fig. 3 layout, or the 16-MMA one when the
    // handle's engine asks for it.
    if constexpr (EAGER) {
        if constexpr (Lay<SIGMA, LPV>::TC_OK) {
            if (tc && P.tc16) { push_level<true, 2, 1, SIGMA, LPV>(P, st, grab, acc, ell, bc, bn, sn, qlen, bsel); return; }
            if (tc) { push_level<true, 1, 1, SIGMA, LPV>(P, st, grab, acc, ell, bc, bn, sn, qlen, bsel); return; }
        }
        push_level<true, 0, 1, SIGMA, LPV>(P, st, grab, acc, ell, bc, bn, sn, qlen, bsel);
    } else {
        if constexpr (Lay<SIGMA, LPV>::TC_OK) {
            if (tc && P.tc16) { push_level<false, 2, 1, SIGMA, LPV>(P, st, grab, acc, ell, bc, bn, sn, qlen, bsel); return; }
            if (tc) {
                if (batch >= 4) push_level<false, 1, 4, SIGMA, LPV>(P, st, grab, acc, ell, bc, bn, sn, qlen, bsel);
                else if (batch >= 2) push_level<false, 1, 2, SIGMA, LPV>(P, st, grab, acc, ell, bc, bn, sn, qlen, bsel);
                else push_level<false, 1, 1, SIGMA, LPV>(P, st, grab, acc, ell, bc, bn, sn, qlen, bsel);
                return;
            }
        }
        if (batch >= 4) push_level<false, 0, 4, SIGMA, LPV>(P, st, grab, acc, ell, bc, bn, sn, qlen, bsel);
        else if (batch >= 2) push_level<false, 0, 2, SIGMA, LPV>(P, st, grab, acc, ell, bc, bn, sn, qlen, bsel);
        else push_level<false, 0, 1, SIGMA, LPV>(P, st, grab, acc, ell, bc, bn, sn, qlen, bsel);
    }
}

// One register budget for every CTA size: 64 a thread (1024 threads per
// SM).  Measured on GB300, 16 resident warps at 128 registers were 20-50 %
// slower and 48 warps at 40 registers (heavy spilling) up to 40 % slower on
// the road-like grid: the kernel is latency-bound and 32 warps is the best
// trade.
template <int SIGMA, int LPV>
__global__ void __launch_bounds__(BFS_MAX_THREADS, 1) k_bfs(const BfsParams Pk) {
    using LY = Lay<SIGMA, LPV>;
    __shared__ unsigned s_found[BFS_MAX_THREADS];
    __shared__ float s_mlp[MLP_NW];
    extern __shared__ __align__(16) unsigned char s_stage[];   // STG_BYTES per warp
    // The parameters live in shared memory for the whole launch: the level
    // functions take them by reference and index the buffer rings (F, Q, SQ)
    // with the level, which would otherwise place a copy of the struct in
    // local memory and turn every field read into a local load.
    __shared__ BfsParams s_par;
    if (threadIdx.x == 0) {
        s_par = Pk;
        if (Pk.policy == BLEST_POLICY_LEARNED && Pk.mlp) s_par.mlp = s_mlp;
    }
    if (Pk.policy == BLEST_POLICY_LEARNED && Pk.mlp) mlp_stage_weights(Pk.mlp, s_mlp);
    __syncthreads();
    const BfsParams &P = s_par;
    const int tid = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int nthreads = (int)(gridDim.x * blockDim.x);
    const int lane = lane_id();
    const unsigned bsel = (lane % 9 == 0) ? 1u : ((lane % 9 == 4) ? 256u : 0u);
    Ctl *ctl = P.ctl;
    unsigned epoch = 0;
    Stage st;
    st.q = reinterpret_cast<int2 *>(s_stage + (size_t)(threadIdx.x >> 5) * STG_BYTES);
    st.sq = reinterpret_cast<int *>(s_stage + (size_t)(threadIdx.x >> 5) * STG_BYTES + STG_Q * 8);
    st.qn = 0;
    st.sqn = 0;
    st.defer = 0;
    st.qdef = 0;
    __shared__ int s_mode;
    __shared__ long long s_lvl[5];
    __shared__ int s_grab[3];   // per-level work claims: push passes, stage-2 groups, bottom-up groups
    __shared__ BlkAcc s_acc;    // per-level CTA totals for the last flush

    // ---- level 0 (Algorithm 2/3 init): L = inf except the source, frontier
    // and visited bits hold the source, Q = VSSs of the source's slice set.
    const int src = P.new_of_old ? __ldg(&P.new_of_old[P.src]) : P.src;
    if ((reinterpret_cast<uintptr_t>(P.L) & 15u) == 0) {   // 16-byte stores where aligned
        const long long n4 = P.n & ~3;
        const int4 m1 = make_int4(-1, -1, -1, -1);
        for (long long i = (long long)tid * 4; i < n4; i += (long long)nthreads * 4) {
            int4 v = m1;
            if (src >= i && src < i + 4) {
                if (src == i) v.x = 0; else if (src == i + 1) v.y = 0; else if (src == i + 2) v.z = 0; else v.w = 0;
            }
            reinterpret_cast<int4 *>(P.L + i)[0] = v;
        }
        for (long long i = n4 + tid; i < P.n; i += nthreads) P.L[i] = (i == src) ? 0 : -1;
    } else {
        for (int i = tid; i < P.n; i += nthreads) P.L[i] = (i == src) ? 0 : -1;
    }
    for (int w = tid; w < P.W; w += nthreads) {
        const unsigned b = (w == (src >> 5)) ? (1u << (src & 31)) : 0u;
        P.Vc[w] = b;
        P.Vn[w] = b;
        P.F[0][w] = b;
        P.F[1][w] = 0u;
        P.F[2][w] = 0u;
    }
    {
        const int ss = src >> LY::LOGS;
        const int a = __ldg(&P.realPtrs[ss]), e = __ldg(&P.realPtrs[ss + 1]);
        for (int k = tid; k < e - a; k += nthreads) P.Q[0][k] = make_int2(a + k, ss);
        if (tid == 0) {
            P.SQ[0][0] = ss;
            ctl->qlen[0] = e - a;
            ctl->sqlen[0] = 1;
            ctl->newv[0] = 1;
            ctl->fedges[0] = (unsigned long long)__ldg(&P.deg[src]);
        }
    }
    if (!grid_barrier(ctl, epoch, P.budget_ns)) return;

    long long visited = 0;
    int ell = 1;
    for (;; ++ell) {
        const int bc = (ell - 1) % 3, bn = ell % 3, bo = (ell + 1) % 3;
        const int sc = (ell - 1) & 3, sn = ell & 3, so = (ell + 2) & 3, sz = (ell + 1) & 3;
        // One warp per block reads the level's counters (every thread reading the
        // same control-block words would pile ~20K requests onto one L2 line),
        // decides the mode and publishes both through shared memory.
        if (threadIdx.x < 32) {
            long long c4[5] = {0, 0, 0, 0, 0};
            if (threadIdx.x == 0) {
                c4[0] = ld_volatile_i32(&ctl->qlen[sc]);
                c4[1] = (long long)*(volatile unsigned long long *)&ctl->newv[sc];
                c4[2] = (long long)*(volatile unsigned long long *)&ctl->fedges[sc];
                c4[3] = ell >= 2 ? ld_volatile_i32(&ctl->sqlen[so]) : 0;
                c4[4] = ld_volatile_i32(&ctl->sqlen[sc]);
            }
#pragma unroll
            for (int i = 0; i < 5; ++i) c4[i] = __shfl_sync(FULL_MASK, c4[i], 0);
            const long long unv = (long long)P.n - (visited + c4[1]);
            const int m = c4[0] > 0 ? decide_mode<LY::TC_OK>(P, ell, c4[1], c4[2], unv, c4[0] * LY::TAU,
                                                             (int)c4[0])
                                    : 0;
            if (threadIdx.x == 0) {
                s_lvl[0] = c4[0];
                s_lvl[1] = c4[1];
                s_lvl[2] = c4[2];
                s_lvl[3] = c4[3];
                s_lvl[4] = c4[4];
                s_mode = m;
                s_grab[0] = 0;
                s_grab[1] = 0;
                s_grab[2] = 0;
                s_acc.q = 0;
                s_acc.s = 0;
                s_acc.nv = 0;
                s_acc.fe = 0;
                s_acc.sv = 0;
                s_acc.sa = 0;
            }
        }
        __syncthreads();
        const int qlen = (int)s_lvl[0];
        const long long frontier = s_lvl[1];
        const long long fedges = s_lvl[2];
        const int sql_old = (int)s_lvl[3];
        const int sql_cur = (int)s_lvl[4];
        const int choice = s_mode;
        const int mode = mlp_choice_mode(choice);
        // VSS passes in flight: the learned choice's, else the launch's setting
        const int batch = (P.policy == BLEST_POLICY_LEARNED && P.mlp) ? mlp_choice_batch(choice) : P.batch;
        __syncthreads();   // s_lvl / s_mode are rewritten at the next level start
        visited += frontier;
        const long long unvisited = (long long)P.n - visited;
        const bool logger = blockIdx.x == 0 && threadIdx.x == 32;
        if (logger) {
            const long long t = (long long)global_ns();
            if (ell >= 2 && ell - 2 < P.log_cap) {
                blest_level_log &prev = P.log[ell - 2];
                prev.t_ns = t - prev.t_ns;
                if (prev.mode == BLEST_MODE_PUSH_EAGER_CC || prev.mode == BLEST_MODE_PUSH_EAGER_TC ||
                    prev.mode == BLEST_MODE_BOTTOM_UP)
                    prev.t_stage1_ns = prev.t_ns;
                prev.scanned_vertices = (long long)*(volatile unsigned long long *)&ctl->scan_v[sc];
                prev.scanned_arcs = (long long)*(volatile unsigned long long *)&ctl->scan_a[sc];
            }
            if (qlen > 0 && ell - 1 < P.log_cap) {
                blest_level_log rec;
                rec.level = ell;
                rec.mode = mode;
                rec.frontier = frontier;
                rec.frontier_edges = fedges;
                rec.unvisited = unvisited;
                rec.queue = qlen;
                rec.t_ns = t;
                rec.scanned_vertices = 0;
                rec.scanned_arcs = 0;
                rec.slots = (long long)qlen * LY::TAU;
                rec.t_stage1_ns = 0;
                rec.vss_batch = (mode == BLEST_MODE_BOTTOM_UP) ? 0
                              : (mode == BLEST_MODE_PUSH_EAGER_CC || mode == BLEST_MODE_PUSH_EAGER_TC) ? 1 : batch;
                P.log[ell - 1] = rec;
            }
        }
        if (qlen == 0) break;

        // A top-down level after a level that deferred its VSS queue writes
        // the queue first (one pass over the slice-set queue and a barrier).
        if (st.defer && mode != BLEST_MODE_BOTTOM_UP) {
            expand_queue(P, bc, sc, sql_cur);
            if (!grid_barrier(ctl, epoch, P.budget_ns)) return;
        }
        // Lazy and bottom-up levels of graphs with bottom-up switching defer
        // their VSS queue: the level after them is most often bottom-up,
        // which reads only the frontier bits.
        st.defer = P.defer_queue && (mode == BLEST_MODE_BOTTOM_UP || mode == BLEST_MODE_PUSH_LAZY_CC ||
                                     mode == BLEST_MODE_PUSH_LAZY_TC);

        if (mode == BLEST_MODE_PUSH_EAGER_CC || mode == BLEST_MODE_PUSH_EAGER_TC) {
            push_dispatch<true, SIGMA, LPV>(P, st, &s_grab[0], &s_acc, mode == BLEST_MODE_PUSH_EAGER_TC, ell, bc, bn, sn, qlen, bsel);
            housekeeping<SIGMA>(P, ell, bo, sql_old, sz, tid, nthreads);
            if (!grid_barrier(ctl, epoch, P.budget_ns)) return;
        } else if (mode == BLEST_MODE_BOTTOM_UP) {
            // direct probes while at least a quarter of the vertices are unvisited
            bottom_up_level<SIGMA>(P, st, &s_grab[2], &s_acc, ell, bc, bn, sn, s_found, unvisited * 4 >= (long long)P.n);
            housekeeping<SIGMA>(P, ell, bo, sql_old, sz, tid, nthreads);
            if (!grid_barrier(ctl, epoch, P.budget_ns)) return;
        } else {
            {
                push_dispatch<false, SIGMA, LPV>(P, st, &s_grab[0], &s_acc, mode == BLEST_MODE_PUSH_LAZY_TC, ell, bc, bn, sn, qlen,
                                                 bsel, batch);
            }
            housekeeping<SIGMA>(P, ell, bo, sql_old, sz, tid, nthreads);
            if (!grid_barrier(ctl, epoch, P.budget_ns)) return;
            if (logger && ell - 1 < P.log_cap)
                P.log[ell - 1].t_stage1_ns = (long long)global_ns() - P.log[ell - 1].t_ns;
            finalize_level<SIGMA>(P, st, &s_grab[1], &s_acc, ell, bn, sn);
            if (!grid_barrier(ctl, epoch, P.budget_ns)) return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->nlevels = ell - 1;
    // undo the reordering: out[v] = L[new_of_old[v]].  Eight vertices a
    // thread per step: two 16-byte loads of the permutation, then eight
    // independent gathers, so each thread pays the gather latency once per
    // eight vertices rather than once per vertex.
    if (P.new_of_old) {
        const bool vec = (reinterpret_cast<uintptr_t>(P.out) & 15u) == 0;
        const long long n8 = P.n & ~7;
        for (long long v0 = (long long)tid * 8; v0 < n8; v0 += (long long)nthreads * 8) {
            const int4 pa = __ldg(reinterpret_cast<const int4 *>(P.new_of_old + v0));
            const int4 pb = __ldg(reinterpret_cast<const int4 *>(P.new_of_old + v0) + 1);
            const int4 ga = make_int4(P.L[pa.x], P.L[pa.y], P.L[pa.z], P.L[pa.w]);
            const int4 gb = make_int4(P.L[pb.x], P.L[pb.y], P.L[pb.z], P.L[pb.w]);
            if (vec) {
                reinterpret_cast<int4 *>(P.out + v0)[0] = ga;
                reinterpret_cast<int4 *>(P.out + v0)[1] = gb;
            } else {
                P.out[v0] = ga.x; P.out[v0 + 1] = ga.y; P.out[v0 + 2] = ga.z; P.out[v0 + 3] = ga.w;
                P.out[v0 + 4] = gb.x; P.out[v0 + 5] = gb.y; P.out[v0 + 6] = gb.z; P.out[v0 + 7] = gb.w;
            }
        }
        for (long long v = n8 + tid; v < P.n; v += nthreads) P.out[v] = P.L[__ldg(&P.new_of_old[v])];
    }
}

// the kernel instance of a (sigma, tau) layout (nullptr for other pairs)
const void *bfs_kernel_for(int sigma, int tau, int /*block*/) {
    if (sigma == 8 && tau == 128) return (const void *)k_bfs<8, 32>;
    if (sigma == 8 && tau == 32) return (const void *)k_bfs<8, 8>;
    if (sigma == 16 && tau == 64) return (const void *)k_bfs<16, 32>;
    if (sigma == 32 && tau == 32) return (const void *)k_bfs<32, 32>;
    return nullptr;
}

}  // namespace

// dynamic shared memory of a k_bfs launch: the warps' queue staging areas
static size_t bfs_smem(int block) { return (size_t)(block / 32) * STG_BYTES; }

static int bfs_grid_for_layout(int sigma, int tau, int block, int *num_sms) {
    const void *kern = bfs_kernel_for(sigma, tau, block);
    if (!kern) return 0;
    int dev = 0;
    cudaGetDevice(&dev);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bfs_smem(block)) != cudaSuccess)
        return 0;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, bfs_smem(block));
    if (num_sms) *num_sms = sms;
    return per_sm * sms;
}

int bfs_grid_for(const blest_graph *h, int block, int *num_sms) {
    return bfs_grid_for_layout(h->sigma, h->tau, block, num_sms);
}

// nz[w] bit b set iff vertex 32w+b has an in-neighbour (a nonempty row of
// the in-neighbour CSR); bottom-up levels never probe the others.
__global__ void k_nz_mask(const long long *__restrict__ rp, int n, int W, unsigned *nz) {
    const int stride = gridDim.x * blockDim.x;
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < W; w += stride) {
        unsigned m = 0;
        for (int b = 0; b < 32; ++b) {
            const int u = (w << 5) + b;
            if (u < n && rp[u + 1] > rp[u]) m |= 1u << b;
        }
        nz[w] = m;
    }
}

blest_status bfs_prepare(blest_graph *h) {
    const int64_t n = h->n;
    const int64_t W = (n + 31) / 32;
    blest_status bs;
    if ((bs = dev_alloc_t(h, &h->w.L, (size_t)n)) != BLEST_OK) return bs;
    if ((bs = dev_alloc_t(h, &h->w.Vc, (size_t)W + 1)) != BLEST_OK) return bs;
    if ((bs = dev_alloc_t(h, &h->w.Vn, (size_t)W + 1)) != BLEST_OK) return bs;
    for (int i = 0; i < 3; ++i) {
        if ((bs = dev_alloc_t(h, &h->w.F[i], (size_t)W + 1)) != BLEST_OK) return bs;
        if ((bs = dev_alloc_t(h, &h->w.Q[i], (size_t)(h->Nv > 0 ? h->Nv : 1))) != BLEST_OK) return bs;  // int2
        if ((bs = dev_alloc_t(h, &h->w.SQ[i], (size_t)h->Ns + 1)) != BLEST_OK) return bs;
    }
    if ((bs = dev_alloc_t(h, &h->w.ctl, 1)) != BLEST_OK) return bs;
    if ((bs = dev_alloc_t(h, &h->g.nz, (size_t)W + 1)) != BLEST_OK) return bs;
    k_nz_mask<<<(unsigned)((W + 255) / 256 < 65535 ? (W + 255) / 256 : 65535), 256, 0, h->stream>>>(
        h->g.rp, (int)n, (int)W, h->g.nz);
    if (cudaGetLastError() != cudaSuccess) return BLEST_ERR_CUDA;
    h->w.log_cap = 1 << 16;
    if ((bs = dev_alloc_t(h, &h->w.log, (size_t)h->w.log_cap)) != BLEST_OK) return bs;
    if (h->g.new_of_old)
        if ((bs = dev_alloc_t(h, &h->w.out_tmp, (size_t)n)) != BLEST_OK) return bs;
    int sms = 0;
    h->grid = bfs_grid_for(h, h->block, &sms);
    h->num_sms = sms;
    if (h->grid <= 0) return BLEST_ERR_CUDA;
    return BLEST_OK;
}

// Enqueue one BFS on h->stream; levels (original ids) land in dev_out.
blest_status bfs_run(blest_graph *h, int32_t source, int32_t *dev_out) {
    BfsParams P;
    memset(&P, 0, sizeof P);
    P.n = (int)h->n;
    P.W = (int)((h->n + 31) / 32);
    const void *kern = bfs_kernel_for(h->sigma, h->tau, h->block);
    if (!kern) return BLEST_ERR_INTERNAL;
    P.rowIds = h->g.rowIds;
    P.masks = h->g.masks;
    P.realPtrs = h->g.realPtrs;
    P.v2r = h->g.v2r;
    P.rp = h->g.rp;
    P.col = h->g.col;
    P.deg = h->g.deg;
    P.Vc = h->w.Vc;
    P.Vn = h->w.Vn;
    for (int i = 0; i < 3; ++i) {
        P.F[i] = h->w.F[i];
        P.Q[i] = h->w.Q[i];
        P.SQ[i] = h->w.SQ[i];
    }
    P.ctl = h->w.ctl;
    P.log = h->w.log;
    P.log_cap = h->w.log_cap;
    P.policy = h->policy;
    P.fixed_mode = h->fixed_mode;
    P.lazy = h->lazy;
    P.tc = h->engine_tc != 0;
    P.tc16 = h->engine_tc == 2;
    P.switching = h->switching;
    P.defer_queue = h->defer_queue < 0 ? h->switching : h->defer_queue;
    P.eta = h->eta;
    P.schedule = h->d_schedule;
    P.sched_len = h->sched_len;
    P.mlp = h->d_mlp;
    P.nz = h->g.nz;
    P.head = h->g.head;
    P.batch = h->vss_batch;
    P.avg_deg = h->n ? (float)((double)h->nnz / (double)h->n) : 0.f;
    P.budget_ns = (unsigned long long)h->timeout_ms * 1000000ull;
    P.src = source;
    if (h->g.new_of_old) {
        P.L = h->w.out_tmp;
        P.new_of_old = h->g.new_of_old;
        P.out = dev_out;
    } else {
        P.L = dev_out;
    }
    cudaError_t e = cudaMemsetAsync(h->w.ctl, 0, sizeof(Ctl), h->stream);
    if (e != cudaSuccess) return BLEST_ERR_CUDA;
    void *args[] = {&P};
    e = cudaLaunchCooperativeKernel(kern, dim3(h->grid), dim3(h->block), args, bfs_smem(h->block), h->stream);
    if (e != cudaSuccess) {
        blest_internal_record_cuda_error(e, "cudaLaunchCooperativeKernel(k_bfs)", __FILE__, __LINE__);
        return BLEST_ERR_CUDA;
    }
    return BLEST_OK;
}

// ------------------------------------------------------------------------
// Allocation-free single-source BFS (blest_bfs_noalloc in blest.h).
//
// Some callers cannot allocate device memory: a framework that reserves the
// whole device pool for its own allocator up front, or a latency-critical
// path where cudaMalloc's implicit device synchronisation is not allowed.
// This entry point runs the same persistent kernel (k_bfs) as blest_bfs, but
// its scratch -- visited and frontier bitvectors, the three VSS and
// slice-set queues and the control block -- lives in the file-scope array
// below, so the call allocates nothing.  The array is part of the library's
// device image: every GPU that loads the library holds it (about 5.3 MB)
// until the process exits.  All calls share it and it keeps the last call's
// contents; the kernel rewrites every bitvector and queue it reads and the
// control block is cleared before each launch.  Calls that overlap on the
// GPU (different streams, or different host threads) race on the array.
// ------------------------------------------------------------------------
namespace {

constexpr long long NOALLOC_MAX_N = 1ll << 20;     // vertices
constexpr long long NOALLOC_MAX_NV = 1ll << 17;    // VSSs
constexpr long long NOALLOC_W = NOALLOC_MAX_N / 32;           // bitvector words
constexpr long long NOALLOC_NS = NOALLOC_MAX_N / 8 + 1;       // slice sets + 1
constexpr size_t NOALLOC_CTL_BYTES = 256;
constexpr size_t NOALLOC_BITS_BYTES = 5ull * (NOALLOC_W + 1) * 4;
constexpr size_t NOALLOC_Q_BYTES = 3ull * NOALLOC_MAX_NV * 8;   // int2 queue entries
constexpr size_t NOALLOC_SQ_BYTES = 3ull * NOALLOC_NS * 4;
// every sub-array starts on a 256-byte boundary (11 arrays after the control block)
constexpr size_t NOALLOC_BYTES = NOALLOC_CTL_BYTES + NOALLOC_BITS_BYTES + NOALLOC_Q_BYTES + NOALLOC_SQ_BYTES + 12 * 256;
static_assert(sizeof(Ctl) <= NOALLOC_CTL_BYTES, "control block fits its slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
unsigned char *g_noalloc_addr[NOALLOC_MAX_DEVICES];   // device address per device ordinal
int g_noalloc_grid[NOALLOC_MAX_DEVICES];

std::mutex g_noalloc_mu;   // guards the per-device set-up above

// Once per device, with that device current: the host-side symbol is only a
// stand-in, so look up the array's device address.
blest_status noalloc_setup(int dev, unsigned char **base, int *grid) {
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return BLEST_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            blest_internal_record_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
            return BLEST_ERR_CUDA;
        }
        int sms = 0;
        const int g = bfs_grid_for_layout(8, 128, 512, &sms);
        if (g <= 0) return BLEST_ERR_CUDA;
        g_noalloc_grid[dev] = g;
        g_noalloc_addr[dev] = (unsigned char *)p;
    }
    *base = g_noalloc_addr[dev];
    *grid = g_noalloc_grid[dev];
    return BLEST_OK;
}

}  // namespace

extern "C" blest_status blest_bfs_noalloc(const blest_bvss_view *g, int32_t source, int32_t *levels,
                                          void *stream) {
    if (!g || !levels || !g->row_ids || !g->masks || !g->real_ptrs || !g->virtual_to_real || !g->out_degree)
        return BLEST_ERR_INVALID;
    if (g->n < 1 || g->num_vss < 0 || g->num_slice_sets != (g->n + 7) / 8) return BLEST_ERR_INVALID;
    // the kernel instance below reads rowIds at a stride of 128 per VSS
    if (g->sigma != 8 || g->tau != 128) return BLEST_ERR_UNSUPPORTED;
    if (g->n > NOALLOC_MAX_N || g->num_vss > NOALLOC_MAX_NV) return BLEST_ERR_UNSUPPORTED;
    if (source < 0 || (int64_t)source >= g->n) return BLEST_ERR_INVALID;
    if (!is_device_ptr(levels)) return BLEST_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BLEST_ERR_CUDA;
    unsigned char *base = nullptr;
    int grid = 0;
    blest_status st = noalloc_setup(dev, &base, &grid);
    if (st != BLEST_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    const long long n = g->n, W = (n + 31) / 32, Ns = g->num_slice_sets;
    const long long nv = g->num_vss > 0 ? g->num_vss : 1;
    // carve the scratch: control block, 5 bitvectors, 3 queues of 8-byte
    // entries, 3 slice-set queues, each on a 256-byte boundary
    size_t off = 0;
    auto carve = [&](size_t bytes) -> unsigned char * {
        unsigned char *q = base + off;
        off = (off + bytes + 255) & ~(size_t)255;
        return q;
    };
    Ctl *ctl = (Ctl *)carve(NOALLOC_CTL_BYTES);
    BfsParams P;
    memset(&P, 0, sizeof P);
    P.Vc = (unsigned *)carve((size_t)(W + 1) * 4);
    P.Vn = (unsigned *)carve((size_t)(W + 1) * 4);
    for (int i = 0; i < 3; ++i) P.F[i] = (unsigned *)carve((size_t)(W + 1) * 4);
    for (int i = 0; i < 3; ++i) P.Q[i] = (int2 *)carve((size_t)nv * 8);
    for (int i = 0; i < 3; ++i) P.SQ[i] = (int *)carve((size_t)(Ns + 1) * 4);
    if (off > NOALLOC_BYTES) return BLEST_ERR_INTERNAL;
    P.n = (int)n;
    P.W = (int)W;
    P.rowIds = g->row_ids;
    P.masks = g->masks;
    P.realPtrs = g->real_ptrs;
    P.v2r = g->virtual_to_real;
    P.rp = nullptr;              // bottom-up levels are never chosen: fixed top-down mode
    P.col = nullptr;
    P.deg = g->out_degree;
    P.L = levels;
    P.ctl = ctl;
    P.log = nullptr;
    P.log_cap = 0;
    P.src = source;
    P.policy = BLEST_POLICY_FIXED;
    P.fixed_mode = g->engine_tc ? BLEST_MODE_PUSH_EAGER_TC : BLEST_MODE_PUSH_EAGER_CC;
    P.eta = 10.f;
    P.budget_ns = 5000ull * 1000000ull;
    P.new_of_old = nullptr;
    P.out = nullptr;
    if (cudaMemsetAsync(ctl, 0, sizeof(Ctl), s) != cudaSuccess) return BLEST_ERR_CUDA;
    void *args[] = {&P};
    cudaError_t e =
        cudaLaunchCooperativeKernel(bfs_kernel_for(8, 128, 512), dim3(grid), dim3(512), args, bfs_smem(512), s);
    if (e != cudaSuccess) {
        blest_internal_record_cuda_error(e, "cudaLaunchCooperativeKernel(k_bfs, no-alloc)", __FILE__, __LINE__);
        return BLEST_ERR_CUDA;
    }
    Ctl hc;
    if (cudaMemcpyAsync(&hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s) != cudaSuccess) return BLEST_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return BLEST_ERR_CUDA;
    return hc.err ? (blest_status)hc.err : BLEST_OK;
}
