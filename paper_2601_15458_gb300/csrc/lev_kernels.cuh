// Bit-vector Levenshtein kernels (A2 match masks, A3 distance).
//
// Column j of the edit-distance matrix D of a (rows) against b (columns) is
// held as vertical deltas D[i][j] - D[i-1][j] in {-1, 0, +1}, one bit per
// row in two masks Pv (+1) and Mv (-1) (Myers 1999, "A fast bit-vector
// algorithm for approximate string matching based on dynamic programming";
// global-distance form after Hyyro 2001).  With Eq the rows whose symbol
// equals b_j, the horizontal deltas of column j follow from
//     Xh = (((Eq & Pv) + Pv) ^ Pv) | Eq        (one carry chain over all rows)
//     Ph = Mv | ~(Xh | Pv),  Mh = Pv & Xh
// and the next vertical deltas from the horizontal ones shifted down a row,
// with row 0 contributing +1 (D[0][j] = j):
//     Pv' = Mh<< | ~(Xv | Ph<<),  Mv' = Ph<< & Xv,  Xv = Eq | Mv.
// The carry of the addition out of row i equals Mh[i], so a vector longer
// than one 32-bit word is handled by feeding the top bit of the previous
// word's Mh into the next word's addition and both top bits into its shifts.
// After the last column, D[m][n] = n + popc(Pv) - popc(Mv) over rows 1..m.
//
// Rows beyond m (padding up to the kernel's word capacity) never influence
// rows <= m: information only moves to higher rows.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "carry_chain.cuh"
#include "msa_internal.cuh"

namespace msa {

constexpr unsigned kFull = 0xffffffffu;

struct LevArgs {
    const uint32_t *planes;   // bit planes of the arena
    const uint8_t *codes;     // byte codes of the arena
    const int64_t *offs;      // [n_seqs + 1]
    const int32_t *sorted_t;  // targets, grouped by query
    const int32_t *sorted_p;  // original pair id of each grouped entry
    const int32_t *qstart;    // [n_seqs + 1] group starts
    int32_t *qcursor;         // [n_seqs] next entry to hand out, per query
    const int2 *tasks;        // all tasks, bucket-major
    const int32_t *boff;      // [NB] first task of each bucket
    const int32_t *bcount;    // [NB] tasks per bucket
    int32_t *bcounter;        // [NB] tasks handed out per bucket
    const int32_t *bsum;      // [NB] targets per bucket (slot kernels)
    int32_t *d_out;
    int32_t *err;
    int32_t bucket;
};

// 32 match bits of the query for rows 32k+1 .. 32k+32 and every symbol c.
// planes: B bit planes per 32-position arena word.  Bits for rows > m are 0.
template <int B>
__device__ __forceinline__ void query_planes(const uint32_t *__restrict__ planes, int64_t qpos, int m,
                                             int k, uint32_t (&pl)[B], uint32_t &mask) {
    const int rem = m - 32 * k;
    if (rem <= 0) {
        mask = 0u;
#pragma unroll
        for (int p = 0; p < B; ++p) pl[p] = 0u;
        return;
    }
    mask = rem >= 32 ? kFull : ((1u << rem) - 1u);
    const int64_t bit = qpos + 32 * (int64_t)k;
    const int64_t wi = bit >> 5;
    const int r = (int)(bit & 31);
#pragma unroll
    for (int p = 0; p < B; ++p) {
        uint32_t lo = __ldg(planes + wi * B + p);
        uint32_t hi = __ldg(planes + (wi + 1) * B + p);
        pl[p] = __funnelshift_r(lo, hi, r);
    }
}

template <int B, int SIGMA>
__device__ __forceinline__ uint32_t match_mask(const uint32_t (&pl)[B], uint32_t mask, int c) {
    uint32_t eq = mask;
#pragma unroll
    for (int p = 0; p < B; ++p) eq &= ((c >> p) & 1) ? pl[p] : ~pl[p];
    return eq;
}

// Lane kernel match masks: [symbol][word], WC words padded to a stride of 4
// mod 8 words, so a 16-byte load of 4 words starts aligned and the 4 symbols'
// rows fall on disjoint bank groups (lanes of a warp reading different
// symbols never conflict; lanes reading the same symbol share a broadcast).
__host__ __device__ constexpr int lane_peq_stride(int WC) {
    return ((WC + 3) / 4 * 4) % 8 == 0 ? (WC + 3) / 4 * 4 + 4 : (WC + 3) / 4 * 4;
}

// shared memory of one warp of the lane kernel, in words: SLOTS mask tables
// and, with several slots, 4 * SLOTS + 4 words of slot bookkeeping (a
// multiple of 4, so every table stays 16-byte aligned)
__host__ __device__ constexpr int lane_smem_words(int WC, int SIGMA, int SLOTS) {
    return SLOTS * lane_peq_stride(WC) * SIGMA + (SLOTS > 1 ? 4 * SLOTS + 4 : 0);
}

// One column over WC words, in chunks of up to 8 words: the chunk's
// (Eq & Pv) + Pv additions run on the hardware carry chain (add.cc/addc), and
// the Ph shift by one takes the lower word's top bit by funnel shift.
//
// The carry into row i of the addition is Mh of row i - 1 (and the word's
// carry-in for its first row), so the shifted Mh vector is the carry-in
// vector sum ^ u ^ Pv, one logic op, and with it neither Mh nor Xh is formed
// (Ph = Mv | ~(Xh | Pv) = Mv | ~(sum | Pv | Eq)): 9 ops per word.
template <int WC>
__device__ __forceinline__ void lane_column_chain(const uint32_t *row, uint32_t (&Pv)[WC], uint32_t (&Mv)[WC]) {
    uint32_t cy = 0u, ph_prev = 0u;
#pragma unroll
    for (int k0 = 0; k0 < WC; k0 += 8) {
        constexpr int kMax = 8;
        const int len = WC - k0 < kMax ? WC - k0 : kMax;
        if (len == 8) {
            uint32_t eq[8], u[8], pv[8], s[8];
            const uint4 e0 = reinterpret_cast<const uint4 *>(row + k0)[0];
            const uint4 e1 = reinterpret_cast<const uint4 *>(row + k0)[1];
            eq[0] = e0.x; eq[1] = e0.y; eq[2] = e0.z; eq[3] = e0.w;
            eq[4] = e1.x; eq[5] = e1.y; eq[6] = e1.z; eq[7] = e1.w;
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                pv[w] = Pv[k0 + w];
                u[w] = eq[w] & pv[w];
            }
            cy = CarryChainIn<8>::add(s, u, pv, cy);
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                const int k = k0 + w;
                const uint32_t mhs = s[w] ^ u[w] ^ pv[w];
                const uint32_t ph = Mv[k] | ~(s[w] | pv[w] | eq[w]);
                const uint32_t phs = k == 0 ? (ph << 1) | 1u : __funnelshift_l(ph_prev, ph, 1);
                ph_prev = ph;
                const uint32_t xv = eq[w] | Mv[k];
                Pv[k] = mhs | ~(xv | phs);
                Mv[k] = phs & xv;
            }
        } else {
            // the tail of fewer than 8 words (WC % 8), same steps
#pragma unroll
            for (int w = 0; w < kMax; ++w) {
                if (w >= len) break;
                const int k = k0 + w;
                const uint32_t eq = row[k];
                const uint32_t pv = Pv[k];
                const uint32_t u = eq & pv;
                const uint64_t t = (uint64_t)u + pv + cy;
                const uint32_t sum = (uint32_t)t;
                cy = (uint32_t)(t >> 32);
                const uint32_t mhs = sum ^ u ^ pv;
                const uint32_t ph = Mv[k] | ~(sum | pv | eq);
                const uint32_t phs = k == 0 ? (ph << 1) | 1u : __funnelshift_l(ph_prev, ph, 1);
                ph_prev = ph;
                const uint32_t xv = eq | Mv[k];
                Pv[k] = mhs | ~(xv | phs);
                Mv[k] = phs & xv;
            }
        }
    }
}

// (Eq & Pv) + Pv + cin over N words on the carry chain, in chunks of at
// most 8 words; returns the carry out of the last word.
template <int N, int K0 = 0>
__device__ __forceinline__ uint32_t chain_add_all(uint32_t (&s)[N], const uint32_t (&u)[N], const uint32_t (&pv)[N],
                                                  uint32_t cy) {
    if constexpr (K0 >= N) {
        return cy;
    } else {
        constexpr int L = N - K0 < 8 ? N - K0 : 8;
        uint32_t ss[L], uu[L], pp[L];
#pragma unroll
        for (int i = 0; i < L; ++i) {
            uu[i] = u[K0 + i];
            pp[i] = pv[K0 + i];
        }
        cy = CarryChainIn<L>::add(ss, uu, pp, cy);
#pragma unroll
        for (int i = 0; i < L; ++i) s[K0 + i] = ss[i];
        return chain_add_all<N, K0 + L>(s, u, pv, cy);
    }
}

// One column over N consecutive words, 9 ops a word (the carry-in vector
// sum ^ u ^ Pv is Mh shifted down a row, see lane_column_chain).  ph_in and
// cin are the Ph bit and the addition carry (= Mh bit) of the row above the
// first word; ph_out and cout those of the last word's top row.
template <int N>
__device__ __forceinline__ void bv_column(const uint32_t (&eq)[N], uint32_t (&Pv)[N], uint32_t (&Mv)[N],
                                          uint32_t ph_in, uint32_t cin, uint32_t &ph_out, uint32_t &cout) {
    uint32_t u[N], sum[N], pv[N];
#pragma unroll
    for (int w = 0; w < N; ++w) {
        pv[w] = Pv[w];
        u[w] = eq[w] & pv[w];
    }
    cout = chain_add_all<N>(sum, u, pv, cin);
    uint32_t php = ph_in << 31;
#pragma unroll
    for (int w = 0; w < N; ++w) {
        const uint32_t mhs = sum[w] ^ u[w] ^ pv[w];
        const uint32_t ph = Mv[w] | ~(sum[w] | pv[w] | eq[w]);
        const uint32_t phs = __funnelshift_l(php, ph, 1);
        php = ph;
        const uint32_t xv = eq[w] | Mv[w];
        Pv[w] = mhs | ~(xv | phs);
        Mv[w] = phs & xv;
    }
    ph_out = php >> 31;
}

// bv_column with the boundary bits in place: the Ph bit of the row above is
// bit 31 of php_in, the carry into the first row is 1 iff cin != 0; on return
// bit 31 of php_out is the last row's Ph bit and cout its carry (Mh bit).
template <int N>
__device__ __forceinline__ void bv_column_raw(const uint32_t (&eq)[N], uint32_t (&Pv)[N], uint32_t (&Mv)[N],
                                              uint32_t php_in, uint32_t cin, uint32_t &php_out, uint32_t &cout) {
    uint32_t u[N], sum[N], pv[N];
#pragma unroll
    for (int w = 0; w < N; ++w) {
        pv[w] = Pv[w];
        u[w] = eq[w] & pv[w];
    }
    cout = chain_add_all<N>(sum, u, pv, cin);
    uint32_t php = php_in;
#pragma unroll
    for (int w = 0; w < N; ++w) {
        const uint32_t mhs = sum[w] ^ u[w] ^ pv[w];
        const uint32_t ph = Mv[w] | ~(sum[w] | pv[w] | eq[w]);
        const uint32_t phs = __funnelshift_l(php, ph, 1);
        php = ph;
        const uint32_t xv = eq[w] | Mv[w];
        Pv[w] = mhs | ~(xv | phs);
        Mv[w] = phs & xv;
    }
    php_out = php;
}

// d = a * b + c on the integer multiply-add pipe (used for bit packing that
// would otherwise take shifts and ORs on the logic pipe; b a power of two and
// a * b disjoint from c)
__device__ __forceinline__ uint32_t mad_u32(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// A warp whose index in the grid is past the bucket's task count leaves
// before claiming anything: a bucket with few tasks then keeps only its
// lowest blocks (their warps claim all its tasks from the counter), and the
// others free their SM slots at once, without a round of atomics on the
// bucket's counter, for the buckets running beside it on other streams.
__device__ __forceinline__ bool warp_has_no_task(int ntasks) {
    return (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5) >= ntasks;
}

__device__ __forceinline__ int next_task(int32_t *counter, int lane) {
    int t = 0;
    if (lane == 0) t = atomicAdd(counter, 1);
    return __shfl_sync(kFull, t, 0);
}

// ---------------------------------------------------------------------------
// Lane kernel: one warp per query, each lane streams its own targets.
// Match masks of the query live in shared memory, layout [c][k] with a padded
// stride (lane_peq_stride), read 4 words per load.  Pv/Mv: WC words in
// registers.
// SLOTS > 1 gives a warp up to SLOTS queries with few targets each, the
// masks of all of them in shared memory: lane l takes targets l, l + 32, ...
// of the concatenated target lists, so a batch of queries with 2..31 targets
// keeps the lanes busy, where a warp per query would leave most of them idle.
// ---------------------------------------------------------------------------
template <int WC, int B, int SIGMA, int SLOTS = 1>
__global__ void __launch_bounds__(128) lev_lane_kernel(LevArgs a) {
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31;
    constexpr int S = lane_peq_stride(WC);
    // per warp: SLOTS mask tables, then (SLOTS > 1) the slots' query, first
    // sorted target, length and prefix sums of their target counts
    uint32_t *sPeq = smem + (threadIdx.x >> 5) * lane_smem_words(WC, SIGMA, SLOTS);
    int32_t *sQ = (int32_t *)(sPeq + SLOTS * S * SIGMA);
    int32_t *sBeg = sQ + SLOTS, *sM = sBeg + SLOTS, *sPre = sM + SLOTS;
    const int nent = a.bcount[a.bucket];
    // queries per warp: as many as make about 32 targets (one per lane, so
    // no lane runs two targets one after another), 32 / (mean targets per
    // query), and all SLOTS once the bucket gives every resident warp that
    // many anyway (then lanes kept busy matter more than the length of one
    // warp's work)
    int ns = 1;
    if constexpr (SLOTS > 1) {
        const int resident = gridDim.x * (blockDim.x >> 5);
        const long long tot = max(1, a.bsum[a.bucket]);
        const long long per = 32ll * nent / tot;
        const int one_round = per < SLOTS ? (int)per : SLOTS;
        ns = max(1, max(one_round, min(SLOTS, nent / resident)));
    }
    const int ntasks = (nent + ns - 1) / ns;
    const int2 *tasks = a.tasks + a.boff[a.bucket];
    int32_t *counter = a.bcounter + a.bucket;

    if (warp_has_no_task(ntasks)) return;
    for (int task = next_task(counter, lane); task < ntasks; task = next_task(counter, lane)) {
        int q = -1, m = 0, cbeg = 0, cnt = 0, total = 0;
        const uint32_t *peq = sPeq;
        __syncwarp();
        if constexpr (SLOTS == 1) {
            q = tasks[task].x;
            const int64_t qpos = a.offs[q];
            m = (int)(a.offs[q + 1] - qpos);
            for (int k = lane; k < WC; k += 32) {
                uint32_t pl[B], mask;
                query_planes<B>(a.planes, qpos, m, k, pl, mask);
#pragma unroll
                for (int c = 0; c < SIGMA; ++c) sPeq[c * S + k] = match_mask<B, SIGMA>(pl, mask, c);
            }
            cbeg = a.qstart[q];
            cnt = a.qstart[q + 1] - cbeg;
        } else {
            // lane i < ns reads slot i; a slot past ns or the bucket's end is empty
            int cq = -1, cc = 0, cb = 0, cm = 0;
            const int ent = task * ns + lane;
            if (lane < ns && ent < nent) {
                cq = tasks[ent].x;
                cb = a.qstart[cq];
                cc = a.qstart[cq + 1] - cb;
                cm = (int)(a.offs[cq + 1] - a.offs[cq]);
            }
            int incl = cc;
#pragma unroll
            for (int o = 1; o < SLOTS; o <<= 1) {
                const int v = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane < SLOTS) {
                sQ[lane] = cq;
                sBeg[lane] = cb;
                sM[lane] = cm;
                sPre[lane + 1] = incl;
            }
            if (lane == 0) sPre[0] = 0;
            total = __shfl_sync(kFull, incl, SLOTS - 1);
            __syncwarp();
            for (int t = lane; t < SLOTS * WC; t += 32) {
                const int sl = t / WC, k = t - sl * WC;
                const int qs = sQ[sl];
                if (qs < 0) continue;
                const int64_t qpos = a.offs[qs];
                uint32_t pl[B], mask;
                query_planes<B>(a.planes, qpos, sM[sl], k, pl, mask);
                uint32_t *dst = sPeq + sl * (S * SIGMA);
#pragma unroll
                for (int c = 0; c < SIGMA; ++c) dst[c * S + k] = match_mask<B, SIGMA>(pl, mask, c);
            }
        }
        __syncwarp();

        // warp-synchronous stream: every iteration starts with a vote over
        // the whole warp, so lanes that switch targets rejoin the others
        // before the next column instead of running it separately
        uint32_t Pv[WC], Mv[WC];
#pragma unroll
        for (int k = 0; k < WC; ++k) {
            Pv[k] = kFull;
            Mv[k] = 0u;
        }
        int n = 0, j = 0, pid = -1, c_next = 0, c_next2 = 0, idx = lane;
        bool has = false, more = true;
        const uint8_t *tc = nullptr;
        while (true) {
            if (!has && more) {
                int pos = -1;
                if constexpr (SLOTS == 1) {
                    idx = atomicAdd(a.qcursor + q, 1);
                    if (idx < cnt) pos = cbeg + idx;
                } else if (idx < total) {
                    int sl = 0;
#pragma unroll
                    for (int i = 1; i < SLOTS; ++i) sl += sPre[i] <= idx;
                    pos = sBeg[sl] + idx - sPre[sl];
                    m = sM[sl];
                    peq = sPeq + sl * (S * SIGMA);
                    idx += 32;
                }
                if (pos < 0) {
                    more = false;
                } else {
                    const int t = a.sorted_t[pos];
                    pid = a.sorted_p[pos];
                    const int64_t tp = a.offs[t];
                    n = (int)(a.offs[t + 1] - tp);
                    tc = a.codes + tp;
                    j = 0;
                    c_next = n > 0 ? __ldg(tc) : 0;
                    c_next2 = n > 1 ? __ldg(tc + 1) : 0;
#pragma unroll
                    for (int k = 0; k < WC; ++k) {
                        Pv[k] = kFull;
                        Mv[k] = 0u;
                    }
                    has = true;
                }
            }
            if (!__any_sync(kFull, has)) break;
            // two columns per iteration while every busy lane has two left:
            // the second column's first words overlap the first column's
            // last ones, and the vote is paid once per two columns
            const bool pair2 = __all_sync(kFull, !has || j + 1 < n);
            if (has) {
                if (pair2) {
                    const int c0 = c_next, c1 = c_next2;
                    c_next = j + 2 < n ? __ldg(tc + j + 2) : 0;
                    c_next2 = j + 3 < n ? __ldg(tc + j + 3) : 0;
                    lane_column_chain<WC>(peq + c0 * S, Pv, Mv);
                    lane_column_chain<WC>(peq + c1 * S, Pv, Mv);
                    j += 2;
                } else if (j < n) {
                    const int c = c_next;
                    c_next = c_next2;
                    c_next2 = j + 2 < n ? __ldg(tc + j + 2) : 0;
                    const uint32_t *row = peq + c * S;
                    lane_column_chain<WC>(row, Pv, Mv);
                    ++j;
                }
                if (j == n) {
                    int d = n;
#pragma unroll
                    for (int k = 0; k < WC; ++k) {
                        const int rem = m - 32 * k;
                        const uint32_t mk = rem >= 32 ? kFull : (rem <= 0 ? 0u : ((1u << rem) - 1u));
                        d += __popc(Pv[k] & mk) - __popc(Mv[k] & mk);
                    }
                    a.d_out[pid] = d;
                    has = false;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Warp kernel: one warp per (query, target); lane g holds words
// g*WPL .. g*WPL+WPL-1 and works on column s - g at step s, receiving the
// top bits of lane g-1's Ph/Mh for that column through __shfl_up_sync.
// Targets of the same query follow back to back: lane 0 pulls the next one
// into a small ring in shared memory and every lane reaches it g steps later.
// The distance is summed down the pipeline and written by lane 31.
// Match masks: layout [w][c][lane], conflict-free for any mix of symbols.
// ---------------------------------------------------------------------------
constexpr int kRing = 32;

template <int WPL, int B, int SIGMA>
__global__ void __launch_bounds__(128) lev_warp_kernel(LevArgs a) {
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    uint32_t *sPeq = smem + wid * (WPL * SIGMA * 32 + 3 * kRing + 2);
    int32_t *ring_t = reinterpret_cast<int32_t *>(sPeq + WPL * SIGMA * 32);
    int32_t *ring_p = ring_t + kRing;
    int32_t *ring_n = ring_p + kRing;
    volatile int32_t *end_step = ring_n + kRing;
    const int ntasks = a.bcount[a.bucket];
    const int2 *tasks = a.tasks + a.boff[a.bucket];
    int32_t *counter = a.bcounter + a.bucket;

    if (warp_has_no_task(ntasks)) return;
    for (int task = next_task(counter, lane); task < ntasks; task = next_task(counter, lane)) {
        const int q = tasks[task].x;
        const int64_t qpos = a.offs[q];
        const int m = (int)(a.offs[q + 1] - qpos);
        const int cbeg = a.qstart[q];
        const int cnt = a.qstart[q + 1] - cbeg;
        __syncwarp();
        uint32_t maskw[WPL];
#pragma unroll
        for (int w = 0; w < WPL; ++w) {
            uint32_t pl[B], mask;
            query_planes<B>(a.planes, qpos, m, lane * WPL + w, pl, mask);
            maskw[w] = mask;
#pragma unroll
            for (int c = 0; c < SIGMA; ++c) sPeq[(w * SIGMA + c) * 32 + lane] = match_mask<B, SIGMA>(pl, mask, c);
        }
        if (lane == 0) *end_step = 0x3fffffff;
        __syncwarp();

        uint32_t Pv[WPL], Mv[WPL];
        int seq = -1;          // ring slot of the current target of this lane
        int n = 0, j = 0, pid = -1;
        const uint8_t *tc = nullptr;
        bool started = false, finished = false;
        int msg = 0;
        for (int s = 0;; ++s) {
            // lane 0 feeds the ring whenever it needs a target
            if (lane == 0 && !finished && j == n) {
                int nn = 0, t = -1, p = -1;
                while (true) {
                    const int idx = atomicAdd(a.qcursor + q, 1);
                    if (idx >= cnt) break;
                    t = a.sorted_t[cbeg + idx];
                    p = a.sorted_p[cbeg + idx];
                    nn = (int)(a.offs[t + 1] - a.offs[t]);
                    if (nn > 0) break;
                    a.d_out[p] = m;   // empty target: f = m
                    t = -1;
                }
                const int slot = (seq + 1) & (kRing - 1);
                ring_t[slot] = t;
                ring_p[slot] = p;
                ring_n[slot] = nn;
                if (t < 0) *end_step = s;
            }
            __syncwarp();
            if (s >= *end_step + 32) break;
            const int msg_in = __shfl_up_sync(kFull, msg, 1);
            msg = 0;
            if (!finished && s >= lane) {
                if (!started || j == n) {
                    seq = (seq + 1) & (kRing - 1);
                    const int t = ring_t[seq];
                    if (t < 0) {
                        finished = true;
                    } else {
                        pid = ring_p[seq];
                        n = ring_n[seq];
                        const int64_t tp = a.offs[t];
                        tc = a.codes + tp;
                        j = 0;
                        started = true;
#pragma unroll
                        for (int w = 0; w < WPL; ++w) {
                            Pv[w] = kFull;
                            Mv[w] = 0u;
                        }
                    }
                }
                if (!finished) {
                    const int c = __ldg(tc + j);
                    uint32_t ph_in = lane == 0 ? 1u : (uint32_t)(msg_in & 1);
                    uint32_t mh_in = lane == 0 ? 0u : (uint32_t)((msg_in >> 1) & 1);
                    const uint32_t *col = sPeq + c * 32 + lane;
                    uint32_t eq[WPL], ph_out, mh_out;
#pragma unroll
                    for (int w = 0; w < WPL; ++w) eq[w] = col[w * SIGMA * 32];
                    bv_column<WPL>(eq, Pv, Mv, ph_in, mh_in, ph_out, mh_out);
                    msg = (int)(ph_out | (mh_out << 1));
                    ++j;
                    if (j == n) {
                        int part = lane == 0 ? 0 : (msg_in >> 2);
#pragma unroll
                        for (int w = 0; w < WPL; ++w) part += __popc(Pv[w] & maskw[w]) - __popc(Mv[w] & maskw[w]);
                        msg |= part << 2;
                        if (lane == 31) a.d_out[pid] = n + part;
                    }
                }
            }
        }
    }
}

using LevLauncher = void (*)(const LevArgs &, int grid, cudaStream_t);

struct LevKernelInfo {
    int kind;       // 0 = lane, 1 = warp
    int words;      // WC (lane) or WPL (warp)
    int alphabet;
    size_t smem_per_warp;
    LevLauncher launch;
    const void *fn;
};

template <int WC, int B, int SIGMA, int SLOTS = 1>
void launch_lane(const LevArgs &a, int grid, cudaStream_t st) {
    lev_lane_kernel<WC, B, SIGMA, SLOTS><<<grid, 128, 4 * lane_smem_words(WC, SIGMA, SLOTS) * sizeof(uint32_t), st>>>(a);
}

template <int WPL, int B, int SIGMA>
void launch_warp(const LevArgs &a, int grid, cudaStream_t st) {
    lev_warp_kernel<WPL, B, SIGMA><<<grid, 128, 4 * (WPL * SIGMA * 32 + 3 * kRing + 2) * sizeof(uint32_t), st>>>(a);
}

// Registries defined in the instantiation units.
extern const LevKernelInfo kLevLaneDna[];
extern const int kLevLaneDnaCount;
extern const LevKernelInfo kLevLaneProt[];
extern const int kLevLaneProtCount;
// lane kernel with 8 queries per warp (4 lanes each)
constexpr int kLevSlots = 8;
extern const LevKernelInfo kLevSlotDna[];
extern const int kLevSlotDnaCount;
extern const LevKernelInfo kLevSlotProt[];
extern const int kLevSlotProtCount;
extern const LevKernelInfo kLevWarpDna[];
extern const int kLevWarpDnaCount;
extern const LevKernelInfo kLevWarpProt[];
extern const int kLevWarpProtCount;

}  // namespace msa
