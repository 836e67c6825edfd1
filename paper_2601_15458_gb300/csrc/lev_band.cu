// Banded bit-vector Levenshtein with an exactness certificate (A4) and the
// C entry point msa_lev_banded_batch.
//
// Ukkonen's band: a global alignment path through cell (i, j) of an m x n
// problem costs at least |j - i| + |(n - j) - (m - i)|, so when the distance
// d is at most k every optimal path stays on the diagonals delta = j - i with
// |delta| + |(n - m) - delta| <= k, i.e. delta in
// [ceil((n-m-k)/2), floor((n-m+k)/2)].  A DP restricted to any superset of
// that band, with every cell outside it given a value no smaller than its
// true value, returns some d_k with d <= d_k; and d_k <= k implies d_k = d.
// So the result is accepted exactly when d_k <= k, else k doubles.
//
// Kernel: a group of G lanes per pair (32 / G pairs per warp).  The rows
// are cut into blocks of H = 32 WPL rows; lane l of a group holds blocks
// l, l + G, l + 2G, ... one at a time, each as WPL words of Pv, Mv and the
// query's bit planes in registers.  Block b computes column j at the group's
// step j + b, one step behind the block above it (a skewed pipeline), so the
// carry into its top row and the shifted-in Ph/Mh bits of column j arrive
// from the lane above by one shuffle per step; the carry of the addition out
// of a row equals that row's Mh bit, so the two Ph/Mh bits are all that
// crosses.  Block b is live on the columns where its rows meet the band,
// [max(1, bH + 1 + dlo), min(n, bH + H + dhi)] for the band diagonals
// [dlo, dhi]; before its first column it holds the upper bound "+1 on every
// row" (D[i][j] <= D[i-1][j] + 1), and once the block above it has passed its
// last column it takes that row to grow by +1 per column (D[i][j] <=
// D[i][j-1] + 1), the top-of-matrix boundary.  The value of D on the row just
// above a block (T) is handed down with the carries when the block above
// leaves.  A lane whose block leaves takes its next block, so the group
// covers any band with dhi - dlo <= (G - 1) H: the computed rows per column
// follow the requested band, not the group's capacity.
// At column n each live block adds its vertical deltas over rows <= m (the
// top one also its T), and the group's sum is D[m][n].
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "carry_chain.cuh"
#include "lev_kernels.cuh"
#include "msa_internal.cuh"

namespace msa {

// (G, WPL) of the pipelined kernel, in increasing cost per step (G lanes x
// about 10 WPL + 26 instructions) and increasing capacity (G - 1) x 32 WPL;
// a pair goes to the first one that holds its band.
constexpr int kBandBuckets = 24;
#define BAND_G_LIST {2, 2, 2, 2, 2, 4, 4, 4, 4, 4, 8, 8, 8, 8, 8, 16, 16, 16, 16, 16, 32, 32, 32, 32}
#define BAND_WPL_LIST {2, 3, 4, 6, 8, 3, 4, 5, 6, 8, 4, 5, 6, 7, 8, 4, 5, 6, 7, 8, 4, 5, 6, 8}
__constant__ int kBandG[kBandBuckets] = BAND_G_LIST;
__constant__ int kBandWPL[kBandBuckets] = BAND_WPL_LIST;
static const int kBandGHost[kBandBuckets] = BAND_G_LIST;
static const int kBandWPLHost[kBandBuckets] = BAND_WPL_LIST;
// One-lane buckets (DNA): a pair in a single lane, its band held as a window
// of W 32-row words in registers (band_lane_kernel), for bands up to
// 32 W - 63 rows.  Indices kBandBuckets .. kBandAll - 1 after the group
// buckets.
constexpr int kLaneBuckets = 8;
constexpr int kBandAll = kBandBuckets + kLaneBuckets;
#define BAND_LANE_W_LIST {4, 8, 12, 16, 24, 32, 40, 48}
__constant__ int kLaneW[kLaneBuckets] = BAND_LANE_W_LIST;
static const int kLaneWHost[kLaneBuckets] = BAND_LANE_W_LIST;
// band rows a W-word window covers at every column of a 32-column phase
__host__ __device__ constexpr int lane_capacity(int W) { return 32 * W - 63; }
// a band whose rows per column (k + H) exceed this share of the column goes
// to the full bit-vector DP, whose kernels need no band bookkeeping
constexpr float kBandMaxShare = 0.75f;
// rounds of band retries per call (all enqueued; pairs still pending after
// the last one go to the full DP)
constexpr int kBandRounds = 3;
constexpr int kBandThreads = 128;
// dynamic shared memory of a one-lane block: each thread's match masks of
// its window rows, 4 symbols x W words
constexpr size_t lane_band_smem(int W) { return (size_t)W * 4 * kBandThreads * 4; }

struct BandArgs {
    const uint32_t *planes;
    const uint8_t *codes;
    const int64_t *offs;
    const int32_t *pairs;
    const int32_t *blist;     // pending pair ids, bucket-major
    const int32_t *boff;      // [kBandBuckets]
    const int32_t *bcount;    // [kBandBuckets]
    int32_t *bcounter;        // [kBandBuckets]
    int32_t *k_cur;           // [P] band requested for the pair's next attempt
    int32_t *d_out;
    int32_t *k_used;
    int32_t *next_list;       // failures
    int32_t *next_count;
    int32_t bucket;
};

// Per-lane match masks of DNA blocks in shared memory, [symbol][word][thread]
// (thread-minor, so a warp's loads hit 32 distinct banks whatever symbols
// its lanes read); other alphabets form each column's mask from the bit
// planes held in registers.
template <int WPL, int B>
struct BandEq {
    static constexpr bool kShared = B == 2;
    static constexpr int kSigma = 4;
    uint32_t pl[kShared ? 1 : WPL][kShared ? 1 : B];
};

// Columns per pipeline step: each step a block computes a chunk of CPS
// consecutive columns, so the per-step bookkeeping (the shuffle, the live
// tests, the vote) is paid once per chunk.  A block's live columns are
// widened to whole chunks (a superset of the band, so still exact), and the
// lane above sends the Ph/Mh bits of all CPS columns in one word.
constexpr int kBandCps = 4;
// The word sent down holds 2 bits per column below T, the value of D on the
// row above (at most m + n <= 32,768 for sequences of up to 16,384), so
// 2 CPS + 16 bits must fit in 32.
static_assert(kBandCps >= 1 && 2 * kBandCps + 16 <= 32, "columns per step");
// the carry word of a top block: Ph = 1, Mh (carry) = 0 for each column
constexpr uint32_t kBandTopBits = 0x55555555u & ((1u << (2 * kBandCps)) - 1u);
// capacity of a (G, WPL) group at CPS columns per step: the lane that holds
// block b must have finished it before block b + G needs it
__host__ __device__ constexpr int band_capacity(int G, int WPL) { return (G - 1) * 32 * WPL - 2 * kBandCps; }

// The 4 code bytes at p .. p + 3, from the two aligned words that hold them
// (bytes past a sequence's end come from the next sequence or the arena's
// padding of at least 32 bytes; they only feed columns past n, never read).
__device__ __forceinline__ uint32_t load_codes4(const uint8_t *p) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uint32_t *w = reinterpret_cast<const uint32_t *>(a & ~uintptr_t(3));
    return __funnelshift_r(__ldg(w), __ldg(w + 1), (int)(a & 3) * 8);
}
static_assert(kBandCps == 4, "a chunk's codes are one packed word");

// Takes block bk of the current pair: its live chunks [qs, qe] (columns
// widened to whole chunks), the last live column of the block above (0 for
// the top block) and its chunk, fresh +1 vertical deltas, the query's match
// masks of its rows and the symbols of its first chunk.
template <int WPL, int B>
__device__ __forceinline__ void band_block_setup(int bk, int dlo, int dhi, int m, int n, const uint32_t *planes,
                                                 int64_t qa, const uint8_t *tc, int &qs, int &qe, int &jep, int &qep,
                                                 uint32_t (&Pv)[WPL], uint32_t (&Mv)[WPL], BandEq<WPL, B> &E,
                                                 uint32_t *sPeq, uint32_t &cw_next) {
    constexpr int H = 32 * WPL;
    const int js = max(1, bk * H + 1 + dlo);
    const int je = min(n, bk * H + H + dhi);
    qs = (js - 1) / kBandCps + 1;
    qe = (je - 1) / kBandCps + 1;
    if (bk == 0) {
        jep = 0;
        qep = 0;
    } else {
        const int jp = min(n, (bk - 1) * H + H + dhi);      // last live column of the block above, widened
        qep = (jp - 1) / kBandCps + 1;
        jep = min(n, qep * kBandCps);
    }
#pragma unroll
    for (int w = 0; w < WPL; ++w) {
        Pv[w] = kFull;
        Mv[w] = 0u;
        uint32_t pl[B], mask;
        query_planes<B>(planes, qa, m, bk * WPL + w, pl, mask);
        if constexpr (BandEq<WPL, B>::kShared) {
#pragma unroll
            for (int c = 0; c < 4; ++c) sPeq[(c * WPL + w) * kBandThreads] = match_mask<B, 4>(pl, mask, c);
        } else {
#pragma unroll
            for (int q = 0; q < B; ++q) E.pl[w][q] = pl[q];
        }
    }
    cw_next = load_codes4(tc + (qs - 1) * kBandCps);
}

// Column c of a block's chunk: the match masks of the column's code (from
// shared memory for DNA, from the bit planes in registers otherwise), the
// column step with the row-above bits of inb, and the block's bottom bits
// packed into o.
template <int WPL, int B>
__device__ __forceinline__ void band_chunk_column(int c, uint32_t cw, uint32_t inb, const uint32_t *sPeq,
                                                  const BandEq<WPL, B> &E, uint32_t (&Pv)[WPL], uint32_t (&Mv)[WPL],
                                                  uint32_t &o) {
    const uint32_t cc = (cw >> (8 * c)) & 0xffu;
    uint32_t eq[WPL];
    if constexpr (BandEq<WPL, B>::kShared) {
        const uint32_t *row = sPeq + (cc & 3) * WPL * kBandThreads;
#pragma unroll
        for (int w = 0; w < WPL; ++w) eq[w] = row[w * kBandThreads];
    } else {
        uint32_t x[B];
#pragma unroll
        for (int b = 0; b < B; ++b) x[b] = ((cc >> b) & 1) ? 0u : kFull;
#pragma unroll
        for (int w = 0; w < WPL; ++w) {
            uint32_t e = E.pl[w][0] ^ x[0];
#pragma unroll
            for (int b = 1; b < B; ++b) e &= E.pl[w][b] ^ x[b];
            eq[w] = e;
        }
    }
    // the Ph bit of the row above goes in as bit 31 of php, its carry as any
    // nonzero value; the block's bottom bits are packed into o on the
    // multiply-add pipe
    uint32_t php_out, mh_out;
    bv_column_raw<WPL>(eq, Pv, Mv, inb << (31 - 2 * c), inb & (2u << (2 * c)), php_out, mh_out);
    o = mad_u32(mh_out, 2u << (2 * c), mad_u32(php_out >> 31, 1u << (2 * c), o));
}

template <int G, int WPL, int B>
__global__ void __launch_bounds__(kBandThreads) band_pipe_kernel(BandArgs a) {
    static_assert(G >= 2 && G <= 32 && (G & (G - 1)) == 0, "group size");
    constexpr int H = 32 * WPL;
    constexpr int CPS = kBandCps;
    constexpr bool kShared = BandEq<WPL, B>::kShared;
    __shared__ uint32_t sPeqAll[kShared ? 4 * WPL * kBandThreads : 1];
    uint32_t *sPeq = sPeqAll + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int gbase = lane - gl;
    const int src = gbase + ((gl + G - 1) & (G - 1));    // the lane holding the block above
    const int cnt = a.bcount[a.bucket];
    const int32_t *list = a.blist + a.boff[a.bucket];
    int32_t *counter = a.bcounter + a.bucket;
    uint32_t Pv[WPL], Mv[WPL];
    BandEq<WPL, B> E;
#pragma unroll
    for (int w = 0; w < WPL; ++w) {
        Pv[w] = kFull;
        Mv[w] = 0u;
    }
    if constexpr (!kShared) {
#pragma unroll
        for (int w = 0; w < WPL; ++w)
#pragma unroll
            for (int q = 0; q < B; ++q) E.pl[w][q] = 0u;
    }
    // per group (the same in each of its lanes)
    int p = -1, m = 0, n = 0, k = 0, dlo = 0, dhi = 0, bm = -1, t = 0, tend = 0;
    bool has = false, more = true;
    int64_t qa = 0;
    const uint8_t *tc = nullptr;
    // per lane: its block, that block's live chunks, the last live column of
    // the block above and its chunk, T, the lane's share of D[m][n] and the
    // word sent down
    int bk = 0, qs = 1, qe = 0, jep = 0, qep = 0, Tb = 0, acc = 0;
    uint32_t cw_next = 0u;   // the codes of the block's next chunk, one byte per column
    uint32_t out = 0u;
    bool fin = false;
    while (true) {
        // 1. groups whose pair is done report it; groups without a pair take
        //    the next one (one vote per step: this runs only when some group
        //    of the warp finished, and once at the start)
        if (__any_sync(kFull, fin || (!has && more))) {
            if (__any_sync(kFull, fin)) {
                int d = fin ? acc : 0;
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) d += __shfl_xor_sync(kFull, d, o, G);
                if (fin) {
                    // d_k > k is an upper bound of the distance, so a band of
                    // d_k certifies; the band at most doubles.  A retry that
                    // still fits this group runs at once, in place.
                    const int k2 = min(d, 2 * k + 1);
                    if (d <= k) {
                        if (gl == 0) {
                            a.d_out[p] = d;
                            a.k_used[p] = k;
                        }
                        has = false;
                    } else if (k2 <= band_capacity(G, WPL) && k2 < m) {
                        k = k2;
                        dlo = -((k + m - n) >> 1);
                        dhi = (n - m + k) >> 1;
                        t = 0;
                        Tb = 0;
                        acc = 0;
                        out = 0u;
                        bk = gl;
                        if (bk <= bm)
                            band_block_setup<WPL, B>(bk, dlo, dhi, m, n, a.planes, qa, tc, qs, qe, jep, qep, Pv, Mv,
                                                     E, sPeq, cw_next);
                    } else {
                        if (gl == 0) {
                            a.k_cur[p] = k2;
                            a.next_list[atomicAdd(a.next_count, 1)] = p;
                        }
                        has = false;
                    }
                    fin = false;
                }
            }
            const bool need = !has && more;
            if (__any_sync(kFull, need)) {
                // one claim per warp for all its groups that need a pair, so
                // the queue is handed out in whole warps: claimed one group
                // at a time, a persistent grid with more groups than pairs
                // spreads the pairs one per warp and leaves most lanes idle
                const unsigned leaders = __ballot_sync(kFull, need && gl == 0);
                int base = 0;
                if (lane == 0) base = atomicAdd(counter, __popc(leaders));
                base = __shfl_sync(kFull, base, 0);
                int i = base + __popc(leaders & ((1u << lane) - 1u));
                i = __shfl_sync(kFull, i, gbase);
                if (need) {
                    if (i >= cnt) {
                        more = false;
                    } else {
                        p = list[i];
                        const int q = a.pairs[2 * p], r = a.pairs[2 * p + 1];
                        int64_t qb = a.offs[q + 1], ta = a.offs[r], tb = a.offs[r + 1];
                        qa = a.offs[q];
                        if (qb - qa < tb - ta) {     // longer sequence on the rows
                            int64_t y = qa; qa = ta; ta = y;
                            y = qb; qb = tb; tb = y;
                        }
                        m = (int)(qb - qa);
                        n = (int)(tb - ta);
                        k = min(max(a.k_cur[p], m - n), m);
                        dlo = -((k + m - n) >> 1);   // ceil((n - m - k) / 2)
                        dhi = (n - m + k) >> 1;      // floor((n - m + k) / 2)
                        tc = a.codes + ta;
                        t = 0;
                        Tb = 0;
                        acc = 0;
                        out = 0u;
                        if (n == 0) {                // no columns: D[m][0] = m
                            if (gl == 0) {
                                a.d_out[p] = m;
                                a.k_used[p] = k;
                            }
                        } else {
                            bm = (m - 1) / H;
                            tend = (n - 1) / CPS + 1 + bm;
                            bk = gl;
                            if (bk <= bm)
                                band_block_setup<WPL, B>(bk, dlo, dhi, m, n, a.planes, qa, tc, qs, qe, jep, qep, Pv,
                                                         Mv, E, sPeq, cw_next);
                            has = true;
                        }
                    }
                }
            }
            if (!__any_sync(kFull, has)) break;
        }
        // 2. one pipeline step: block bk computes chunk t - bk
        const uint32_t in = __shfl_sync(kFull, out, src);
        if (has) {
            ++t;
            fin = t == tend;
            const int q = t - bk;
            if (bk <= bm) {
                if (q == qep) Tb = (int)(in >> (2 * CPS));    // the block above leaves after this chunk
                if (q >= qs && q <= qe) {
                    const uint32_t cw = cw_next;
                    const int j0 = (q - 1) * CPS;              // columns j0 + 1 .. j0 + CPS
                    if (q < qe) cw_next = load_codes4(tc + j0 + CPS);
                    // the block above leaves at a chunk end, so a chunk is
                    // either all below it or all on top (row above: +1 per
                    // column, Ph = 1, carry 0 for every column)
                    const bool top = q > qep;
                    const uint32_t inb = top ? kBandTopBits : in;
                    if (top) Tb += min(CPS, n - j0);
                    const bool last = j0 + CPS >= n;          // the chunk holds column n
                    uint32_t o = 0u;
                    if (!last) {
#pragma unroll
                        for (int c = 0; c < CPS; ++c) band_chunk_column<WPL, B>(c, cw, inb, sPeq, E, Pv, Mv, o);
                    } else {
                        // the chunk holding column n: columns past n run on
                        // whatever bytes follow and are never read
#pragma unroll
                        for (int c = 0; c < CPS; ++c) {
                            band_chunk_column<WPL, B>(c, cw, inb, sPeq, E, Pv, Mv, o);
                            if (j0 + 1 + c == n) {
                                // this block's share of D[m][n]: its rows <= m (and T if on top)
                                int part = top ? Tb : 0;
#pragma unroll
                                for (int w = 0; w < WPL; ++w) {
                                    const int rem = m - 32 * (bk * WPL + w);
                                    const uint32_t mk = rem >= 32 ? kFull : (rem <= 0 ? 0u : ((1u << rem) - 1u));
                                    part += __popc(Pv[w] & mk) - __popc(Mv[w] & mk);
                                }
                                acc += part;
                            }
                        }
                    }
                    out = o;
                    if (q == qe) {
                        // the block's last chunk: hand D on its bottom row to
                        // the block below and move on to the next block
                        int delta = 0;
#pragma unroll
                        for (int w = 0; w < WPL; ++w) delta += __popc(Pv[w]) - __popc(Mv[w]);
                        out |= (uint32_t)(Tb + delta) << (2 * CPS);
                        bk += G;
                        if (bk <= bm)
                            band_block_setup<WPL, B>(bk, dlo, dhi, m, n, a.planes, qa, tc, qs, qe, jep, qep, Pv, Mv,
                                                     E, sPeq, cw_next);
                    }
                }
            }
        }
    }
}

// One-lane banded kernel (DNA): each lane holds a whole pair.  The band of
// column j spans rows [j - dhi, j - dlo]; the lane keeps a window of W
// 32-row words (Pv and Mv in registers, the query's two bit planes of the
// window's rows in shared memory) that moves down one word at a time, only
// at 32-column phase boundaries, so that it covers every band row of the
// next 32 columns (32 W >= k + 63).  The row just above the window is taken
// to grow by +1 per column (the upper bound D[i][j] <= D[i][j-1] + 1, the
// same boundary as row 0, whose value T is carried along), and a word
// entering at the bottom starts at "+1 on every row" (D[i][j] <= D[i-1][j] +
// 1); every computed value is then an upper bound of D, and exact on every
// cell whose optimal paths stay in the window, so the certificate of the
// group kernel applies unchanged.  All lanes of a warp start pairs only at
// phase boundaries, so the window moves (or not) for every lane at the same
// iteration.

// One column over the window, in chunks of up to 8 words on the carry chain
// (as in the lane kernel), the match masks of the column's symbol read from
// shared memory (sEq: word w of the window at sEq[4 w kBandThreads]).  The
// row above the window adds +1 (Ph in = 1, carry in = 0).
template <int W, int K0 = 0>
__device__ __forceinline__ void lane_band_column(const uint32_t *sEq, uint32_t (&Pv)[W], uint32_t (&Mv)[W],
                                                 uint32_t cy = 0u, uint32_t php = 1u << 31) {
    if constexpr (K0 < W) {
        constexpr int L = W - K0 < 8 ? W - K0 : 8;
        uint32_t eq[L], u[L], pv[L], sm[L];
#pragma unroll
        for (int i = 0; i < L; ++i) {
            eq[i] = sEq[(K0 + i) * 4 * kBandThreads];
            pv[i] = Pv[K0 + i];
            u[i] = eq[i] & pv[i];
        }
        cy = CarryChainIn<L>::add(sm, u, pv, cy);
#pragma unroll
        for (int i = 0; i < L; ++i) {
            const uint32_t mhs = sm[i] ^ u[i] ^ pv[i];
            const uint32_t ph = Mv[K0 + i] | ~(sm[i] | pv[i] | eq[i]);
            const uint32_t phs = __funnelshift_l(php, ph, 1);
            php = ph;
            const uint32_t xv = eq[i] | Mv[K0 + i];
            Pv[K0 + i] = mhs | ~(xv | phs);
            Mv[K0 + i] = phs & xv;
        }
        lane_band_column<W, K0 + L>(sEq, Pv, Mv, cy, php);
    }
}

// the target's 2-bit codes at arena positions pos .. pos + 31, as two planes
__device__ __forceinline__ void lane_target_bits(const uint32_t *__restrict__ planes, int64_t pos, uint32_t &t0,
                                                 uint32_t &t1) {
    const int64_t wi = pos >> 5;
    const int r = (int)(pos & 31);
    t0 = __funnelshift_r(__ldg(planes + 2 * wi), __ldg(planes + 2 * wi + 2), r);
    t1 = __funnelshift_r(__ldg(planes + 2 * wi + 1), __ldg(planes + 2 * wi + 3), r);
}

template <int W>
__global__ void __launch_bounds__(kBandThreads) band_lane_kernel(BandArgs a) {
    extern __shared__ uint32_t sMasks[];
    // the match mask of symbol c for word w of this lane's window at
    // sM[(4 w + c) kBandThreads] (thread-minor: conflict-free for any mix of
    // symbols across the warp)
    uint32_t *sM = sMasks + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int cnt = a.bcount[a.bucket];
    const int32_t *list = a.blist + a.boff[a.bucket];
    int32_t *counter = a.bcounter + a.bucket;
    uint32_t Pv[W], Mv[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        Pv[w] = kFull;
        Mv[w] = 0u;
    }
    int p = -1, m = 0, n = 0, k = 0, dhi = 0, j = 0, w0 = 0, T = 0;
    int64_t qa = 0, ta = 0;
    bool has = false, more = true, start = false;
    uint32_t t0 = 0u, t1 = 0u, nt0 = 0u, nt1 = 0u;
    uint2 nb = make_uint2(0u, 0u);     // planes and row mask of the word that enters at the next move
    uint32_t nbm = 0u;
    while (true) {
        // ---- phase boundary -------------------------------------------
        // a lane whose pair has reached column n applies the certificate;
        // a failed band that still fits the window restarts at once
        if (has && j == n) {
            int d = T;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const int rem = m - 32 * (w0 + w);
                const uint32_t mk = rem >= 32 ? kFull : (rem <= 0 ? 0u : ((1u << rem) - 1u));
                d += __popc(Pv[w] & mk) - __popc(Mv[w] & mk);
            }
            const int k2 = min(d, 2 * k + 1);
            if (d <= k) {
                a.d_out[p] = d;
                a.k_used[p] = k;
                has = false;
            } else if (k2 <= lane_capacity(W) && k2 < m) {
                k = k2;
                start = true;
            } else {
                a.k_cur[p] = k2;
                a.next_list[atomicAdd(a.next_count, 1)] = p;
                has = false;
            }
        }
        // lanes without a pair take the next ones (one claim per warp)
        const bool need = !has && more;
        if (__any_sync(kFull, need)) {
            const unsigned who = __ballot_sync(kFull, need);
            int base = 0;
            if (lane == 0) base = atomicAdd(counter, __popc(who));
            base = __shfl_sync(kFull, base, 0);
            if (need) {
                const int i = base + __popc(who & ((1u << lane) - 1u));
                if (i >= cnt) {
                    more = false;
                } else {
                    p = list[i];
                    const int q = a.pairs[2 * p], r = a.pairs[2 * p + 1];
                    int64_t qb = a.offs[q + 1], tb = a.offs[r + 1];
                    qa = a.offs[q];
                    ta = a.offs[r];
                    if (qb - qa < tb - ta) {     // longer sequence on the rows
                        int64_t y = qa; qa = ta; ta = y;
                        y = qb; qb = tb; tb = y;
                    }
                    m = (int)(qb - qa);
                    n = (int)(tb - ta);
                    k = min(max(a.k_cur[p], m - n), m);
                    has = true;
                    start = true;
                }
            }
        }
        if (!__any_sync(kFull, has)) break;
        if (start) {
            // (re)start the pair at column 0: window at row 1, rows +1
            start = false;
            dhi = (n - m + k) >> 1;
            j = 0;
            w0 = 0;
            T = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                Pv[w] = kFull;
                Mv[w] = 0u;
                uint32_t pl[2], mask;
                query_planes<2>(a.planes, qa, m, w, pl, mask);
#pragma unroll
                for (int c = 0; c < 4; ++c) sM[(4 * w + c) * kBandThreads] = match_mask<2, 4>(pl, mask, c);
            }
            uint32_t pl[2], mask;
            query_planes<2>(a.planes, qa, m, W, pl, mask);
            nb = make_uint2(pl[0], pl[1]);
            nbm = mask;
            lane_target_bits(a.planes, ta, nt0, nt1);
        } else if (has) {
            // the window moves down a word when the band's top row passes it:
            // w0 = floor((j - dhi) / 32) for the columns j + 1 .. j + 32
            const int w0n = j - dhi < 0 ? 0 : (j - dhi) >> 5;
            if (w0n > w0) {
                T += __popc(Pv[0]) - __popc(Mv[0]);
#pragma unroll
                for (int w = 0; w + 1 < W; ++w) {
                    Pv[w] = Pv[w + 1];
                    Mv[w] = Mv[w + 1];
#pragma unroll
                    for (int c = 0; c < 4; ++c) sM[(4 * w + c) * kBandThreads] = sM[(4 * w + 4 + c) * kBandThreads];
                }
                Pv[W - 1] = kFull;
                Mv[W - 1] = 0u;
                {
                    const uint32_t pl[2] = {nb.x, nb.y};
#pragma unroll
                    for (int c = 0; c < 4; ++c) sM[(4 * (W - 1) + c) * kBandThreads] = match_mask<2, 4>(pl, nbm, c);
                }
                w0 = w0n;
                uint32_t pl[2], mask;
                query_planes<2>(a.planes, qa, m, w0 + W, pl, mask);
                nb = make_uint2(pl[0], pl[1]);
                nbm = mask;
            }
        }
        // the target's codes for this phase, and a prefetch of the next
        t0 = nt0;
        t1 = nt1;
        if (has && j + 32 < n) lane_target_bits(a.planes, ta + j + 32, nt0, nt1);
        // ---- 32 columns ------------------------------------------------
        const int cols = has ? min(32, n - j) : 0;
#pragma unroll 1
        for (int c = 0; c < 32; ++c) {
            if (c < cols) lane_band_column<W>(sM + (int)((t0 & 1u) | ((t1 & 1u) << 1)) * kBandThreads, Pv, Mv);
            t0 >>= 1;
            t1 >>= 1;
        }
        j += cols;
        T += cols;
    }
}

template <int W>
void launch_band_lane(const BandArgs &a, int grid, cudaStream_t st) {
    band_lane_kernel<W><<<grid, kBandThreads, lane_band_smem(W), st>>>(a);
}

using BandLauncher = void (*)(const BandArgs &, int, cudaStream_t);

template <int G, int WPL, int B>
void launch_band_pipe(const BandArgs &a, int grid, cudaStream_t st) {
    band_pipe_kernel<G, WPL, B><<<grid, kBandThreads, 0, st>>>(a);
}

#define BAND_TABLE(B) \
    {launch_band_pipe<2, 2, B>, launch_band_pipe<2, 3, B>, launch_band_pipe<2, 4, B>, launch_band_pipe<2, 6, B>, launch_band_pipe<2, 8, B>,            \
         launch_band_pipe<4, 3, B>, launch_band_pipe<4, 4, B>, launch_band_pipe<4, 5, B>, launch_band_pipe<4, 6, B>, launch_band_pipe<4, 8, B>,        \
         launch_band_pipe<8, 4, B>, launch_band_pipe<8, 5, B>, launch_band_pipe<8, 6, B>, launch_band_pipe<8, 7, B>, launch_band_pipe<8, 8, B>,        \
         launch_band_pipe<16, 4, B>, launch_band_pipe<16, 5, B>, launch_band_pipe<16, 6, B>, launch_band_pipe<16, 7, B>, launch_band_pipe<16, 8, B>,   \
         launch_band_pipe<32, 4, B>, launch_band_pipe<32, 5, B>, launch_band_pipe<32, 6, B>, launch_band_pipe<32, 8, B>}
#define BAND_FNS(B) \
    {(const void *)band_pipe_kernel<2, 2, B>, (const void *)band_pipe_kernel<2, 3, B>, (const void *)band_pipe_kernel<2, 4, B>,          \
         (const void *)band_pipe_kernel<2, 6, B>, (const void *)band_pipe_kernel<2, 8, B>, (const void *)band_pipe_kernel<4, 3, B>,      \
         (const void *)band_pipe_kernel<4, 4, B>, (const void *)band_pipe_kernel<4, 5, B>, (const void *)band_pipe_kernel<4, 6, B>,      \
         (const void *)band_pipe_kernel<4, 8, B>, (const void *)band_pipe_kernel<8, 4, B>, (const void *)band_pipe_kernel<8, 5, B>,      \
         (const void *)band_pipe_kernel<8, 6, B>, (const void *)band_pipe_kernel<8, 7, B>, (const void *)band_pipe_kernel<8, 8, B>,      \
         (const void *)band_pipe_kernel<16, 4, B>, (const void *)band_pipe_kernel<16, 5, B>, (const void *)band_pipe_kernel<16, 6, B>,   \
         (const void *)band_pipe_kernel<16, 7, B>, (const void *)band_pipe_kernel<16, 8, B>, (const void *)band_pipe_kernel<32, 4, B>,   \
         (const void *)band_pipe_kernel<32, 5, B>, (const void *)band_pipe_kernel<32, 6, B>, (const void *)band_pipe_kernel<32, 8, B>}
static const BandLauncher kBandDna[kBandBuckets] = BAND_TABLE(2);
static const BandLauncher kBandProt[kBandBuckets] = BAND_TABLE(5);
static const void *kBandFnDna[kBandBuckets] = BAND_FNS(2);
static const void *kBandFnProt[kBandBuckets] = BAND_FNS(5);
static const BandLauncher kBandLane[kLaneBuckets] = {launch_band_lane<4>, launch_band_lane<8>, launch_band_lane<12>,
                                                     launch_band_lane<16>, launch_band_lane<24>, launch_band_lane<32>,
                                                     launch_band_lane<40>, launch_band_lane<48>};
static const void *kBandLaneFn[kLaneBuckets] = {
    (const void *)band_lane_kernel<4>,  (const void *)band_lane_kernel<8>,  (const void *)band_lane_kernel<12>,
    (const void *)band_lane_kernel<16>, (const void *)band_lane_kernel<24>, (const void *)band_lane_kernel<32>,
    (const void *)band_lane_kernel<40>, (const void *)band_lane_kernel<48>};

// Pairs of a bucket are ordered longest first (by half-octave classes of
// the column count), so that the long pairs start early and the short ones
// fill the end of the persistent launch.
constexpr int kLenClasses = 64;
// per round: bcount, boff, bcounter [buckets]; ccount, coff, cfill [buckets x classes], over the
// group buckets and then the one-lane buckets
constexpr int kBandMeta = 3 * kBandAll + 3 * kBandAll * kLenClasses;
static_assert(kBandAll * kLenClasses <= 2048, "band_scan_kernel scans two counts per thread");
static_assert(kBandAll <= msa_ctx::kBandSide, "one side stream per band bucket");
__device__ __forceinline__ int band_len_class(int n) {
    if (n <= 1) return kLenClasses - 1;
    const int lg = 31 - __clz(n);
    return kLenClasses - 1 - min(kLenClasses - 1, 2 * lg + ((n >> (lg - 1)) & 1));
}

// Sorts the pending pairs of one round into band buckets (pass 0 counts,
// pass 1 writes); pairs whose band is too wide for a bucket go to the exact
// full-DP list.  Round 0 reads all pairs (cur == nullptr) and checks every
// index.
template <int PASS>
__global__ void __launch_bounds__(256) band_plan_kernel(const int32_t *__restrict__ pairs, int64_t P,
                                                        const int32_t *__restrict__ cur, const int32_t *cur_count,
                                                        const int64_t *__restrict__ offs, int32_t n, int64_t total,
                                                        int32_t *__restrict__ k_cur, int32_t *__restrict__ bcount,
                                                        int32_t *__restrict__ ccount, int32_t *__restrict__ cfill,
                                                        const int32_t *__restrict__ coff, int32_t *__restrict__ blist,
                                                        int32_t *__restrict__ full_list, int32_t *full_count, int32_t nb,
                                                        bool lane_ok, int32_t *err) {
    const int64_t N = cur ? (int64_t)*cur_count : P;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int p = cur ? cur[i] : (int)i;
        const int x = pairs[2 * p], y = pairs[2 * p + 1];
        if (!cur) {
            bool ok = x >= 0 && x < n && y >= 0 && y < n;
            if (ok) {
                const int64_t xa = offs[x], xb = offs[x + 1], ya = offs[y], yb = offs[y + 1];
                ok = xa >= 0 && xa <= xb && xb <= total && ya >= 0 && ya <= yb && yb <= total;
            }
            if (!ok) {
                if (PASS == 0) record_error(err, kErrIndex, p, x);
                continue;
            }
        }
        const int lx = (int)(offs[x + 1] - offs[x]), ly = (int)(offs[y + 1] - offs[y]);
        const int m = max(lx, ly), dl = abs(lx - ly);
        const int k = min(max(k_cur[p], dl), m);
        int b = -1;
        if (ly > 0 && lx > 0) {
            // DNA bands that a one-lane window holds go to the one-lane
            // kernel, wider ones to the first group bucket that holds them
            if (lane_ok && k <= lane_capacity(kLaneW[kLaneBuckets - 1])) {
                for (int c = 0; c < kLaneBuckets; ++c)
                    if (lane_capacity(kLaneW[c]) >= k) {
                        b = kBandBuckets + c;
                        break;
                    }
                if ((float)(k + 63) > kBandMaxShare * (float)m) b = -1;
            } else {
                for (int c = 0; c < nb; ++c)
                    if (band_capacity(kBandG[c], kBandWPL[c]) >= k) {
                        b = c;
                        break;
                    }
                if (b >= 0 && (float)(k + 32 * kBandWPL[b]) > kBandMaxShare * (float)m) b = -1;
            }
        }
        if (b < 0) {
            if (PASS == 0) full_list[atomicAdd(full_count, 1)] = p;
            continue;
        }
        const int slot = b * kLenClasses + band_len_class(min(lx, ly));
        if (PASS == 0) {
            atomicAdd(bcount + b, 1);
            atomicAdd(ccount + slot, 1);
        } else {
            blist[coff[slot] + atomicAdd(cfill + slot, 1)] = p;
        }
    }
}

// Offsets of the buckets and of their length classes in the pair list: an
// exclusive scan of the bucket-major counts (at most 2,048 of them) by one
// block, two counts per thread.
__global__ void __launch_bounds__(1024) band_scan_kernel(const int32_t *__restrict__ ccount,
                                                         int32_t *__restrict__ coff, int32_t *__restrict__ boff,
                                                         int32_t nb) {
    __shared__ int32_t wpre[32];
    const int total = nb * kLenClasses;
    const int i0 = 2 * threadIdx.x;
    const int x0 = i0 < total ? ccount[i0] : 0, x1 = i0 + 1 < total ? ccount[i0 + 1] : 0;
    const int own = x0 + x1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wpre[w] = inc;
    __syncthreads();
    if (w == 0) {
        int t = wpre[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wpre[lane] = t;
    }
    __syncthreads();
    const int run = (w ? wpre[w - 1] : 0) + inc - own;
    if (i0 < total) coff[i0] = run;
    if (i0 + 1 < total) coff[i0 + 1] = run + x0;
    if (i0 < total && i0 % kLenClasses == 0) boff[i0 / kLenClasses] = run;
    if (i0 + 1 < total && (i0 + 1) % kLenClasses == 0) boff[(i0 + 1) / kLenClasses] = run + x0;
}

__global__ void band_append_kernel(const int32_t *__restrict__ cur, const int32_t *cur_count,
                                   int32_t *__restrict__ full_list, int32_t *full_count) {
    const int N = *cur_count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        full_list[atomicAdd(full_count, 1)] = cur[i];
}

__global__ void band_full_kused_kernel(const int32_t *__restrict__ pairs, const int64_t *__restrict__ offs,
                                       const int32_t *__restrict__ full_list, const int32_t *full_count,
                                       int32_t *__restrict__ k_used) {
    const int N = *full_count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const int p = full_list[i];
        const int x = pairs[2 * p], y = pairs[2 * p + 1];
        k_used[p] = (int)max(offs[x + 1] - offs[x], offs[y + 1] - offs[y]);
    }
}

}  // namespace msa

using namespace msa;

extern "C" {

int64_t msa_lev_banded_workspace_bytes(int64_t P, int32_t n_seqs) {
    auto r = [](int64_t b) { return (b + 255) & ~int64_t(255); };
    return r(4 * P) * 6 + r(4 * kBandMeta) + r(16) + lev_workspace(P, n_seqs);
}

}  // extern "C"

namespace msa {

msa_status lev_banded_run(msa_ctx *ctx, const msa_seqset *s, const int32_t *pairs, int64_t P, const int32_t *k0,
                          int32_t *d_out, int32_t *k_used_out, cudaStream_t st, Arena &ar) {
    msa_status rc = MSA_OK;
    int32_t *k_cur = ar.take<int32_t>(P);
    int32_t *list_a = ar.take<int32_t>(P);
    int32_t *list_b = ar.take<int32_t>(P);
    int32_t *blist = ar.take<int32_t>(P);
    int32_t *meta = ar.take<int32_t>(kBandMeta);
    int32_t *counts = ar.take<int32_t>(4);                  // count_a, count_b, full (round 0), full (later)
    // the full-DP fallback list reuses list storage: pairs that reach it are
    // never pending again, so it gets its own array
    int32_t *full_list = ar.take<int32_t>(P);
    int32_t *full_list2 = ar.take<int32_t>(P);
    if (!full_list2 || ar.cap - ar.used < lev_workspace(P, s->n_seqs))
        return set_error(ctx, MSA_ENOMEM, "msa_lev_banded_batch: needs %lld workspace bytes, context has %lld",
                         (long long)msa_lev_banded_workspace_bytes(P, s->n_seqs), (long long)ctx->ws_bytes);
    int32_t *bcount = meta, *boff = meta + kBandAll, *bcounter = meta + 2 * kBandAll;
    int32_t *ccount = meta + 3 * kBandAll, *coff = ccount + kBandAll * kLenClasses,
            *cfill = coff + kBandAll * kLenClasses;
    cudaError_t e = cudaMemcpyAsync(k_cur, k0, P * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, 4 * sizeof(int32_t), st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "msa_lev_banded_batch setup");
    const void *const *fns = s->alphabet == MSA_DNA ? kBandFnDna : kBandFnProt;
    const BandLauncher *launch = s->alphabet == MSA_DNA ? kBandDna : kBandProt;
    const int nb = kBandBuckets;
    for (int b = 1; b < nb; ++b) {
        const int c0 = band_capacity(kBandGHost[b - 1], kBandWPLHost[b - 1]);
        const int c1 = band_capacity(kBandGHost[b], kBandWPLHost[b]);
        if (c1 <= c0) return set_error(ctx, MSA_EUNSUPPORTED, "band bucket table not increasing at %d", b);
    }
    const bool lane_ok = s->alphabet == MSA_DNA;
    if (lane_ok && !ctx->band_lane_smem_set) {
        for (int c = 0; c < kLaneBuckets; ++c)
            if (lane_band_smem(kLaneWHost[c]) > 48 * 1024 &&
                (e = cudaFuncSetAttribute(kBandLaneFn[c], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)lane_band_smem(kLaneWHost[c]))) != cudaSuccess)
                return cuda_check(ctx, e, "band lane shared memory");
        ctx->band_lane_smem_set = true;
    }
    int occ[kBandAll];
    for (int b = 0; b < kBandAll; ++b)
        if (b < nb || lane_ok)
            if ((rc = occupancy(ctx, b < nb ? fns[b] : kBandLaneFn[b - nb], kBandThreads,
                                b < nb ? 0 : lane_band_smem(kLaneWHost[b - nb]), &occ[b])))
                return rc;
    // buckets beyond the first that holds a band as wide as the longest
    // sequence of this set are never used
    int last = nb - 1;
    for (int b = 0; b < nb; ++b)
        if (band_capacity(kBandGHost[b], kBandWPLHost[b]) >= s->max_len) {
            last = b;
            break;
        }
    // the launches of a round: the one-lane buckets (DNA), then the group buckets
    std::vector<int> buckets;
    if (lane_ok)
        for (int c = 0; c < kLaneBuckets; ++c) {
            buckets.push_back(nb + c);
            if (lane_capacity(kLaneWHost[c]) >= s->max_len) break;
        }
    for (int b = 0; b <= last; ++b) buckets.push_back(b);
    const int nl = (int)buckets.size();
    const int g = (int)std::min<int64_t>((P + 255) / 256, ctx->sm_count * 8);
    int32_t *cur = nullptr, *cur_count = nullptr;
    for (int r = 0; r < kBandRounds; ++r) {
        int32_t *nxt = (r & 1) ? list_b : list_a;
        int32_t *nxt_count = counts + (r & 1);
        if ((e = cudaMemsetAsync(meta, 0, kBandMeta * sizeof(int32_t), st)) != cudaSuccess ||
            (e = cudaMemsetAsync(nxt_count, 0, sizeof(int32_t), st)) != cudaSuccess)
            return cuda_check(ctx, e, "band round memset");
        // round 0 sends wide bands straight to the full DP, which then runs
        // beside the band kernels; later rounds collect theirs for the end
        int32_t *flist = r == 0 ? full_list : full_list2;
        int32_t *fcount = counts + (r == 0 ? 2 : 3);
        band_plan_kernel<0><<<std::max(g, 1), 256, 0, st>>>(pairs, P, cur, cur_count, s->offs, s->n_seqs, s->total,
                                                            k_cur, bcount, ccount, cfill, coff, blist, flist, fcount,
                                                            nb, lane_ok, ctx->dev_err);
        band_scan_kernel<<<1, 1024, 0, st>>>(ccount, coff, boff, kBandAll);
        band_plan_kernel<1><<<std::max(g, 1), 256, 0, st>>>(pairs, P, cur, cur_count, s->offs, s->n_seqs, s->total,
                                                            k_cur, bcount, ccount, cfill, coff, blist, flist, fcount,
                                                            nb, lane_ok, ctx->dev_err);
        ctx->launches += 3;
        BandArgs a{s->planes, s->codes, s->offs, pairs, blist, boff, bcount, bcounter, k_cur, d_out, k_used_out,
                   nxt, nxt_count, 0};
        {
            ProfScope prof(ctx, st);
            e = run_concurrent(ctx, st, nl, [&](int i, cudaStream_t s2) {
                BandArgs ab = a;
                ab.bucket = buckets[i];
                const int b = buckets[i];
                (b < nb ? launch[b] : kBandLane[b - nb])(ab, ctx->sm_count * occ[b], s2);
            }, 0, msa_ctx::kBandSide, /*join=*/r != 0);
            ctx->launches += nl;
            if (e != cudaSuccess) return cuda_check(ctx, e, "band launch");
            if (r == 0) {
                band_full_kused_kernel<<<std::max(g, 1), 256, 0, st>>>(pairs, s->offs, full_list, counts + 2,
                                                                       k_used_out);
                ++ctx->launches;
                Arena tmp = ar;
                if ((rc = lev_run(ctx, s, pairs, P, d_out, st, full_list, counts + 2, &tmp, msa_ctx::kBandSide)))
                    return rc;
                if ((e = join_side(ctx, st, 0, std::min(nl, msa_ctx::kBandSide))) != cudaSuccess)
                    return cuda_check(ctx, e, "band join");
            }
        }
        cur = nxt;
        cur_count = nxt_count;
    }
    // pairs still pending after the last round join the full-DP list; every
    // pair on it is computed exactly by the plain bit-vector schedule
    band_append_kernel<<<std::max(g, 1), 256, 0, st>>>(cur, cur_count, full_list2, counts + 3);
    band_full_kused_kernel<<<std::max(g, 1), 256, 0, st>>>(pairs, s->offs, full_list2, counts + 3, k_used_out);
    ctx->launches += 2;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(ctx, e, "band launch");
    return lev_run(ctx, s, pairs, P, d_out, st, full_list2, counts + 3, &ar);
}

}  // namespace msa

extern "C" {

msa_status msa_lev_banded_batch(msa_ctx *ctx, const msa_seqset *s, const int32_t *pairs, int64_t P,
                                const int32_t *k0, int32_t *d_out, int32_t *k_used_out, void *stream) {
    msa_status rc = lev_validate(ctx, s, pairs, P, d_out, "msa_lev_banded_batch");
    if (rc || P == 0) return rc;
    if (!k0 || !k_used_out) return set_error(ctx, MSA_EINVAL, "msa_lev_banded_batch: null pointer");
    if (s->n_seqs == 0) return set_error(ctx, MSA_EINVAL, "msa_lev_banded_batch: pairs given for an empty set");
    Arena ar{ctx->ws, ctx->ws_bytes};
    return lev_banded_run(ctx, s, pairs, P, k0, d_out, k_used_out, (cudaStream_t)stream, ar);
}

}  // extern "C"
