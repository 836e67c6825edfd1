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
// Kernel: one lane per pair; the longer sequence sits on the rows.  The lane
// keeps a window of WB consecutive 32-row words of the bit-vector column in
// registers (Pv, Mv and the query's bit planes, from which each column's
// match mask is formed with a few logic ops).  The window starts at the top
// and moves down one word whenever the band's first row passes a word
// boundary (at most once per 32 columns): the word leaving at the top adds
// its vertical deltas to T, the value of D on the row just above the window,
// and a fresh word (all vertical deltas +1) enters at the bottom.  The rows
// above the window are taken to grow by +1 per column (exact for row 0, an
// upper bound elsewhere), which is the carry-in of the window's top word; the
// rows below it start from the +1 vertical deltas of a fresh word, also an
// upper bound.  The window moves at warp-uniform points (every 32 steps of
// the warp's loop, each lane by as many words as its band has moved), so
// lanes never run the move separately, and the planes of the next word to
// enter are loaded one move ahead.  Trailing the band by at most one word,
// the window covers the band of half-width k_w = 32 (WB - 2) - 1, so an
// accepted pair is certified for k_w >= k.
// At the end D[m][n] = T + popc(Pv) - popc(Mv) over the window's rows <= m.
#include <cuda_runtime.h>

#include <algorithm>

#include "carry_chain.cuh"
#include "lev_kernels.cuh"
#include "msa_internal.cuh"

namespace msa {

constexpr int kBandBuckets = 18;
// buckets 0..6: one lane per pair, window of WB words in registers;
// buckets 7..17: G lanes per pair, window of G x WPL words, (G, WPL) =
// (4,4) (8,3) (8,4) (8,5) (8,6) (16,4) (16,5) (16,6) (16,8) (32,5) (32,6)
// half-widths: lane buckets 32 (WB - 2) - 1, group buckets 32 (G WPL - 1) - 1
#define BAND_KW_LIST {-1, 31, 63, 95, 127, 191, 255, 479, 735, 991, 1247, 1503, 2015, 2527, 3039, 4063, 5087, 6111}
__constant__ int kBandKW[kBandBuckets] = BAND_KW_LIST;
static const int kBandKWHost[kBandBuckets] = BAND_KW_LIST;
__constant__ int kBandCap[kBandBuckets] = {2, 3, 4, 5, 6, 8, 10, 16, 24, 32, 40, 48, 64, 80, 96, 128, 160, 192};
static const int kBandCapHost[kBandBuckets] = {2, 3, 4, 5, 6, 8, 10, 16, 24, 32, 40, 48, 64, 80, 96, 128, 160, 192};
// a window taller than this share of the column costs more than the full DP
// (the multi-lane window pays carry-lookahead and ballots per column), so
// such pairs go straight to the full bit-vector DP
constexpr float kBandMaxShare = 0.6f;
constexpr int kBandRounds = 8;
static int band_buckets(int) { return kBandBuckets; }


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
    uint32_t one, two;        // 1 and 2, as runtime values (see bv_word)
};

template <int WB, int B>
__global__ void __launch_bounds__(128) band_kernel(BandArgs a) {
    const int cnt = a.bcount[a.bucket];
    const int32_t *list = a.blist + a.boff[a.bucket];
    int32_t *counter = a.bcounter + a.bucket;
    constexpr int KW = 32 * (WB - 2) - 1;
    const uint32_t one = a.one, two = a.two;
    uint32_t Pv[WB], Mv[WB], Pl[WB][B], Pn[B];
    // per-lane pair state; a warp-synchronous loop (a vote over the whole
    // warp each iteration) so that lanes with pairs of different lengths and
    // band positions rejoin before every column
    int p = -1, m = 0, n = 0, j = 0, wlo = 0, wmax = 0, dmax = 0, T = 0, c_next = 0;
    bool full = true, has = false, more = true;
    int64_t qa = 0;
    const uint8_t *tc = nullptr;
    for (uint32_t it = 0;; ++it) {
        if (!has && more) {
            const int k = atomicAdd(counter, 1);
            if (k >= cnt) {
                more = false;
            } else {
                p = list[k];
                const int q = a.pairs[2 * p], t = a.pairs[2 * p + 1];
                int64_t qb = a.offs[q + 1], ta = a.offs[t], tb = a.offs[t + 1];
                qa = a.offs[q];
                if (qb - qa < tb - ta) {     // longer sequence on the rows
                    int64_t y = qa; qa = ta; ta = y;
                    y = qb; qb = tb; tb = y;
                }
                m = (int)(qb - qa);
                n = (int)(tb - ta);
                const int W = max(1, (m + 31) / 32);
                full = W <= WB;                        // the window holds the whole column: plain DP
                dmax = (n - m + KW) >> 1;              // floor((n - m + k_w) / 2), >= 0 since k_w >= m - n
                wmax = full ? 0 : W - WB;
                tc = a.codes + ta;
                wlo = 0;
                T = 0;
                j = 0;
                c_next = n > 0 ? __ldg(tc) : 0;
#pragma unroll
                for (int s = 0; s < WB; ++s) {
                    Pv[s] = kFull;
                    Mv[s] = 0u;
                    uint32_t mask;
                    uint32_t pl[B];
                    query_planes<B>(a.planes, qa, m, s, pl, mask);
#pragma unroll
                    for (int b = 0; b < B; ++b) Pl[s][b] = pl[b];
                }
                {
                    uint32_t mask;
                    query_planes<B>(a.planes, qa, m, WB, Pn, mask);
                }
                has = true;
            }
        }
        if (!__any_sync(kFull, has)) break;
        // warp-uniform window moves: every 32 iterations each lane catches its
        // window up with the band's first row for its next column
        if ((it & 31u) == 0u && has && !full) {
            const int num = j - dmax;            // next column is j + 1
            const int target = num < 0 ? 0 : min(num >> 5, wmax);
            while (wlo < target) {
                T += __popc(Pv[0]) - __popc(Mv[0]);
#pragma unroll
                for (int s = 0; s < WB - 1; ++s) {
                    Pv[s] = Pv[s + 1];
                    Mv[s] = Mv[s + 1];
#pragma unroll
                    for (int b = 0; b < B; ++b) Pl[s][b] = Pl[s + 1][b];
                }
                ++wlo;
                Pv[WB - 1] = kFull;
                Mv[WB - 1] = 0u;
#pragma unroll
                for (int b = 0; b < B; ++b) Pl[WB - 1][b] = Pn[b];
                uint32_t mask;
                query_planes<B>(a.planes, qa, m, wlo + WB, Pn, mask);   // one move ahead
            }
        }
        if (!has) continue;
        if (j < n) {
            ++j;
            T += 1;
            const int c = c_next;
            if (j < n) c_next = __ldg(tc + j);
            uint32_t x[B];
#pragma unroll
            for (int b = 0; b < B; ++b) x[b] = ((c >> b) & 1) ? 0u : kFull;
            uint32_t ph_in = 1u, mh_in = 0u;
#pragma unroll
            for (int s = 0; s < WB; ++s) {
                uint32_t eq = Pl[s][0] ^ x[0];
#pragma unroll
                for (int b = 1; b < B; ++b) eq &= Pl[s][b] ^ x[b];
                bv_word(eq, Pv[s], Mv[s], ph_in, mh_in, one, two);
            }
        }
        if (j == n) {
            // T = D[32 wlo][n] (exactly n while the window still starts at row 0)
            int d = T;
#pragma unroll
            for (int s = 0; s < WB; ++s) {
                const int rem = m - 32 * (wlo + s);
                const uint32_t mk = rem >= 32 ? kFull : (rem <= 0 ? 0u : ((1u << rem) - 1u));
                d += __popc(Pv[s] & mk) - __popc(Mv[s] & mk);
            }
            if (full || d <= KW) {
                a.d_out[p] = d;
                a.k_used[p] = full ? max(m, n) : KW;
            } else {
                a.k_cur[p] = 2 * KW + 1;
                a.next_list[atomicAdd(a.next_count, 1)] = p;
            }
            has = false;
        }
    }
}

// Group banded kernel: G lanes per pair (32 / G pairs per warp), the band
// window of G x WPL words spread over the group's lanes (lane l of a group
// holds window words l*WPL .. l*WPL+WPL-1); all lanes of the warp step in
// lockstep, each group on its own pair and column.  The carry of a column's
// addition crosses the group's lanes by carry-lookahead on two ballots
// (generate / propagate of each lane's WPL-word sum), the Ph/Mh top bits by
// two more; a group's window moves down one word (shuffled up from the next
// lane of the group) when its band's first row passes a word boundary, so
// the window covers the band of half-width 32 (G WPL - 1) - 1.
template <int G, int WPL, int B>
__global__ void __launch_bounds__(128) band_group_kernel(BandArgs a) {
    constexpr int NW = G * WPL;
    constexpr int KW = 32 * (NW - 1) - 1;
    constexpr uint32_t GM = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
    const int lane = threadIdx.x & 31;
    const int gl = lane % G;
    const int gbase = lane - gl;
    const int cnt = a.bcount[a.bucket];
    const int32_t *list = a.blist + a.boff[a.bucket];
    int32_t *counter = a.bcounter + a.bucket;
    uint32_t Pv[WPL], Mv[WPL], Pl[WPL][B], Pn[B];
#pragma unroll
    for (int w = 0; w < WPL; ++w) {
        Pv[w] = kFull;
        Mv[w] = 0u;
#pragma unroll
        for (int b = 0; b < B; ++b) Pl[w][b] = 0u;
    }
#pragma unroll
    for (int b = 0; b < B; ++b) Pn[b] = 0u;
    int p = -1, m = 0, n = 0, j = 0, wlo = 0, wmax = 0, dmax = 0, T = 0, c_next = 0;
    bool full = true, has = false, more = true;
    int64_t qa = 0;
    const uint8_t *tc = nullptr;
    while (true) {
        // 1. groups without a pair take the next one
        const bool need = !has && more;
        if (__any_sync(kFull, need)) {
            int k = 0;
            if (need && gl == 0) k = atomicAdd(counter, 1);
            k = __shfl_sync(kFull, k, gbase);
            if (need) {
                if (k >= cnt) {
                    more = false;
                } else {
                    p = list[k];
                    const int q = a.pairs[2 * p], t = a.pairs[2 * p + 1];
                    int64_t qb = a.offs[q + 1], ta = a.offs[t], tb = a.offs[t + 1];
                    qa = a.offs[q];
                    if (qb - qa < tb - ta) {     // longer sequence on the rows
                        int64_t y = qa; qa = ta; ta = y;
                        y = qb; qb = tb; tb = y;
                    }
                    m = (int)(qb - qa);
                    n = (int)(tb - ta);
                    const int W = max(1, (m + 31) / 32);
                    full = W <= NW;
                    dmax = (n - m + KW) >> 1;
                    wmax = full ? 0 : W - NW;
                    tc = a.codes + ta;
                    wlo = 0;
                    T = 0;
                    j = 0;
                    c_next = n > 0 ? __ldg(tc) : 0;
#pragma unroll
                    for (int w = 0; w < WPL; ++w) {
                        Pv[w] = kFull;
                        Mv[w] = 0u;
                        uint32_t mask;
                        uint32_t pl[B];
                        query_planes<B>(a.planes, qa, m, gl * WPL + w, pl, mask);
#pragma unroll
                        for (int b = 0; b < B; ++b) Pl[w][b] = pl[b];
                    }
                    if (gl == G - 1) {
                        uint32_t mask;
                        query_planes<B>(a.planes, qa, m, NW, Pn, mask);
                    }
                    has = true;
                }
            }
        }
        if (!__any_sync(kFull, has)) break;
        // 2. window moves before the next column (j + 1)
        bool move = false;
        if (has && !full && j < n) {
            const int num = j - dmax;
            const int target = num < 0 ? 0 : min(num >> 5, wmax);
            move = target > wlo;
        }
        if (__any_sync(kFull, move)) {
            const int dT = __shfl_sync(kFull, __popc(Pv[0]) - __popc(Mv[0]), gbase);
            const uint32_t pv0 = __shfl_down_sync(kFull, Pv[0], 1, G);
            const uint32_t mv0 = __shfl_down_sync(kFull, Mv[0], 1, G);
            uint32_t pl0[B];
#pragma unroll
            for (int b = 0; b < B; ++b) pl0[b] = __shfl_down_sync(kFull, Pl[0][b], 1, G);
            if (move) {
                T += dT;
#pragma unroll
                for (int w = 0; w < WPL - 1; ++w) {
                    Pv[w] = Pv[w + 1];
                    Mv[w] = Mv[w + 1];
#pragma unroll
                    for (int b = 0; b < B; ++b) Pl[w][b] = Pl[w + 1][b];
                }
                ++wlo;
                if (gl == G - 1) {
                    Pv[WPL - 1] = kFull;
                    Mv[WPL - 1] = 0u;
#pragma unroll
                    for (int b = 0; b < B; ++b) Pl[WPL - 1][b] = Pn[b];
                    uint32_t mask;
                    query_planes<B>(a.planes, qa, m, wlo + NW, Pn, mask);   // one move ahead
                } else {
                    Pv[WPL - 1] = pv0;
                    Mv[WPL - 1] = mv0;
#pragma unroll
                    for (int b = 0; b < B; ++b) Pl[WPL - 1][b] = pl0[b];
                }
            }
        }
        // 3. one column for every group that has one
        const bool act = has && j < n;
        const int c = c_next;
        uint32_t x[B];
#pragma unroll
        for (int b = 0; b < B; ++b) x[b] = ((c >> b) & 1) ? 0u : kFull;
        uint32_t eq[WPL], u[WPL], s0[WPL];
#pragma unroll
        for (int w = 0; w < WPL; ++w) {
            uint32_t e = Pl[w][0] ^ x[0];
#pragma unroll
            for (int b = 1; b < B; ++b) e &= Pl[w][b] ^ x[b];
            eq[w] = e;
            u[w] = e & Pv[w];
        }
        // the lane's words added on the carry chain with carry-in 0
        const uint32_t cy = CarryChain<WPL>::add(s0, u, Pv);
        uint32_t all = kFull;
#pragma unroll
        for (int w = 0; w < WPL; ++w) all &= s0[w];
        // carry into each lane of the group: c_{l+1} = g_l | (p_l & c_l), c_0 = 0
        const uint32_t Gb = (__ballot_sync(kFull, act && cy != 0u) >> gbase) & GM;
        const uint32_t Pb = (__ballot_sync(kFull, act && all == kFull) >> gbase) & GM;
        const uint32_t GP = Gb | Pb;
        const uint32_t carries = (Gb + GP) ^ GP ^ Gb;
        const uint32_t ci = gl == 0 ? 0u : (carries >> gl) & 1u;
        CarryChain<WPL>::inc(s0, ci);
        uint32_t ph[WPL], mh[WPL];
#pragma unroll
        for (int w = 0; w < WPL; ++w) {
            const uint32_t xh = (s0[w] ^ Pv[w]) | eq[w];
            ph[w] = Mv[w] | ~(xh | Pv[w]);
            mh[w] = Pv[w] & xh;
        }
        const uint32_t PT = (__ballot_sync(kFull, (ph[WPL - 1] >> 31) != 0u) >> gbase) & GM;
        const uint32_t MT = (__ballot_sync(kFull, (mh[WPL - 1] >> 31) != 0u) >> gbase) & GM;
        if (act) {
            uint32_t ph_in = gl == 0 ? 1u : (PT >> (gl - 1)) & 1u;
            uint32_t mh_in = gl == 0 ? 0u : (MT >> (gl - 1)) & 1u;
#pragma unroll
            for (int w = 0; w < WPL; ++w) {
                const uint32_t phs = (ph[w] << 1) | ph_in;
                const uint32_t mhs = (mh[w] << 1) | mh_in;
                ph_in = ph[w] >> 31;
                mh_in = mh[w] >> 31;
                const uint32_t xv = eq[w] | Mv[w];
                Pv[w] = mhs | ~(xv | phs);
                Mv[w] = phs & xv;
            }
            ++j;
            T += 1;
            if (j < n) c_next = __ldg(tc + j);
        }
        // 4. groups whose pair is done report it
        const bool fin = has && j == n;
        if (__any_sync(kFull, fin)) {
            int part = 0;
            if (fin) {
#pragma unroll
                for (int w = 0; w < WPL; ++w) {
                    const int rem = m - 32 * (wlo + gl * WPL + w);
                    const uint32_t mk = rem >= 32 ? kFull : (rem <= 0 ? 0u : ((1u << rem) - 1u));
                    part += __popc(Pv[w] & mk) - __popc(Mv[w] & mk);
                }
            }
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o, G);
            if (fin) {
                if (gl == 0) {
                    const int d = T + part;
                    if (full || d <= KW) {
                        a.d_out[p] = d;
                        a.k_used[p] = full ? max(m, n) : KW;
                    } else {
                        a.k_cur[p] = 2 * KW + 1;
                        a.next_list[atomicAdd(a.next_count, 1)] = p;
                    }
                }
                has = false;
            }
        }
    }
}

using BandLauncher = void (*)(const BandArgs &, int, cudaStream_t);

template <int WB, int B>
void launch_band(const BandArgs &a, int grid, cudaStream_t st) {
    band_kernel<WB, B><<<grid, 128, 0, st>>>(a);
}

template <int G, int WPL, int B>
void launch_band_group(const BandArgs &a, int grid, cudaStream_t st) {
    band_group_kernel<G, WPL, B><<<grid, 128, 0, st>>>(a);
}

#define BAND_TABLE(B)                                                                                        \
    {launch_band<2, B>, launch_band<3, B>, launch_band<4, B>, launch_band<5, B>, launch_band<6, B>,          \
     launch_band<8, B>, launch_band<10, B>, launch_band_group<4, 4, B>, launch_band_group<8, 3, B>,           \
     launch_band_group<8, 4, B>, launch_band_group<8, 5, B>, launch_band_group<8, 6, B>,                      \
     launch_band_group<16, 4, B>, launch_band_group<16, 5, B>, launch_band_group<16, 6, B>,                  \
     launch_band_group<16, 8, B>, launch_band_group<32, 5, B>, launch_band_group<32, 6, B>}
#define BAND_FNS(B)                                                                                          \
    {(const void *)band_kernel<2, B>, (const void *)band_kernel<3, B>, (const void *)band_kernel<4, B>,      \
     (const void *)band_kernel<5, B>, (const void *)band_kernel<6, B>, (const void *)band_kernel<8, B>,      \
     (const void *)band_kernel<10, B>, (const void *)band_group_kernel<4, 4, B>,                             \
     (const void *)band_group_kernel<8, 3, B>, (const void *)band_group_kernel<8, 4, B>,                     \
     (const void *)band_group_kernel<8, 5, B>, (const void *)band_group_kernel<8, 6, B>,                     \
     (const void *)band_group_kernel<16, 4, B>, (const void *)band_group_kernel<16, 5, B>,                   \
     (const void *)band_group_kernel<16, 6, B>, (const void *)band_group_kernel<16, 8, B>,                   \
     (const void *)band_group_kernel<32, 5, B>, (const void *)band_group_kernel<32, 6, B>}
static const BandLauncher kBandDna[kBandBuckets] = BAND_TABLE(2);
static const BandLauncher kBandProt[kBandBuckets] = BAND_TABLE(5);
static const void *kBandFnDna[kBandBuckets] = BAND_FNS(2);
static const void *kBandFnProt[kBandBuckets] = BAND_FNS(5);

// Sorts the pending pairs of one round into window buckets (pass 0 counts,
// pass 1 writes); pairs whose band needs more than the largest window go to
// the exact full-DP list.  Round 0 reads all pairs (cur == nullptr) and
// checks every index.
template <int PASS>
__global__ void __launch_bounds__(256) band_plan_kernel(const int32_t *__restrict__ pairs, int64_t P,
                                                        const int32_t *__restrict__ cur, const int32_t *cur_count,
                                                        const int64_t *__restrict__ offs, int32_t n, int64_t total,
                                                        int32_t *__restrict__ k_cur, int32_t *__restrict__ bcount,
                                                        int32_t *__restrict__ bfill, int32_t *__restrict__ boff,
                                                        int32_t *__restrict__ blist, int32_t *__restrict__ full_list,
                                                        int32_t *full_count, int32_t nb, int32_t *err) {
    __shared__ int32_t sboff[kBandBuckets];
    if (PASS == 1) {
        if (threadIdx.x == 0) {
            int run = 0;
            for (int b = 0; b < nb; ++b) {
                sboff[b] = run;
                run += bcount[b];
            }
        }
        __syncthreads();
        if (blockIdx.x == 0 && threadIdx.x < nb) boff[threadIdx.x] = sboff[threadIdx.x];
    }
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
        const int W = max(1, (m + 31) / 32);
        const int k = max(k_cur[p], dl);
        int b = -1;
        if (k < m) {
            for (int c = 0; c < nb; ++c)
                if (kBandCap[c] >= W || kBandKW[c] >= k) {
                    b = c;
                    break;
                }
            if (b >= 0 && kBandCap[b] < W && (float)kBandCap[b] > kBandMaxShare * (float)W) b = -1;
        } else {
            // the band is the whole matrix: a window as tall as the column is a plain DP
            for (int c = 0; c < nb; ++c)
                if (kBandCap[c] >= W) {
                    b = c;
                    break;
                }
        }
        if (PASS == 0) {
            if (b < 0)
                full_list[atomicAdd(full_count, 1)] = p;
            else
                atomicAdd(bcount + b, 1);
        } else if (b >= 0) {
            blist[sboff[b] + atomicAdd(bfill + b, 1)] = p;
        }
    }
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
    return r(4 * P) * 6 + r(4 * 4 * kBandBuckets) + r(16) + lev_workspace(P, n_seqs);
}

msa_status msa_lev_banded_batch(msa_ctx *ctx, const msa_seqset *s, const int32_t *pairs, int64_t P,
                                const int32_t *k0, int32_t *d_out, int32_t *k_used_out, void *stream) {
    msa_status rc = lev_validate(ctx, s, pairs, P, d_out, "msa_lev_banded_batch");
    if (rc || P == 0) return rc;
    if (!k0 || !k_used_out) return set_error(ctx, MSA_EINVAL, "msa_lev_banded_batch: null pointer");
    if (s->n_seqs == 0) return set_error(ctx, MSA_EINVAL, "msa_lev_banded_batch: pairs given for an empty set");
    cudaStream_t st = (cudaStream_t)stream;
    Arena ar{ctx->ws, ctx->ws_bytes};
    int32_t *k_cur = ar.take<int32_t>(P);
    int32_t *list_a = ar.take<int32_t>(P);
    int32_t *list_b = ar.take<int32_t>(P);
    int32_t *blist = ar.take<int32_t>(P);
    int32_t *meta = ar.take<int32_t>(4 * kBandBuckets);     // bcount, bfill, boff, bcounter
    int32_t *counts = ar.take<int32_t>(4);                  // count_a, count_b, full (round 0), full (later)
    // the full-DP fallback list reuses list storage: pairs that reach it are
    // never pending again, so it gets its own array
    int32_t *full_list = ar.take<int32_t>(P);
    int32_t *full_list2 = ar.take<int32_t>(P);
    if (!full_list2 || ar.cap - ar.used < lev_workspace(P, s->n_seqs))
        return set_error(ctx, MSA_ENOMEM, "msa_lev_banded_batch: needs %lld workspace bytes, context has %lld",
                         (long long)msa_lev_banded_workspace_bytes(P, s->n_seqs), (long long)ctx->ws_bytes);
    int32_t *bcount = meta, *bfill = meta + kBandBuckets, *boff = meta + 2 * kBandBuckets,
            *bcounter = meta + 3 * kBandBuckets;
    cudaError_t e = cudaMemcpyAsync(k_cur, k0, P * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, 4 * sizeof(int32_t), st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "msa_lev_banded_batch setup");
    const void *const *fns = s->alphabet == MSA_DNA ? kBandFnDna : kBandFnProt;
    const BandLauncher *launch = s->alphabet == MSA_DNA ? kBandDna : kBandProt;
    const int nb = band_buckets(s->alphabet);
    {
        static const int wb[7] = {2, 3, 4, 5, 6, 8, 10};
        for (int b = 0; b < kBandBuckets; ++b) {
            const int expect = b < 7 ? 32 * (wb[b] - 2) - 1 : 32 * (kBandCapHost[b] - 1) - 1;
            if (kBandKWHost[b] != expect || (b < 7 && kBandCapHost[b] != wb[b]))
                return set_error(ctx, MSA_EUNSUPPORTED, "band bucket table inconsistent at %d", b);
        }
    }
    static int occ[2][kBandBuckets] = {};
    for (int b = 0; b < nb; ++b)
        if (occ[s->alphabet][b] == 0) {
            int o = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fns[b], 128, 0);
            if (e != cudaSuccess) return cuda_check(ctx, e, "band occupancy");
            occ[s->alphabet][b] = std::max(o, 1);
        }
    // windows taller than any sequence of this set are never needed beyond the first that holds it
    const int Wmax = std::max(1, (s->max_len + 31) / 32);
    int last = nb - 1;
    for (int b = 0; b < nb; ++b)
        if (kBandCapHost[b] >= Wmax) {
            last = b;
            break;
        }
    const int g = (int)std::min<int64_t>((P + 255) / 256, ctx->sm_count * 8);
    int32_t *cur = nullptr, *cur_count = nullptr;
    for (int r = 0; r < kBandRounds; ++r) {
        int32_t *nxt = (r & 1) ? list_b : list_a;
        int32_t *nxt_count = counts + (r & 1);
        if ((e = cudaMemsetAsync(meta, 0, 4 * kBandBuckets * sizeof(int32_t), st)) != cudaSuccess ||
            (e = cudaMemsetAsync(nxt_count, 0, sizeof(int32_t), st)) != cudaSuccess)
            return cuda_check(ctx, e, "band round memset");
        // round 0 sends wide bands straight to the full DP, which then runs
        // beside the band kernels; later rounds collect theirs for the end
        int32_t *flist = r == 0 ? full_list : full_list2;
        int32_t *fcount = counts + (r == 0 ? 2 : 3);
        band_plan_kernel<0><<<std::max(g, 1), 256, 0, st>>>(pairs, P, cur, cur_count, s->offs, s->n_seqs, s->total,
                                                            k_cur, bcount, bfill, boff, blist, flist, fcount,
                                                            nb, ctx->dev_err);
        band_plan_kernel<1><<<std::max(g, 1), 256, 0, st>>>(pairs, P, cur, cur_count, s->offs, s->n_seqs, s->total,
                                                            k_cur, bcount, bfill, boff, blist, flist, fcount,
                                                            nb, ctx->dev_err);
        ctx->launches += 2;
        BandArgs a{s->planes, s->codes, s->offs, pairs, blist, boff, bcount, bcounter, k_cur, d_out, k_used_out,
                   nxt, nxt_count, 0, 1u, 2u};
        {
            ProfScope prof(ctx, st);
            e = run_concurrent(ctx, st, last + 1, [&](int b, cudaStream_t s2) {
                BandArgs ab = a;
                ab.bucket = b;
                launch[b](ab, ctx->sm_count * occ[s->alphabet][b], s2);
            }, 0, 8, /*join=*/r != 0);
            ctx->launches += last + 1;
            if (e != cudaSuccess) return cuda_check(ctx, e, "band launch");
            if (r == 0) {
                band_full_kused_kernel<<<std::max(g, 1), 256, 0, st>>>(pairs, s->offs, full_list, counts + 2,
                                                                       k_used_out);
                ++ctx->launches;
                Arena tmp = ar;
                if ((rc = lev_run(ctx, s, pairs, P, d_out, st, full_list, counts + 2, &tmp, 8))) return rc;
                if ((e = join_side(ctx, st, 0, std::min(last + 1, 8))) != cudaSuccess)
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

}  // extern "C"
