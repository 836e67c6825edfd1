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

#include "lev_kernels.cuh"
#include "msa_internal.cuh"

namespace msa {

constexpr int kBandBuckets = 13;
__constant__ int kBandWB[kBandBuckets] = {2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 24, 32, 40};
static const int kBandWBHost[kBandBuckets] = {2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 24, 32, 40};
constexpr int kBandRounds = 8;
// windows held in registers without spilling: DNA up to 32 words (k_w 991),
// protein (5 bit planes per word) up to 16 words (k_w 479)
static int band_buckets(int alphabet) { return alphabet == MSA_DNA ? 12 : 9; }

// The window may trail its ideal position by one word between two moves
// (moves happen at warp-uniform points, every 32 steps), so a window of WB
// words covers the band of half-width 32 (WB - 2) - 1.
__host__ __device__ __forceinline__ int band_kw(int WB) { return 32 * (WB - 2) - 1; }

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

using BandLauncher = void (*)(const BandArgs &, int, cudaStream_t);

template <int WB, int B>
void launch_band(const BandArgs &a, int grid, cudaStream_t st) {
    band_kernel<WB, B><<<grid, 128, 0, st>>>(a);
}

static const BandLauncher kBandDna[kBandBuckets] = {
    launch_band<2, 2>,  launch_band<3, 2>,  launch_band<4, 2>,  launch_band<5, 2>,  launch_band<6, 2>,
    launch_band<8, 2>,  launch_band<10, 2>, launch_band<12, 2>, launch_band<16, 2>, launch_band<20, 2>,
    launch_band<24, 2>, launch_band<32, 2>, nullptr};
static const BandLauncher kBandProt[kBandBuckets] = {
    launch_band<2, 5>, launch_band<3, 5>,  launch_band<4, 5>,  launch_band<5, 5>, launch_band<6, 5>,
    launch_band<8, 5>, launch_band<10, 5>, launch_band<12, 5>, launch_band<16, 5>, nullptr, nullptr, nullptr, nullptr};
static const void *kBandFnDna[kBandBuckets] = {
    (const void *)band_kernel<2, 2>,  (const void *)band_kernel<3, 2>,  (const void *)band_kernel<4, 2>,
    (const void *)band_kernel<5, 2>,  (const void *)band_kernel<6, 2>,  (const void *)band_kernel<8, 2>,
    (const void *)band_kernel<10, 2>, (const void *)band_kernel<12, 2>, (const void *)band_kernel<16, 2>,
    (const void *)band_kernel<20, 2>, (const void *)band_kernel<24, 2>, (const void *)band_kernel<32, 2>, nullptr};
static const void *kBandFnProt[kBandBuckets] = {
    (const void *)band_kernel<2, 5>,  (const void *)band_kernel<3, 5>,  (const void *)band_kernel<4, 5>,
    (const void *)band_kernel<5, 5>,  (const void *)band_kernel<6, 5>,  (const void *)band_kernel<8, 5>,
    (const void *)band_kernel<10, 5>, (const void *)band_kernel<12, 5>, (const void *)band_kernel<16, 5>,
    nullptr, nullptr, nullptr, nullptr};

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
                if (kBandWB[c] >= W || band_kw(kBandWB[c]) >= k) {
                    b = c;
                    break;
                }
        } else {
            // the band is the whole matrix: a window as tall as the column is a plain DP
            for (int c = 0; c < nb; ++c)
                if (kBandWB[c] >= W) {
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
    return r(4 * P) * 4 + r(4 * 4 * kBandBuckets) + r(16) + lev_workspace(P, n_seqs);
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
    int32_t *counts = ar.take<int32_t>(4);                  // count_a, count_b, full_count
    // the full-DP fallback list reuses list storage: pairs that reach it are
    // never pending again, so it gets its own array
    int32_t *full_list = ar.take<int32_t>(P);
    if (!full_list || ar.cap - ar.used < lev_workspace(P, s->n_seqs))
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
        if (kBandWBHost[b] >= Wmax) {
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
        band_plan_kernel<0><<<std::max(g, 1), 256, 0, st>>>(pairs, P, cur, cur_count, s->offs, s->n_seqs, s->total,
                                                            k_cur, bcount, bfill, boff, blist, full_list, counts + 2,
                                                            nb, ctx->dev_err);
        band_plan_kernel<1><<<std::max(g, 1), 256, 0, st>>>(pairs, P, cur, cur_count, s->offs, s->n_seqs, s->total,
                                                            k_cur, bcount, bfill, boff, blist, full_list, counts + 2,
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
            });
            ctx->launches += last + 1;
            if (e != cudaSuccess) return cuda_check(ctx, e, "band launch");
        }
        cur = nxt;
        cur_count = nxt_count;
    }
    // pairs still pending after the last round join the full-DP list; every
    // pair on it is computed exactly by the plain bit-vector schedule
    band_append_kernel<<<std::max(g, 1), 256, 0, st>>>(cur, cur_count, full_list, counts + 2);
    band_full_kused_kernel<<<std::max(g, 1), 256, 0, st>>>(pairs, s->offs, full_list, counts + 2, k_used_out);
    ctx->launches += 2;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(ctx, e, "band launch");
    return lev_run(ctx, s, pairs, P, d_out, st, full_list, counts + 2, &ar);
}

}  // extern "C"
