// Alignment quality of an MSA (section "Evaluation"): percentage of gaps,
// p-score and distance distortion over a sample of its rows, and the C entry
// point msa_msa_metrics.
//
// * Gaps and p-score come from per-column byte histograms of the sampled
//   rows: a column with g gaps and counts c_b of the other bytes holds
//   C(S - g, 2) pairs of non-gap units, sum_b C(c_b, 2) of them equal.
// * Distortion: the Levenshtein distance of every sampled pair (the library's
//   batch schedule, in chunks) and the Hamming distance of their aligned rows.
//   Rows are bit-sliced into 8 planes per 32 columns (plane p holds bit p of
//   each byte), so two rows differ in column k of a word iff bit k of
//   OR_p (x_p ^ y_p) is set: 8 logic ops and a popcount per 32 columns.  A
//   block takes a 64 x 64 tile of pairs (upper triangle), 16 pairs a thread,
//   staging the tiles' plane words in shared memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "msa_internal.cuh"

namespace msa {

constexpr int kMetTile = 64;          // rows per tile side
constexpr int kMetChunk = 8;          // plane words staged per round

// Per-column byte histograms over the sampled rows; 32 columns per block.
__global__ void __launch_bounds__(256) metric_hist_kernel(const uint8_t *__restrict__ rows, int64_t W, int R,
                                                          const int32_t *__restrict__ sample, int S, uint8_t gap,
                                                          unsigned long long *tot, int32_t *err) {
    __shared__ uint32_t h[32][256];
    const int cl = threadIdx.x & 31, rg = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < 32 * 256; i += blockDim.x) (&h[0][0])[i] = 0u;
    __syncthreads();
    const int64_t col = (int64_t)blockIdx.x * 32 + cl;
    if (col < W)
        for (int r = rg; r < S; r += 8) {
            const int row = sample[r];
            if (row < 0 || row >= R) {
                if (col == 0) record_error(err, kErrIndex, r, row);
                continue;
            }
            atomicAdd(&h[cl][rows[(int64_t)row * W + col]], 1u);
        }
    __syncthreads();
    if (rg == 0 && col < W) {
        const unsigned long long g = h[cl][gap];
        const unsigned long long ng = (unsigned long long)S - g;
        unsigned long long same = 0;
        for (int b = 0; b < 256; ++b) {
            const unsigned long long c = h[cl][b];
            if (b != gap && c > 1) same += c * (c - 1) / 2;
        }
        const unsigned long long cmp = ng * (ng > 0 ? ng - 1 : 0) / 2;
        atomicAdd(tot + 0, g);
        atomicAdd(tot + 1, cmp);
        atomicAdd(tot + 2, cmp - same);
    }
}

// Bit planes of the sampled rows: planes[(r * Wp + w) * 8 + p], bit k = bit p
// of the byte at column 32 w + k (bytes past W are 0 in every row).
__global__ void metric_planes_kernel(const uint8_t *__restrict__ rows, int64_t W, int R,
                                     const int32_t *__restrict__ sample, int S, int64_t Wp,
                                     uint32_t *__restrict__ planes) {
    const int64_t n = (int64_t)S * Wp;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / Wp, w = t % Wp;
        const int ri = sample[r];
        const uint8_t *row = rows + (int64_t)(ri >= 0 && ri < R ? ri : 0) * W;     // bad indices reported above
        uint32_t pl[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int k = 0; k < 32; ++k) {
            const int64_t c = 32 * w + k;
            const uint32_t b = c < W ? row[c] : 0u;
#pragma unroll
            for (int p = 0; p < 8; ++p) pl[p] |= ((b >> p) & 1u) << k;
        }
#pragma unroll
        for (int p = 0; p < 8; ++p) planes[t * 8 + p] = pl[p];
    }
}

// Pair p of the sampled rows in the order (0,1), (0,2), .., (1,2), ..: row i
// starts at off(i) = i S - i (i + 1) / 2.
__device__ __forceinline__ int64_t metric_pair_off(int64_t i, int64_t S) { return i * S - i * (i + 1) / 2; }

__global__ void metric_pairs_kernel(const int32_t *__restrict__ seq_of, int S, int64_t p0, int64_t np,
                                    int32_t *__restrict__ pairs) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < np; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = p0 + t;
        int64_t lo = 0, hi = S - 1;             // largest i with off(i) <= p
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) / 2;
            if (metric_pair_off(mid, S) <= p) lo = mid;
            else hi = mid - 1;
        }
        const int64_t j = p - metric_pair_off(lo, S) + lo + 1;
        pairs[2 * t] = seq_of[lo];
        pairs[2 * t + 1] = seq_of[j];
    }
}

__global__ void __launch_bounds__(256) metric_hamming_kernel(const uint32_t *__restrict__ planes, int S, int64_t Wp,
                                                             const int32_t *__restrict__ lev, int ntile,
                                                             double *sum, unsigned long long *cnt) {
    // rows padded to 65 words: threads reading 16 different rows hit 16 banks
    __shared__ uint32_t sI[kMetTile][kMetChunk * 8 + 1];
    __shared__ uint32_t sJ[kMetTile][kMetChunk * 8 + 1];
    __shared__ double red[256];
    __shared__ unsigned long long redc[256];
    // tile (ti, tj) with ti <= tj from the block index
    int64_t b = blockIdx.x;
    int ti = 0;
    while (b >= ntile - ti) {
        b -= ntile - ti;
        ++ti;
    }
    const int tj = ti + (int)b;
    const int I0 = ti * kMetTile, J0 = tj * kMetTile;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    int H[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) H[a][c] = 0;
    for (int64_t w0 = 0; w0 < Wp; w0 += kMetChunk) {
        __syncthreads();
        for (int e = threadIdx.x; e < kMetTile * kMetChunk * 8; e += blockDim.x) {
            const int r = e / (kMetChunk * 8), w = (e / 8) % kMetChunk, p = e % 8;
            const int64_t wg = w0 + w;
            const int ri = I0 + r, rj = J0 + r;
            sI[r][w * 8 + p] = (ri < S && wg < Wp) ? planes[((int64_t)ri * Wp + wg) * 8 + p] : 0u;
            sJ[r][w * 8 + p] = (rj < S && wg < Wp) ? planes[((int64_t)rj * Wp + wg) * 8 + p] : 0u;
        }
        __syncthreads();
        for (int w = 0; w < kMetChunk; ++w) {
            uint32_t x[4][8], y[4][8];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int p = 0; p < 8; ++p) {
                    x[a][p] = sI[ty + 16 * a][w * 8 + p];
                    y[a][p] = sJ[tx + 16 * a][w * 8 + p];
                }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    uint32_t d = 0u;
#pragma unroll
                    for (int p = 0; p < 8; ++p) d |= x[a][p] ^ y[c][p];
                    H[a][c] += __popc(d);
                }
        }
    }
    double s = 0.0;
    unsigned long long n = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t i = I0 + ty + 16 * a, j = J0 + tx + 16 * c;
            if (i < j && j < S) {
                const int32_t f = lev[metric_pair_off(i, S) + (j - i - 1)];
                if (f > 0) {                 // identical sequences have no ratio and are left out
                    s += (double)H[a][c] / (double)f;
                    ++n;
                }
            }
        }
    red[threadIdx.x] = s;
    redc[threadIdx.x] = n;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            red[threadIdx.x] += red[threadIdx.x + o];
            redc[threadIdx.x] += redc[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(sum, red[0]);
        atomicAdd(cnt, redc[0]);
    }
}

}  // namespace msa

using namespace msa;

extern "C" {

msa_status msa_msa_metrics(msa_ctx *ctx, const msa_seqset *s, const uint8_t *rows, int32_t R, int32_t W,
                           const int32_t *sample_rows, const int32_t *sample_seqs, int32_t S, uint8_t gap,
                           double *out3, int64_t *counts4, void *stream) {
    if (!ctx) return MSA_EINVAL;
    if (!s || !rows || !sample_rows || !sample_seqs || !out3)
        return set_error(ctx, MSA_EINVAL, "msa_msa_metrics: null pointer");
    if (W <= 0 || S < 2 || R < 1) return set_error(ctx, MSA_EINVAL, "msa_msa_metrics: needs W > 0 and at least 2 rows");
    cudaStream_t st = (cudaStream_t)stream;
    Arena ar{ctx->ws, ctx->ws_bytes};
    const int64_t Wp = ((int64_t)W + 31) / 32;
    const int64_t npairs = (int64_t)S * (S - 1) / 2;
    unsigned long long *tot = ar.take<unsigned long long>(8);
    double *dsum = ar.take<double>(1);
    uint32_t *planes = ar.take<uint32_t>((int64_t)S * Wp * 8);
    int32_t *lev = ar.take<int32_t>(npairs);
    if (!lev) return set_error(ctx, MSA_ENOMEM, "msa_msa_metrics: %d rows need more workspace", S);
    cudaError_t e = cudaMemsetAsync(tot, 0, 8 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dsum, 0, sizeof(double), st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "msa_msa_metrics memset");
    ProfScope prof(ctx, st);
    metric_hist_kernel<<<(int)((W + 31) / 32), 256, 0, st>>>(rows, W, R, sample_rows, S, gap, tot, ctx->dev_err);
    metric_planes_kernel<<<(int)std::min<int64_t>((S * Wp + 255) / 256, ctx->sm_count * 8), 256, 0, st>>>(
        rows, W, R, sample_rows, S, Wp, planes);
    ctx->launches += 2;
    // Levenshtein distances of the sampled pairs, in chunks that fit the rest of the workspace
    int64_t chunk = std::min<int64_t>(npairs, 1 << 23);
    while (chunk > 0) {
        Arena t = ar;
        int32_t *pp = t.take<int32_t>(2 * chunk);
        if (pp && t.cap - t.used >= lev_workspace(chunk, s->n_seqs)) break;
        chunk /= 2;
    }
    if (chunk <= 0) return set_error(ctx, MSA_ENOMEM, "msa_msa_metrics: workspace too small for the distance batches");
    msa_status rc;
    for (int64_t p0 = 0; p0 < npairs; p0 += chunk) {
        const int64_t np = std::min(chunk, npairs - p0);
        Arena t = ar;
        int32_t *pp = t.take<int32_t>(2 * np);
        metric_pairs_kernel<<<(int)std::min<int64_t>((np + 255) / 256, ctx->sm_count * 8), 256, 0, st>>>(
            sample_seqs, S, p0, np, pp);
        ++ctx->launches;
        if ((rc = lev_run(ctx, s, pp, np, lev + p0, st, nullptr, nullptr, &t))) return rc;
    }
    const int ntile = (S + kMetTile - 1) / kMetTile;
    const int64_t nblocks = (int64_t)ntile * (ntile + 1) / 2;
    metric_hamming_kernel<<<(int)nblocks, 256, 0, st>>>(planes, S, Wp, lev, ntile, dsum, tot + 3);
    ++ctx->launches;
    unsigned long long h[4];
    double hs = 0.0;
    if ((e = cudaMemcpyAsync(h, tot, sizeof h, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&hs, dsum, sizeof hs, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_check(ctx, e, "msa_msa_metrics readback");
    if ((rc = msa_ctx_check(ctx, stream))) return rc;
    out3[0] = 100.0 * (double)h[0] / ((double)S * (double)W);
    out3[1] = h[1] ? 100.0 * (double)h[2] / (double)h[1] : 0.0;
    out3[2] = h[3] ? hs / (double)h[3] : 0.0;
    if (counts4) {
        counts4[0] = (int64_t)h[0];
        counts4[1] = (int64_t)h[1];
        counts4[2] = (int64_t)h[2];
        counts4[3] = (int64_t)h[3];
    }
    return MSA_OK;
}

}  // extern "C"
