// Batched Levenshtein distance: device-side schedule (A7) and the C entry
// points msa_lev_batch / msa_lev_autotune.
//
// Schedule of one call, all on the device (no host round trip, so the whole
// call can be captured in a CUDA graph):
//   1. count pairs per first index q (the query), checking every index;
//   2. exclusive scan -> group starts; scatter (target, pair id) by query;
//      the targets of each query with many of them ordered longest first;
//   3. per query pick a kernel configuration from its word count
//      W = ceil(m / 32) and its number of targets c_q: the lane kernel
//      (one warp per query, a lane per target) when W <= 64 and c_q is large
//      enough, otherwise the warp kernel (32 lanes per target); split the
//      query into ceil(c_q / per_task) tasks and append them to the bucket of
//      that configuration;
//   4. one persistent launch per bucket; warps pull tasks from the bucket's
//      counter and, inside a task, targets from the query's shared cursor.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "lev_kernels.cuh"
#include "warp_agg.cuh"
#include "msa_internal.cuh"

namespace msa {

constexpr int kMaxBuckets = 64;

struct Tune {
    int lane_min_targets = 32;  // a query with fewer targets shares a warp (slot kernel)
    int slot_min_targets = 2;   // below this a query goes to the warp kernel
    int lane_per_task = 0;      // targets per task, lane kernel (0: from the batch size)
    int warp_per_task = 4;      // targets per task, warp kernel
    int occupancy[2][kMaxBuckets] = {};  // blocks per SM, per alphabet and bucket
};

Tune *create_tune() { return new Tune(); }
void destroy_tune(Tune *t) { delete t; }

// Buckets: [lane kernels | slot kernels (same word counts) | warp kernels].
struct Registry {
    const LevKernelInfo *lane;
    int nlane;
    const LevKernelInfo *slot;
    const LevKernelInfo *warp;
    int nwarp;
    int count() const { return 2 * nlane + nwarp; }
    const LevKernelInfo &at(int b) const {
        return b < nlane ? lane[b] : b < 2 * nlane ? slot[b - nlane] : warp[b - 2 * nlane];
    }
};

static Registry registry(int alphabet) {
    static_assert(2 * 23 + 16 <= kMaxBuckets, "bucket table too small");
    if (alphabet == MSA_DNA) return {kLevLaneDna, kLevLaneDnaCount, kLevSlotDna, kLevWarpDna, kLevWarpDnaCount};
    return {kLevLaneProt, kLevLaneProtCount, kLevSlotProt, kLevWarpProt, kLevWarpProtCount};
}

struct PlanParams {
    int nlane, nwarp;
    int lane_words[32];
    int warp_words[32];
    int lane_min_targets;
    int slot_min_targets;
    int lane_per_task;
    int warp_per_task;
};

// Lane kernel for queries with many targets, slot kernel (several queries
// per warp) for those with a few, warp kernel for single targets and for
// queries longer than the lane kernels' registers hold.
__device__ __forceinline__ int pick_bucket(const PlanParams &pp, int W, int c) {
    if (W <= pp.lane_words[pp.nlane - 1] && c >= pp.slot_min_targets) {
        const int base = c >= pp.lane_min_targets ? 0 : pp.nlane;
        for (int b = 0; b < pp.nlane; ++b)
            if (pp.lane_words[b] >= W) return base + b;
    }
    for (int b = 0; b < pp.nwarp; ++b)
        if (32 * pp.warp_words[b] >= W) return 2 * pp.nlane + b;
    return -1;
}

// A sequence index is usable when it is in range and its offsets lie inside
// the arena in order (so no kernel can read outside the arena).
__device__ __forceinline__ bool seq_ok(const int64_t *__restrict__ offs, int32_t n, int64_t total, int s) {
    if (s < 0 || s >= n) return false;
    const int64_t a = offs[s], b = offs[s + 1];
    return a >= 0 && a <= b && b <= total;
}

// Pair list: all of pairs[0..P) or, with idx, pairs[idx[0 .. *count)).
struct PairList {
    const int32_t *pairs;
    int64_t P;
    const int32_t *idx;
    const int32_t *count;
    __device__ __forceinline__ int64_t size() const { return idx ? (int64_t)*count : P; }
    __device__ __forceinline__ int64_t id(int64_t k) const { return idx ? (int64_t)idx[k] : k; }
};

__global__ void count_kernel(PairList L, int32_t n, const int64_t *__restrict__ offs, int64_t total,
                             int32_t *__restrict__ qcount, int32_t *err) {
    const int64_t P = L.size();
    // warp-uniform loop (the warp's lanes take consecutive pairs) so that the
    // counts can be aggregated per warp
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); k0 < P; k0 += stride) {
        const int64_t k = k0 + (threadIdx.x & 31);
        bool act = k < P;
        int q = 0;
        if (act) {
            const int64_t p = L.id(k);
            q = L.pairs[2 * p];
            const int t = L.pairs[2 * p + 1];
            if (!seq_ok(offs, n, total, q) || !seq_ok(offs, n, total, t)) {
                record_error(err, kErrIndex, p, seq_ok(offs, n, total, q) ? t : q);
                act = false;
            }
        }
        warp_agg_inc(qcount, q, act);
    }
}

// Exclusive scan of n ints in tiles of 4,096 (1,024 threads x 4 consecutive
// values): one kernel sums each tile, a second scans each tile from the sum
// of the tiles before it.  Loads and stores are coalesced and every tile has
// its own block, so a scan over hundreds of thousands of queries takes a few
// microseconds (one block walking the whole array took ~0.2 ms at 200,000).
constexpr int kScanTile = 4096;

template <class T>
__device__ __forceinline__ T block_sum_1024(T v, T *wsum) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
    __syncthreads();
    T t = threadIdx.x < 32 ? wsum[threadIdx.x] : T(0);
    if (threadIdx.x < 32) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    if (threadIdx.x == 0) wsum[0] = t;
    __syncthreads();
    t = wsum[0];
    __syncthreads();
    return t;
}

template <class T>
__global__ void __launch_bounds__(1024) tile_sum_kernel(const T *__restrict__ in, int32_t n, T *__restrict__ tsum) {
    __shared__ T wsum[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    T v = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t i = base + r * 1024 + threadIdx.x;
        if (i < n) v += in[i];
    }
    v = block_sum_1024(v, wsum);
    if (threadIdx.x == 0) tsum[blockIdx.x] = v;
}

template <class T>
__global__ void __launch_bounds__(1024) tile_scan_kernel(const T *__restrict__ in, int32_t n, const T *__restrict__ tsum,
                                                         T *__restrict__ out) {
    __shared__ T wsum[32];
    __shared__ T wpre[32];
    // the sum of the tiles before this one
    T pre = 0;
    for (int t = threadIdx.x; t < (int)blockIdx.x; t += 1024) pre += tsum[t];
    pre = block_sum_1024(pre, wsum);
    const int64_t base = (int64_t)blockIdx.x * kScanTile + 4 * (int64_t)threadIdx.x;
    T x[4];
    T own = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        x[r] = base + r < n ? in[base + r] : 0;
        own += x[r];
    }
    // exclusive scan of the per-thread sums across the block
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wpre[w] = inc;
    __syncthreads();
    if (w == 0) {
        T t = wpre[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wpre[lane] = t;
    }
    __syncthreads();
    T run = pre + (w ? wpre[w - 1] : T(0)) + inc - own;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        if (base + r < n) out[base + r] = run;
        run += x[r];
    }
    // the total, once, by the thread that holds the last value
    if (base < n && base + 4 >= n) out[n] = run;
    if (n == 0 && blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
}

int64_t scan_tiles(int64_t n) { return std::max<int64_t>(1, (n + kScanTile - 1) / kScanTile); }

// out[0..n] = exclusive prefix sums of in[0..n) and the total; tsum holds
// scan_tiles(n) ints of scratch.
void exclusive_scan(const int32_t *in, int32_t n, int32_t *out, int32_t *tsum, cudaStream_t st) {
    const int tiles = (int)scan_tiles(n);
    tile_sum_kernel<int32_t><<<tiles, 1024, 0, st>>>(in, n, tsum);
    tile_scan_kernel<int32_t><<<tiles, 1024, 0, st>>>(in, n, tsum, out);
}

void exclusive_scan64(const int64_t *in, int32_t n, int64_t *out, int64_t *tsum, cudaStream_t st) {
    const int tiles = (int)scan_tiles(n);
    tile_sum_kernel<int64_t><<<tiles, 1024, 0, st>>>(in, n, tsum);
    tile_scan_kernel<int64_t><<<tiles, 1024, 0, st>>>(in, n, tsum, out);
}

__global__ void scatter_kernel(PairList L, int32_t n, const int64_t *__restrict__ offs, int64_t total,
                               const int32_t *__restrict__ qstart, int32_t *__restrict__ qfill,
                               int32_t *__restrict__ sorted_t, int32_t *__restrict__ sorted_p) {
    const int64_t P = L.size();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); k0 < P; k0 += stride) {
        const int64_t k = k0 + (threadIdx.x & 31);
        bool act = k < P;
        int64_t p = 0;
        int q = 0, t = 0;
        if (act) {
            p = L.id(k);
            q = L.pairs[2 * p];
            t = L.pairs[2 * p + 1];
            act = seq_ok(offs, n, total, q) && seq_ok(offs, n, total, t);
        }
        const int r = warp_agg_inc(qfill, q, act);
        if (act) {
            const int pos = qstart[q] + r;
            sorted_t[pos] = t;
            sorted_p[pos] = (int32_t)p;
        }
    }
}

// Orders the targets of every query that has at least `min_count` of them
// by length, longest first: a counting sort on 32-column length classes,
// one block per query, through tmp_t / tmp_p.  The lanes of a warp then take
// targets of about the same length one after another, so they switch
// targets together and the two-column step holds for more of the work, and
// a query's last targets are its shortest ones.
constexpr int kLenClasses = 256;

__global__ void __launch_bounds__(kLenClasses) length_order_kernel(
    const int64_t *__restrict__ offs, int32_t n, const int32_t *__restrict__ qstart, int32_t min_count,
    int32_t *__restrict__ sorted_t, int32_t *__restrict__ sorted_p, int32_t *__restrict__ tmp_t,
    int32_t *__restrict__ tmp_p) {
    __shared__ int32_t cur[kLenClasses];
    __shared__ int32_t wsum[kLenClasses / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = blockIdx.x; q < n; q += gridDim.x) {
        const int b = qstart[q], e = qstart[q + 1];
        if (e - b < min_count) continue;
        cur[threadIdx.x] = 0;
        __syncthreads();
        for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
            const int t = sorted_t[i];
            const int cls = (int)min((offs[t + 1] - offs[t]) >> 5, (int64_t)(kLenClasses - 1));
            atomicAdd(&cur[kLenClasses - 1 - cls], 1);
        }
        __syncthreads();
        const int v = cur[threadIdx.x];
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        int before = 0;
        for (int w = 0; w < wid; ++w) before += wsum[w];
        cur[threadIdx.x] = b + before + incl - v;
        __syncthreads();
        for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
            const int t = sorted_t[i];
            const int cls = (int)min((offs[t + 1] - offs[t]) >> 5, (int64_t)(kLenClasses - 1));
            const int pos = atomicAdd(&cur[kLenClasses - 1 - cls], 1);
            tmp_t[pos] = t;
            tmp_p[pos] = sorted_p[i];
        }
        __syncthreads();
        for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
            sorted_t[i] = tmp_t[i];
            sorted_p[i] = tmp_p[i];
        }
        __syncthreads();
    }
}

// pass 0: count tasks per bucket; pass 1: write them (bucket offsets by a
// scan over <= kMaxBuckets counts done redundantly by every block).
template <int PASS>
__global__ void __launch_bounds__(256) task_kernel(const int64_t *__restrict__ offs, int32_t n,
                                                   const int32_t *__restrict__ qstart, PlanParams pp,
                                                   int32_t *__restrict__ bcount, int32_t *__restrict__ bfill,
                                                   int32_t *__restrict__ boff, int2 *__restrict__ tasks,
                                                   int32_t *__restrict__ bsum, int32_t *err) {
    __shared__ int32_t sboff[kMaxBuckets];
    const int NB = 2 * pp.nlane + pp.nwarp;
    if (PASS == 1) {
        if (threadIdx.x == 0) {
            int run = 0;
            for (int b = 0; b < NB; ++b) {
                sboff[b] = run;
                run += bcount[b];
            }
        }
        __syncthreads();
        if (blockIdx.x == 0 && threadIdx.x < NB) boff[threadIdx.x] = sboff[threadIdx.x];
    }
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int c = qstart[q + 1] - qstart[q];
        if (c == 0) continue;
        const int m = (int)(offs[q + 1] - offs[q]);
        const int W = max(1, (m + 31) / 32);
        const int b = pick_bucket(pp, W, c);
        if (b < 0) {
            if (PASS == 0) record_error(err, kErrLength, q, m);
            continue;
        }
        // a slot-kernel query is one entry; the others split into tasks
        const int per = b < pp.nlane ? pp.lane_per_task : b < 2 * pp.nlane ? c : pp.warp_per_task;
        const int parts = (c + per - 1) / per;
        if (PASS == 0) {
            atomicAdd(bcount + b, parts);
            if (b >= pp.nlane && b < 2 * pp.nlane) atomicAdd(bsum + b, c);
        } else {
            const int base = sboff[b] + atomicAdd(bfill + b, parts);
            for (int i = 0; i < parts; ++i) tasks[base + i] = make_int2((int)q, i);
        }
    }
}

static int grid_for(int blocks) { return blocks < 1 ? 1 : blocks; }

// pairs (query, idx[i]) of a one-to-many batch
__global__ void __launch_bounds__(256) one_to_many_pairs_kernel(int32_t query, const int32_t *__restrict__ idx,
                                                                int64_t n, int32_t *__restrict__ pairs) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        pairs[2 * i] = query;
        pairs[2 * i + 1] = idx[i];
    }
}

int64_t lev_workspace(int64_t P, int32_t n) {
    auto r = [](int64_t b) { return (b + 255) & ~int64_t(255); };
    return r(4 * int64_t(n)) * 3 + r(4 * (int64_t(n) + 1)) + r(4 * P) * 4 + r(8 * (P + n + 1)) +
           r(4 * kMaxBuckets) * 5 + r(4 * scan_tiles(n));
}

static PlanParams plan_params(const Registry &R, const Tune &T, int64_t P, int sm_count) {
    PlanParams pp{};
    pp.nlane = R.nlane;
    pp.nwarp = R.nwarp;
    for (int b = 0; b < R.nlane; ++b) pp.lane_words[b] = R.lane[b].words;
    for (int b = 0; b < R.nwarp; ++b) pp.warp_words[b] = R.warp[b].words;
    pp.lane_min_targets = T.lane_min_targets;
    pp.slot_min_targets = std::min(T.slot_min_targets, T.lane_min_targets);
    if (T.lane_per_task > 0) {
        pp.lane_per_task = T.lane_per_task;
    } else {
        // about four tasks per resident warp (16 per SM), 32..512 targets each
        int64_t per = P / ((int64_t)sm_count * 16 * 4);
        per = std::max<int64_t>(32, std::min<int64_t>(512, per));
        pp.lane_per_task = (int)(per / 32 * 32);
    }
    pp.warp_per_task = T.warp_per_task;
    return pp;
}

static msa_status ensure_occupancy(msa_ctx *ctx, const Registry &R, int alphabet) {
    Tune &T = *ctx->tune;
    for (int b = 0; b < R.count(); ++b) {
        if (T.occupancy[alphabet][b] > 0) continue;
        const LevKernelInfo &K = R.at(b);
        const size_t smem = K.smem_per_warp * 4;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(K.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return cuda_check(ctx, e, "cudaFuncSetAttribute");
        }
        int blocks = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, K.fn, 128, smem);
        if (e != cudaSuccess) return cuda_check(ctx, e, "occupancy query");
        T.occupancy[alphabet][b] = blocks > 0 ? blocks : 1;
    }
    return MSA_OK;
}

}  // namespace msa

namespace msa {

// Launches the whole schedule.  `max_len` (host) bounds the buckets launched.
// With idx != nullptr the batch is pairs[idx[0 .. *count_dev)), at most P of
// them; the workspace is taken from `ar` (the whole context workspace if null).
msa_status lev_run(msa_ctx *ctx, const msa_seqset *s, const int32_t *pairs, int64_t P, int32_t *d_out,
                   cudaStream_t st, const int32_t *idx, const int32_t *count_dev, Arena *outer, int side_base) {
    const Registry R = registry(s->alphabet);
    msa_status rc = ensure_occupancy(ctx, R, s->alphabet);
    if (rc) return rc;
    const Tune &T = *ctx->tune;
    const int32_t n = s->n_seqs;
    Arena own{ctx->ws, ctx->ws_bytes};
    Arena &ar = outer ? *outer : own;
    int32_t *qcount = ar.take<int32_t>(n);
    int32_t *qfill = ar.take<int32_t>(n);
    int32_t *qcursor = ar.take<int32_t>(n);
    int32_t *qstart = ar.take<int32_t>(int64_t(n) + 1);
    int32_t *sorted_t = ar.take<int32_t>(P);
    int32_t *sorted_p = ar.take<int32_t>(P);
    int32_t *tmp_t = ar.take<int32_t>(P);
    int32_t *tmp_p = ar.take<int32_t>(P);
    int2 *tasks = ar.take<int2>(P + n + 1);
    int32_t *bcount = ar.take<int32_t>(kMaxBuckets);
    int32_t *bfill = ar.take<int32_t>(kMaxBuckets);
    int32_t *boff = ar.take<int32_t>(kMaxBuckets);
    int32_t *bcounter = ar.take<int32_t>(kMaxBuckets);
    int32_t *bsum = ar.take<int32_t>(kMaxBuckets);
    int32_t *tsum = ar.take<int32_t>(scan_tiles(n));
    if (!tsum)
        return set_error(ctx, MSA_ENOMEM, "msa_lev_batch: needs %lld workspace bytes, context has %lld",
                         (long long)lev_workspace(P, n), (long long)ctx->ws_bytes);
    // the three per-query arrays are contiguous: one memset
    cudaError_t e = cudaMemsetAsync(qcount, 0, (char *)qstart - (char *)qcount, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bcount, 0, (char *)bsum - (char *)bcount + 4 * kMaxBuckets, st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "msa_lev_batch memset");

    const int gP = grid_for((int)std::min<int64_t>((P + 255) / 256, ctx->sm_count * 8));
    const int gN = grid_for((int)std::min<int64_t>((n + 255) / 256, ctx->sm_count * 8));
    ctx->launches += 6;
    const PairList L{pairs, P, idx, count_dev};
    count_kernel<<<gP, 256, 0, st>>>(L, n, s->offs, s->total, qcount, ctx->dev_err);
    exclusive_scan(qcount, n, qstart, tsum, st);
    scatter_kernel<<<gP, 256, 0, st>>>(L, n, s->offs, s->total, qstart, qfill, sorted_t, sorted_p);
    const PlanParams pp = plan_params(R, T, P, ctx->sm_count);
    length_order_kernel<<<grid_for((int)std::min<int64_t>(n, ctx->sm_count * 8)), kLenClasses, 0, st>>>(
        s->offs, n, qstart, std::max(pp.lane_min_targets, 2), sorted_t, sorted_p, tmp_t, tmp_p);
    ++ctx->launches;
    task_kernel<0><<<gN, 256, 0, st>>>(s->offs, n, qstart, pp, bcount, bfill, boff, tasks, bsum, ctx->dev_err);
    task_kernel<1><<<gN, 256, 0, st>>>(s->offs, n, qstart, pp, bcount, bfill, boff, tasks, bsum, ctx->dev_err);

    LevArgs a{};
    a.planes = s->planes;
    a.codes = s->codes;
    a.offs = s->offs;
    a.sorted_t = sorted_t;
    a.sorted_p = sorted_p;
    a.qstart = qstart;
    a.qcursor = qcursor;
    a.tasks = tasks;
    a.boff = boff;
    a.bcount = bcount;
    a.bcounter = bcounter;
    a.bsum = bsum;
    a.d_out = d_out;
    a.err = ctx->dev_err;
    // buckets that no sequence of this set can reach are not launched
    const int Wmax = std::max(1, (s->max_len + 31) / 32);
    int lane_last = R.nlane - 1;
    for (int b = 0; b < R.nlane; ++b)
        if (R.lane[b].words >= Wmax) {
            lane_last = b;
            break;
        }
    int warp_last = R.nwarp - 1;
    for (int b = 0; b < R.nwarp; ++b)
        if (32 * R.warp[b].words >= Wmax) {
            warp_last = b;
            break;
        }
    // the buckets are independent: run them side by side so that small or
    // uneven buckets do not leave the GPU idle one after another (on 16 side
    // streams for a call of its own; nested in a banded call, on the streams
    // its band kernels leave free)
    std::vector<int> launch_list;
    for (int b = 0; b < R.count(); ++b) {
        if (b < 2 * R.nlane ? b % R.nlane > lane_last : b - 2 * R.nlane > warp_last) continue;
        if (b >= R.nlane && b < 2 * R.nlane && pp.slot_min_targets >= pp.lane_min_targets) continue;
        launch_list.push_back(b);
    }
    ProfScope prof(ctx, st);
    e = run_concurrent(ctx, st, (int)launch_list.size(), [&](int i, cudaStream_t s2) {
        LevArgs ai = a;
        ai.bucket = launch_list[i];
        const int grid = grid_for(ctx->sm_count * T.occupancy[s->alphabet][ai.bucket]);
        R.at(ai.bucket).launch(ai, grid, s2);
    }, side_base, side_base == 0 ? 16 : msa_ctx::kSide - side_base);
    ctx->launches += (int64_t)launch_list.size();
    if (e != cudaSuccess) return cuda_check(ctx, e, "msa_lev_batch launch");
    return cuda_check(ctx, cudaGetLastError(), "msa_lev_batch launch");
}

msa_status lev_validate(msa_ctx *ctx, const msa_seqset *s, const int32_t *pairs, int64_t P,
                               const void *out, const char *who) {
    if (!ctx || !s) return MSA_EINVAL;
    if (P < 0 || P >= (int64_t(1) << 31)) return set_error(ctx, MSA_EINVAL, "%s: P=%lld out of range", who, (long long)P);
    if (s->alphabet != MSA_DNA && s->alphabet != MSA_PROTEIN)
        return set_error(ctx, MSA_EINVAL, "%s: unknown alphabet %d", who, s->alphabet);
    if (P > 0 && (!pairs || !out || !s->offs || !s->codes || !s->planes))
        return set_error(ctx, MSA_EINVAL, "%s: null pointer", who);
    if (s->n_seqs < 0 || s->max_len < 0) return set_error(ctx, MSA_EINVAL, "%s: negative size", who);
    if (s->max_len > 32 * 32 * 16)
        return set_error(ctx, MSA_EUNSUPPORTED, "%s: max_len %d above the 16384 the kernels support", who, s->max_len);
    return MSA_OK;
}

}  // namespace msa

using namespace msa;

extern "C" {

int64_t msa_lev_workspace_bytes(int64_t P, int32_t n_seqs) { return lev_workspace(P, n_seqs); }

msa_status msa_lev_batch(msa_ctx *ctx, const msa_seqset *s, const int32_t *pairs, int64_t P, int32_t *d_out,
                         void *stream) {
    msa_status rc = lev_validate(ctx, s, pairs, P, d_out, "msa_lev_batch");
    if (rc || P == 0) return rc;
    if (s->n_seqs == 0) return set_error(ctx, MSA_EINVAL, "msa_lev_batch: pairs given for an empty set");
    return lev_run(ctx, s, pairs, P, d_out, (cudaStream_t)stream, nullptr, nullptr, nullptr);
}

int64_t msa_lev_one_to_many_workspace_bytes(int64_t n, int32_t n_seqs) {
    return ((8 * n + 255) & ~int64_t(255)) + lev_workspace(n, n_seqs);
}

msa_status msa_lev_one_to_many(msa_ctx *ctx, const msa_seqset *s, int32_t query, const int32_t *idx, int64_t n,
                               int32_t *d_out, void *stream) {
    msa_status rc = lev_validate(ctx, s, idx, n, d_out, "msa_lev_one_to_many");
    if (rc || n == 0) return rc;
    if (query < 0 || query >= s->n_seqs)
        return set_error(ctx, MSA_EINVAL, "msa_lev_one_to_many: query %d outside [0, %d)", query, s->n_seqs);
    const cudaStream_t st = (cudaStream_t)stream;
    Arena ar{ctx->ws, ctx->ws_bytes};
    int32_t *pairs = ar.take<int32_t>(2 * n);
    if (!pairs || ar.cap - ar.used < lev_workspace(n, s->n_seqs))
        return set_error(ctx, MSA_ENOMEM, "msa_lev_one_to_many: needs %lld workspace bytes, context has %lld",
                         (long long)msa_lev_one_to_many_workspace_bytes(n, s->n_seqs), (long long)ctx->ws_bytes);
    const int g = grid_for((int)std::min<int64_t>((n + 255) / 256, ctx->sm_count * 8));
    one_to_many_pairs_kernel<<<g, 256, 0, st>>>(query, idx, n, pairs);
    ++ctx->launches;
    return lev_run(ctx, s, pairs, n, d_out, st, nullptr, nullptr, &ar);
}

msa_status msa_lev_tune_get(msa_ctx *ctx, int32_t *tune4) {
    if (!ctx || !tune4) return MSA_EINVAL;
    const Tune &T = *ctx->tune;
    tune4[0] = T.lane_min_targets;
    tune4[1] = T.slot_min_targets;
    tune4[2] = T.lane_per_task;
    tune4[3] = T.warp_per_task;
    return MSA_OK;
}

msa_status msa_lev_tune_set(msa_ctx *ctx, const int32_t *tune4) {
    if (!ctx || !tune4) return MSA_EINVAL;
    if (tune4[0] == 0 || tune4[1] == 0 || tune4[3] == 0)
        return set_error(ctx, MSA_EINVAL, "msa_lev_tune_set: zero target threshold or task size");
    Tune &T = *ctx->tune;
    if (tune4[0] > 0) T.lane_min_targets = tune4[0];
    if (tune4[1] > 0) T.slot_min_targets = tune4[1];
    if (tune4[2] >= 0) T.lane_per_task = tune4[2];
    if (tune4[3] > 0) T.warp_per_task = tune4[3];
    return MSA_OK;
}

msa_status msa_lev_autotune(msa_ctx *ctx, const msa_seqset *s, const int32_t *pairs, int64_t P, int32_t *d_out,
                            void *stream) {
    msa_status rc = lev_validate(ctx, s, pairs, P, d_out, "msa_lev_autotune");
    if (rc || P == 0) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *scratch = d_out;
    Tune &T = *ctx->tune;
    const Tune keep = T;
    struct Cand {
        int lane_min, slot_min, lane_per, warp_per;
    };
    // {1 << 30, 1 << 30, ...}: warp kernel only; slot_min >= lane_min: no slot kernel
    // lane_per = 32: one target per lane per task (fastest on long DNA all-pairs
    // batches, slower on short protein ones)
    const Cand cands[] = {{32, 2, 0, 4},   {16, 2, 0, 4},   {64, 2, 0, 4},   {32, 3, 0, 4},
                          {12, 12, 0, 4},  {4, 4, 0, 4},    {32, 2, 32, 4},  {32, 2, 64, 4},
                          {32, 2, 128, 4}, {32, 2, 256, 4}, {32, 2, 512, 4}, {32, 2, 0, 1},
                          {32, 2, 0, 16},  {1 << 30, 1 << 30, 0, 4}};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    Cand pick = {keep.lane_min_targets, keep.slot_min_targets, keep.lane_per_task, keep.warp_per_task};
    for (const Cand &c : cands) {
        T.lane_min_targets = c.lane_min;
        T.slot_min_targets = c.slot_min;
        T.lane_per_task = c.lane_per;
        T.warp_per_task = c.warp_per;
        float ms_best = 1e30f;
        for (int rep = 0; rep < 3 && rc == MSA_OK; ++rep) {
            cudaEventRecord(e0, st);
            rc = lev_run(ctx, s, pairs, P, scratch, st, nullptr, nullptr, nullptr);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) ms_best = std::min(ms_best, ms);
        }
        if (rc) break;
        if (ms_best < best) {
            best = ms_best;
            pick = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    T.lane_min_targets = pick.lane_min;
    T.slot_min_targets = pick.slot_min;
    T.lane_per_task = pick.lane_per;
    T.warp_per_task = pick.warp_per;
    if (rc) return rc;
    return msa_ctx_check(ctx, stream);
}

}  // extern "C"
