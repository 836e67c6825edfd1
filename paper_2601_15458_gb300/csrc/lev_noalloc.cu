// msa_lev_batch_noalloc: the batched Levenshtein distance for callers that
// cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc or create a context
// workspace: code that runs inside another framework's memory budget (a
// caching allocator that owns all free device memory), plug-ins loaded into
// a host that forbids allocations after start-up, or latency-critical loops
// where an allocation's implicit synchronisation is not acceptable.  This
// entry point gives them the same distances as msa_lev_batch without any
// allocation: its scratch lives in one file-scope __device__ array of a fixed
// maximum size, which every GPU that loads the library holds until the
// process exits.
//
// Properties (also stated in include/msa.h):
//  * At most kMaxPairs pairs over at most kMaxSeqs sequences per call;
//    larger calls are rejected with MSA_EINVAL before anything runs.
//  * All calls share the one scratch array per device: calls whose work
//    overlaps on the GPU (other streams, other host threads) race.  Serialise
//    them on one stream.
//  * The first call on a device looks the array's address up
//    (cudaGetSymbolAddress) with that device current, sets the kernels'
//    shared-memory limits and queries their occupancy; make that first call
//    before any stream capture.  The set-up is kept per CUDA context: after
//    the device's context is destroyed and recreated (cudaDeviceReset), the
//    next call on it does the set-up again, so that first call should also
//    come before any capture.
//  * No context, so no error word: pairs with an index outside the set, or
//    whose first sequence is longer than s->max_len, get d_out = -1.
//    max_len < 0 is rejected with MSA_EINVAL, max_len above the 16,384 the
//    kernels hold with MSA_EUNSUPPORTED.
//  * It calls no cudaMalloc, cudaFree or allocating library routine.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "lev_kernels.cuh"
#include "warp_agg.cuh"

namespace msa {
namespace noalloc {

constexpr int64_t kMaxPairs = int64_t(1) << 18;   // 262,144 pairs per call
constexpr int32_t kMaxSeqs = int32_t(1) << 16;    // 65,536 sequences in the set
constexpr int kNB = 64;                           // kernel buckets (>= 2 x lane + warp configurations)
constexpr int kMaxDevices = 64;
constexpr int32_t kMaxQueryLen = 32 * 32 * 16;     // the longest sequence the kernels hold (16,384)

struct Scratch {
    int32_t qcount[kMaxSeqs];
    int32_t qfill[kMaxSeqs];
    int32_t qcursor[kMaxSeqs];
    int32_t qstart[kMaxSeqs + 1];
    int32_t sorted_t[kMaxPairs];
    int32_t sorted_p[kMaxPairs];
    int2 tasks[kMaxPairs + kMaxSeqs + 1];
    int32_t bcount[kNB];
    int32_t bfill[kNB];
    int32_t boff[kNB];
    int32_t bcounter[kNB];
    int32_t bsum[kNB];
    int32_t err[4];
};

// The scratch of every call (about 5.8 MB per device).
static __device__ __align__(256) Scratch g_scratch;

struct Plan {
    int nlane, nwarp;
    int lane_words[32];
    int warp_words[32];
    int lane_per_task;
};

__device__ __forceinline__ bool ok_seq(const int64_t *offs, int32_t n, int64_t total, int s) {
    if (s < 0 || s >= n) return false;
    const int64_t a = offs[s], b = offs[s + 1];
    return a >= 0 && a <= b && b <= total;
}

__global__ void na_count(Scratch *S, const int32_t *__restrict__ pairs, int64_t P, int32_t n,
                         const int64_t *__restrict__ offs, int64_t total) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); p0 < P; p0 += stride) {
        const int64_t p = p0 + (threadIdx.x & 31);
        int q = 0;
        bool act = p < P;
        if (act) {
            q = pairs[2 * p];
            act = ok_seq(offs, n, total, q) && ok_seq(offs, n, total, pairs[2 * p + 1]);
        }
        warp_agg_inc(S->qcount, q, act);
    }
}

__global__ void __launch_bounds__(1024) na_scan(Scratch *S, int32_t n) {
    __shared__ int32_t part[1024];
    const int tid = threadIdx.x;
    const int64_t chunk = (n + 1023) / 1024;
    const int64_t lo = tid * chunk, hi = min((int64_t)n, lo + chunk);
    int32_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += S->qcount[i];
    part[tid] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int32_t v = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int32_t run = tid ? part[tid - 1] : 0;
    for (int64_t i = lo; i < hi; ++i) {
        S->qstart[i] = run;
        run += S->qcount[i];
    }
    if (tid == 1023) S->qstart[n] = part[1023];
}

__global__ void na_scatter(Scratch *S, const int32_t *__restrict__ pairs, int64_t P, int32_t n,
                           const int64_t *__restrict__ offs, int64_t total) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); p0 < P; p0 += stride) {
        const int64_t p = p0 + (threadIdx.x & 31);
        int q = 0, t = 0;
        bool act = p < P;
        if (act) {
            q = pairs[2 * p];
            t = pairs[2 * p + 1];
            act = ok_seq(offs, n, total, q) && ok_seq(offs, n, total, t);
        }
        const int r = warp_agg_inc(S->qfill, q, act);
        if (act) {
            const int pos = S->qstart[q] + r;
            S->sorted_t[pos] = t;
            S->sorted_p[pos] = (int32_t)p;
        }
    }
}

// buckets [lane | slot | warp], the default schedule of msa_lev_batch: a warp
// per query from 32 targets, shared warps (slot kernel) from 2, the
// warp-per-pair kernel for single targets and long queries
__device__ __forceinline__ int na_bucket(const Plan &pl, int W, int c) {
    if (W <= pl.lane_words[pl.nlane - 1] && c >= 2) {
        const int base = c >= 32 ? 0 : pl.nlane;
        for (int b = 0; b < pl.nlane; ++b)
            if (pl.lane_words[b] >= W) return base + b;
    }
    for (int b = 0; b < pl.nwarp; ++b)
        if (32 * pl.warp_words[b] >= W) return 2 * pl.nlane + b;
    return -1;
}

template <int PASS>
__global__ void __launch_bounds__(256) na_tasks(Scratch *S, const int64_t *__restrict__ offs, int32_t n, Plan pl) {
    __shared__ int32_t sboff[kNB];
    const int NB = 2 * pl.nlane + pl.nwarp;
    if (PASS == 1) {
        if (threadIdx.x == 0) {
            int run = 0;
            for (int b = 0; b < NB; ++b) {
                sboff[b] = run;
                run += S->bcount[b];
            }
        }
        __syncthreads();
        if (blockIdx.x == 0 && threadIdx.x < NB) S->boff[threadIdx.x] = sboff[threadIdx.x];
    }
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int c = S->qstart[q + 1] - S->qstart[q];
        if (c == 0) continue;
        const int m = (int)(offs[q + 1] - offs[q]);
        const int b = na_bucket(pl, max(1, (m + 31) / 32), c);
        if (b < 0) continue;   // too long for the kernels: its pairs keep d_out = -1
        const int per = b < pl.nlane ? pl.lane_per_task : b < 2 * pl.nlane ? c : 4;
        const int parts = (c + per - 1) / per;
        if (PASS == 0) {
            atomicAdd(&S->bcount[b], parts);
            if (b >= pl.nlane && b < 2 * pl.nlane) atomicAdd(&S->bsum[b], c);
        } else {
            const int base = sboff[b] + atomicAdd(&S->bfill[b], parts);
            for (int i = 0; i < parts; ++i) S->tasks[base + i] = make_int2((int)q, i);
        }
    }
}

// Kernel of bucket b: lane kernels, then the same word counts with 8 query
// slots, then the warp-per-pair kernels.
static const LevKernelInfo &kernel_at(int alphabet, int b) {
    const bool dna = alphabet == MSA_DNA;
    const int nl = dna ? kLevLaneDnaCount : kLevLaneProtCount;
    if (b < nl) return (dna ? kLevLaneDna : kLevLaneProt)[b];
    if (b < 2 * nl) return (dna ? kLevSlotDna : kLevSlotProt)[b - nl];
    return (dna ? kLevWarpDna : kLevWarpProt)[b - 2 * nl];
}

// Per-device set-up: the scratch address, SM count and kernel occupancies,
// kept for the CUDA context they were taken in.  A context that is torn down
// and created again (cudaDeviceReset) reloads the module, so the array may
// move and the kernels' shared-memory attributes are gone: a call that finds
// a different context on its device than the one recorded redoes the set-up.
struct DeviceInfo {
    unsigned long long ctx_id = 0;   // 0: no set-up yet
    Scratch *scratch = nullptr;
    int sm_count = 0;
    int occ[2][kNB] = {};
};

static DeviceInfo g_dev[kMaxDevices];
static std::mutex g_mu;

// The driver's current-context calls, reached through the runtime (no link
// against the driver library).
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);
static CtxGetCurrentFn g_ctx_current = nullptr;
static CtxGetIdFn g_ctx_id = nullptr;

// Id of the context current on this thread, 0 when there is none.
static unsigned long long current_ctx_id() {
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&c) != CUDA_SUCCESS || !c) return 0;
    if (g_ctx_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Returns a copy of the set-up of device `dev` for `alphabet`, doing it
// first where needed (the first call on a device, and the first after its
// context was recreated).  Called with `dev` current.
static msa_status setup(int dev, int alphabet, DeviceInfo *out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ctx_current) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return MSA_ECUDA;
        g_ctx_id = reinterpret_cast<CtxGetIdFn>(f2);
        g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    }
    DeviceInfo &d = g_dev[dev];
    unsigned long long id = current_ctx_id();
    if (id == 0 || id != d.ctx_id) {
        // the address of the array in this context (this also makes the
        // device's primary context current when no context is yet)
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) return MSA_ECUDA;
        DeviceInfo fresh;
        if (cudaDeviceGetAttribute(&fresh.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return MSA_ECUDA;
        fresh.scratch = static_cast<Scratch *>(ptr);
        fresh.ctx_id = current_ctx_id();
        if (fresh.ctx_id == 0) return MSA_ECUDA;
        d = fresh;
    }
    const int nl = alphabet == MSA_DNA ? kLevLaneDnaCount : kLevLaneProtCount;
    const int nw = alphabet == MSA_DNA ? kLevWarpDnaCount : kLevWarpProtCount;
    if (2 * nl + nw > kNB) return MSA_EUNSUPPORTED;
    for (int b = 0; b < 2 * nl + nw; ++b) {
        if (d.occ[alphabet][b] > 0) continue;
        const LevKernelInfo &K = kernel_at(alphabet, b);
        const size_t smem = K.smem_per_warp * 4;
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(K.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return MSA_ECUDA;
        int blocks = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, K.fn, 128, smem) != cudaSuccess) return MSA_ECUDA;
        d.occ[alphabet][b] = std::max(blocks, 1);
    }
    *out = d;
    return MSA_OK;
}

}  // namespace noalloc
}  // namespace msa

using namespace msa;
using namespace msa::noalloc;

extern "C" msa_status msa_lev_batch_noalloc(const msa_seqset *s, const int32_t *pairs, int64_t P, int32_t *d_out,
                                            void *stream) {
    if (!s || P < 0) return MSA_EINVAL;
    if (P == 0) return MSA_OK;
    if (P > kMaxPairs || s->n_seqs > kMaxSeqs || s->n_seqs <= 0) return MSA_EINVAL;
    if (!pairs || !d_out || !s->offs || !s->codes || !s->planes) return MSA_EINVAL;
    if (s->alphabet != MSA_DNA && s->alphabet != MSA_PROTEIN) return MSA_EINVAL;
    if (s->max_len < 0) return MSA_EINVAL;
    if (s->max_len > kMaxQueryLen) return MSA_EUNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MSA_ECUDA;
    DeviceInfo info;
    msa_status rc = setup(dev, s->alphabet, &info);
    if (rc) return rc;
    const DeviceInfo *D = &info;
    cudaStream_t st = (cudaStream_t)stream;
    Scratch *S = D->scratch;
    const int32_t n = s->n_seqs;
    // the scratch keeps the last call's contents: clear what must start at
    // zero (the per-query counters of this call's n sequences, the bucket
    // counters) and preset every distance to -1 (pairs no kernel takes)
    if (cudaMemsetAsync(S->qcount, 0, sizeof(int32_t) * n, st) != cudaSuccess ||
        cudaMemsetAsync(S->qfill, 0, sizeof(int32_t) * n, st) != cudaSuccess ||
        cudaMemsetAsync(S->qcursor, 0, sizeof(int32_t) * n, st) != cudaSuccess ||
        cudaMemsetAsync(S->bcount, 0, sizeof(int32_t) * 5 * kNB, st) != cudaSuccess ||
        cudaMemsetAsync(d_out, 0xff, sizeof(int32_t) * P, st) != cudaSuccess)
        return MSA_ECUDA;
    const int gP = (int)std::max<int64_t>(1, std::min<int64_t>((P + 255) / 256, D->sm_count * 8));
    const int gN = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, D->sm_count * 8));
    na_count<<<gP, 256, 0, st>>>(S, pairs, P, n, s->offs, s->total);
    na_scan<<<1, 1024, 0, st>>>(S, n);
    na_scatter<<<gP, 256, 0, st>>>(S, pairs, P, n, s->offs, s->total);
    const LevKernelInfo *lane = s->alphabet == MSA_DNA ? kLevLaneDna : kLevLaneProt;
    const LevKernelInfo *warp = s->alphabet == MSA_DNA ? kLevWarpDna : kLevWarpProt;
    Plan pl{};
    pl.nlane = s->alphabet == MSA_DNA ? kLevLaneDnaCount : kLevLaneProtCount;
    pl.nwarp = s->alphabet == MSA_DNA ? kLevWarpDnaCount : kLevWarpProtCount;
    for (int b = 0; b < pl.nlane; ++b) pl.lane_words[b] = lane[b].words;
    for (int b = 0; b < pl.nwarp; ++b) pl.warp_words[b] = warp[b].words;
    int64_t per = P / ((int64_t)D->sm_count * 16 * 4);
    per = std::max<int64_t>(32, std::min<int64_t>(512, per));
    pl.lane_per_task = (int)(per / 32 * 32);
    na_tasks<0><<<gN, 256, 0, st>>>(S, s->offs, n, pl);
    na_tasks<1><<<gN, 256, 0, st>>>(S, s->offs, n, pl);
    LevArgs a{};
    a.planes = s->planes;
    a.codes = s->codes;
    a.offs = s->offs;
    a.sorted_t = S->sorted_t;
    a.sorted_p = S->sorted_p;
    a.qstart = S->qstart;
    a.qcursor = S->qcursor;
    a.tasks = S->tasks;
    a.boff = S->boff;
    a.bcount = S->bcount;
    a.bcounter = S->bcounter;
    a.bsum = S->bsum;
    a.d_out = d_out;
    a.err = S->err;
    const int Wmax = std::max(1, (s->max_len + 31) / 32);
    for (int b = 0; b < 2 * pl.nlane + pl.nwarp; ++b) {
        const bool is_warp = b >= 2 * pl.nlane;
        const int first = is_warp ? 2 * pl.nlane : (b < pl.nlane ? 0 : pl.nlane);
        const LevKernelInfo &K = kernel_at(s->alphabet, b);
        // a bucket whose smaller neighbour already holds the longest sequence is never used
        if (b > first) {
            const LevKernelInfo &prev = kernel_at(s->alphabet, b - 1);
            const int cap_prev = is_warp ? 32 * prev.words : prev.words;
            if (cap_prev >= Wmax) continue;
        }
        a.bucket = b;
        K.launch(a, D->sm_count * D->occ[s->alphabet][b], st);
    }
    return cudaGetLastError() == cudaSuccess ? MSA_OK : MSA_ECUDA;
}
