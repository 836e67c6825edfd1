// Integer-pipe throughput probe: the measured denominator of the
// bit-vector kernels' roofline.
//
// The Levenshtein word step is built from 3-input logic (LOP3), one add on
// the carry chain and one funnel shift; these all issue to the integer ALU
// pipe.  Each probe kernel runs one of those instructions (or the whole
// 9-op word step) as 8 independent dependency chains per thread, from
// registers only, with every SM filled to its occupancy limit, so that its
// rate is the pipe's sustained throughput rather than a latency or memory
// limit.  The inputs come from runtime values and every chain ends in a
// store, so nothing is folded away; each chain mixes several operands, so no
// two steps can merge into one instruction.  The caller times the launch
// (CUDA events on the same stream) and divides the lane-operation count the
// call reports by the elapsed time.
#include <cuda_runtime.h>

#include "lev_kernels.cuh"
#include "msa_internal.cuh"

namespace msa {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;      // independent chains per thread
constexpr int kProbeUnroll = 4;      // steps per chain per loop iteration

__device__ __forceinline__ uint32_t probe_lop3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    // majority(a, b, c): not linear, so a chain of them does not collapse
    asm volatile("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ uint32_t probe_shf(uint32_t lo, uint32_t hi) {
    uint32_t d;
    asm volatile("shf.l.wrap.b32 %0, %1, %2, 1;" : "=r"(d) : "r"(lo), "r"(hi));
    return d;
}

__device__ __forceinline__ uint32_t probe_imad(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// OP: 0 LOP3, 1 SHF (funnel shift by 1), 2 add with carry (8-word chains),
// 3 the Levenshtein word step (bv_column over 8 words, 9 ops per word),
// 4 IMAD (the multiply-add pipe, for comparison).
template <int OP>
__global__ void __launch_bounds__(kProbeThreads) int_probe_kernel(uint32_t *sink, int iters, uint32_t seed) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t a[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) a[r] = (seed + 0x9e3779b9u * (uint32_t)(r + 1)) ^ (tid * 0x85ebca6bu);
    uint32_t out = 0u;
    if constexpr (OP == 3) {
        // two independent columns' worth of state per thread (as the lane
        // kernel gets from its two-column steps), 8 words each
        uint32_t Pv[2][8], Mv[2][8];
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                Pv[s][w] = ~0u ^ (a[w & 3] >> s);
                Mv[s][w] = 0u;
            }
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int r = 0; r < kProbeUnroll; ++r) {
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    uint32_t eq[8], ph_out, cout;
#pragma unroll
                    for (int w = 0; w < 8; ++w) eq[w] = a[(w + r + s) & 3];
                    bv_column<8>(eq, Pv[s], Mv[s], 1u, 0u, ph_out, cout);
                    (void)ph_out;
                    (void)cout;
                }
            }
        }
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int w = 0; w < 8; ++w) out ^= Pv[s][w] + Mv[s][w];
    } else if constexpr (OP == 2) {
        uint32_t x[kProbeChains];
#pragma unroll
        for (int i = 0; i < kProbeChains; ++i) x[i] = a[i & 3] + (uint32_t)i;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int r = 0; r < kProbeUnroll; ++r) {
                asm volatile(
                    "add.cc.u32 %0, %0, %8;\n\taddc.cc.u32 %1, %1, %9;\n\taddc.cc.u32 %2, %2, %8;\n\t"
                    "addc.cc.u32 %3, %3, %9;\n\taddc.cc.u32 %4, %4, %8;\n\taddc.cc.u32 %5, %5, %9;\n\t"
                    "addc.cc.u32 %6, %6, %8;\n\taddc.u32 %7, %7, %9;"
                    : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(x[3]), "+r"(x[4]), "+r"(x[5]), "+r"(x[6]),
                      "+r"(x[7])
                    : "r"(a[r & 3]), "r"(a[(r + 1) & 3]));
            }
        }
#pragma unroll
        for (int i = 0; i < kProbeChains; ++i) out ^= x[i];
    } else {
        uint32_t x[kProbeChains];
#pragma unroll
        for (int i = 0; i < kProbeChains; ++i) x[i] = a[i & 3] ^ (uint32_t)i;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int r = 0; r < kProbeUnroll; ++r) {
#pragma unroll
                for (int i = 0; i < kProbeChains; ++i) {
                    if constexpr (OP == 0) x[i] = probe_lop3(x[i], a[(r + i) & 3], a[(r + i + 1) & 3]);
                    if constexpr (OP == 1) x[i] = probe_shf(a[(r + i) & 3], x[i]);
                    if constexpr (OP == 4) x[i] = probe_imad(x[i], a[(r + i) & 3] | 1u, a[(r + i + 1) & 3]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < kProbeChains; ++i) out ^= x[i];
    }
    sink[tid] = out;
}

// lane operations one thread executes per loop iteration
static int64_t probe_ops_per_iter(int op) {
    switch (op) {
        case 2: return (int64_t)kProbeUnroll * 8;                 // 8 adds per chain step
        case 3: return (int64_t)kProbeUnroll * 2 * 8 * 9;         // 2 columns x 8 words x 9 ops
        default: return (int64_t)kProbeUnroll * kProbeChains;
    }
}

static const void *probe_fn(int op) {
    switch (op) {
        case 0: return (const void *)int_probe_kernel<0>;
        case 1: return (const void *)int_probe_kernel<1>;
        case 2: return (const void *)int_probe_kernel<2>;
        case 3: return (const void *)int_probe_kernel<3>;
        case 4: return (const void *)int_probe_kernel<4>;
        default: return nullptr;
    }
}

}  // namespace msa

using namespace msa;

extern "C" msa_status msa_probe_int_pipe(msa_ctx *ctx, int32_t op, int32_t iters, int64_t *lane_ops, void *stream) {
    if (!ctx || !lane_ops || iters <= 0 || !probe_fn(op))
        return set_error(ctx, MSA_EINVAL, "msa_probe_int_pipe: bad argument");
    int occ = 1;
    if (msa_status rc = occupancy(ctx, probe_fn(op), kProbeThreads, 0, &occ)) return rc;
    const int64_t grid = (int64_t)ctx->sm_count * occ;
    const int64_t threads = grid * kProbeThreads;
    if (threads * (int64_t)sizeof(uint32_t) > ctx->ws_bytes)
        return set_error(ctx, MSA_ENOMEM, "msa_probe_int_pipe: workspace too small");
    uint32_t *sink = reinterpret_cast<uint32_t *>(ctx->ws);
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t seed = 0x2545f491u;
    switch (op) {
        case 0: int_probe_kernel<0><<<(int)grid, kProbeThreads, 0, st>>>(sink, iters, seed); break;
        case 1: int_probe_kernel<1><<<(int)grid, kProbeThreads, 0, st>>>(sink, iters, seed); break;
        case 2: int_probe_kernel<2><<<(int)grid, kProbeThreads, 0, st>>>(sink, iters, seed); break;
        case 3: int_probe_kernel<3><<<(int)grid, kProbeThreads, 0, st>>>(sink, iters, seed); break;
        default: int_probe_kernel<4><<<(int)grid, kProbeThreads, 0, st>>>(sink, iters, seed); break;
    }
    ++ctx->launches;
    *lane_ops = threads * (int64_t)iters * probe_ops_per_iter(op);
    return cuda_check(ctx, cudaGetLastError(), "msa_probe_int_pipe launch");
}
