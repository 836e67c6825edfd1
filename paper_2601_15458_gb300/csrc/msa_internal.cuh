// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "msa.h"

namespace msa {

constexpr int kDeviceErrWords = 4;  // [code, detail0, detail1, detail2]

// Device error codes recorded by kernels (the first one wins).
constexpr int kErrIndex = 1;     // pair index outside [0, n_seqs)
constexpr int kErrSymbol = 2;    // residue outside the alphabet
constexpr int kErrLength = 3;    // sequence longer than max_len / bad offsets
constexpr int kErrTimeout = 4;   // a bounded wait ran out
constexpr int kErrCapacity = 5;  // a device-side capacity bound was exceeded

struct Tune;  // autotune table (lev_plan.cu)

}  // namespace msa

struct msa_ctx {
    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;
    char *ws = nullptr;          // workspace base
    int64_t ws_bytes = 0;
    int32_t *dev_err = nullptr;  // kDeviceErrWords ints
    std::string last_error;
    msa::Tune *tune = nullptr;
    // launch accounting and optional event timing of the DP kernels
    int64_t launches = 0;
    bool prof = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
    double prof_ms = 0.0;
    // side streams for running independent bucket kernels concurrently
    // (fork / join through events, so stream capture still works)
    static constexpr int kSide = 40;
    // streams [0, kBandSide) take the band buckets of a banded call (one
    // bucket each), the rest the full-DP batch running beside them
    static constexpr int kBandSide = 32;
    cudaStream_t side[kSide] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kSide] = {};
    // resident blocks per SM of each kernel launched through this context
    // (its device), keyed by kernel; filled on first use (one host thread at
    // a time uses a context, so no lock is needed)
    std::map<const void *, int> occ;
    bool mlp_smem_set = false;
    bool band_lane_smem_set = false;
};

namespace msa {

msa_status set_error(msa_ctx *ctx, msa_status code, const char *fmt, ...);
msa_status cuda_check(msa_ctx *ctx, cudaError_t e, const char *what);

// Resident blocks per SM (at least 1) of kernel `fn` launched with `threads`
// threads and `smem` bytes of dynamic shared memory, on the context's device;
// cached in the context.
inline msa_status occupancy(msa_ctx *ctx, const void *fn, int threads, size_t smem, int *out) {
    auto it = ctx->occ.find(fn);
    if (it != ctx->occ.end()) {
        *out = it->second;
        return MSA_OK;
    }
    int blocks = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, threads, smem);
    if (e != cudaSuccess) return cuda_check(ctx, e, "occupancy query");
    *out = blocks > 0 ? blocks : 1;
    ctx->occ[fn] = *out;
    return MSA_OK;
}

// Records a device error (first one wins).
__device__ __forceinline__ void record_error(int32_t *err, int code, long long d0, long long d1) {
    if (atomicCAS(err, 0, code) == 0) {
        err[1] = (int32_t)d0;
        err[2] = (int32_t)(d0 >> 32);
        err[3] = (int32_t)d1;
    }
}

// Bump allocator over the context workspace for one call.
struct Arena {
    char *base;
    int64_t cap;
    int64_t used = 0;
    template <class T>
    T *take(int64_t count) {
        int64_t bytes = (count * (int64_t)sizeof(T) + 255) & ~int64_t(255);
        if (used + bytes > cap) return nullptr;
        T *p = reinterpret_cast<T *>(base + used);
        used += bytes;
        return p;
    }
};

// Brackets the DP kernels of one call with events when profiling is on.
struct ProfScope {
    msa_ctx *ctx;
    cudaStream_t st;
    cudaEvent_t e1 = nullptr;
    ProfScope(msa_ctx *c, cudaStream_t s) : ctx(c), st(s) {
        if (!ctx->prof) return;
        cudaEvent_t e0;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
        ctx->prof_events.push_back({e0, e1});
    }
    ~ProfScope() {
        if (e1) cudaEventRecord(e1, st);
    }
};

msa_status lev_run(msa_ctx *ctx, const msa_seqset *s, const int32_t *pairs, int64_t P, int32_t *d_out,
                   cudaStream_t st, const int32_t *idx, const int32_t *count_dev, Arena *outer, int side_base = 0);
msa_status lev_validate(msa_ctx *ctx, const msa_seqset *s, const int32_t *pairs, int64_t P, const void *out,
                        const char *who);
int64_t lev_workspace(int64_t P, int32_t n);
// Certified banded Levenshtein over a pair list with scratch from `ar`
// (msa_lev_banded_batch's body).
msa_status lev_banded_run(msa_ctx *ctx, const msa_seqset *s, const int32_t *pairs, int64_t P, const int32_t *k0,
                          int32_t *d_out, int32_t *k_used_out, cudaStream_t st, Arena &ar);

// Bit-parallel NW for the unit cost model (nw_bv.cu), launched by nw_run.
int64_t nw_bv_slab_bytes(int max_len);
const void *nw_bv_kernel_fn();
constexpr int kBvThreads = 128;
cudaError_t nw_bv_launch(msa_ctx *ctx, const uint8_t *codes, const int64_t *offs, int32_t n_seqs, int64_t total,
                         int32_t max_len, const int32_t *pairs, int64_t P, int32_t gap, int32_t *score,
                         uint8_t *ops, const int64_t *ops_off, int32_t *ops_len, char *slabs, int64_t slab_bytes,
                         int64_t warps, int32_t *counter, int32_t *fb_list, int32_t *fb_count, cudaStream_t st);
// With sub (device int32 [nsym][nsym], nsym <= 32) a substitution costs
// sub[a][b] by code instead of match / mismatch.
msa_status nw_affine_run(msa_ctx *ctx, Arena &ar, const uint8_t *codes, const int64_t *offs, int32_t n_seqs,
                         int64_t total, int32_t max_len, const int32_t *pairs, int64_t P, int32_t match,
                         int32_t mismatch, int32_t open, int32_t ext, int32_t *score_out, uint8_t *ops_out,
                         const int64_t *ops_off, int32_t *ops_len_out, cudaStream_t st, const int32_t *sub = nullptr,
                         int32_t nsym = 0);
// out[0..n] = exclusive prefix sums of in[0..n) and the total (tile scan,
// two launches); tsum: scan_tiles(n) values of scratch.
int64_t scan_tiles(int64_t n);
void exclusive_scan(const int32_t *in, int32_t n, int32_t *out, int32_t *tsum, cudaStream_t st);
void exclusive_scan64(const int64_t *in, int32_t n, int64_t *out, int64_t *tsum, cudaStream_t st);
msa_status nw_run(msa_ctx *ctx, Arena &ar, const uint8_t *codes, const int64_t *offs, int32_t n_seqs, int64_t total,
                  int32_t max_len, const int32_t *pairs, int64_t P, int32_t match, int32_t mismatch, int32_t gap,
                  int32_t *score_out, uint8_t *ops_out, const int64_t *ops_off, int32_t *ops_len_out,
                  cudaStream_t st);

// Runs launch(i, stream) for i < count, spread over side streams
// [base, base + width) of the context after a fork from `st`.  With join
// (the default) `st` then waits for all of them; otherwise the caller joins
// later with join_side().
template <class F>
cudaError_t run_concurrent(msa_ctx *ctx, cudaStream_t st, int count, F launch, int base = 0, int width = 8,
                           bool join = true) {
    if (count <= 1 || !ctx->fork_ev) {
        for (int i = 0; i < count; ++i) launch(i, st);
        return cudaGetLastError();
    }
    cudaError_t e = cudaEventRecord(ctx->fork_ev, st);
    const int used = count < width ? count : width;
    for (int k = 0; k < used && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(ctx->side[base + k], ctx->fork_ev, 0);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < count; ++i) launch(i, ctx->side[base + i % used]);
    if (join) {
        for (int k = 0; k < used && e == cudaSuccess; ++k) {
            e = cudaEventRecord(ctx->join_ev[base + k], ctx->side[base + k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->join_ev[base + k], 0);
        }
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Makes `st` wait for side streams [base, base + width).
inline cudaError_t join_side(msa_ctx *ctx, cudaStream_t st, int base, int width) {
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < width && e == cudaSuccess; ++k) {
        e = cudaEventRecord(ctx->join_ev[base + k], ctx->side[base + k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->join_ev[base + k], 0);
    }
    return e;
}

inline int bits_of(int alphabet) { return alphabet == MSA_DNA ? 2 : 5; }
inline int sigma_of(int alphabet) { return alphabet == MSA_DNA ? 4 : 20; }

}  // namespace msa
