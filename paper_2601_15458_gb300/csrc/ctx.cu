// Context, error reporting, sizes, and the packed-sequence loader (A1).
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>

#include "msa_internal.cuh"

namespace msa {

msa_status set_error(msa_ctx *ctx, msa_status code, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->last_error = buf;
    }
    return code;
}

msa_status cuda_check(msa_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return MSA_OK;
    if (e == cudaErrorMemoryAllocation)
        return set_error(ctx, MSA_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return set_error(ctx, MSA_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void destroy_tune(Tune *t);
Tune *create_tune();

// ---------------------------------------------------------------------------
// A1: ASCII -> byte codes + bit planes.  One thread per 32-position arena
// word: two 16-byte loads, a 256-entry table lookup per byte, two 16-byte
// stores of codes and B plane words.  Traffic 1 + 1 + B/8 bytes per residue.
// ---------------------------------------------------------------------------
// DNA, 4 residues per integer op (SWAR): for A, C, G, T (0x41, 0x43, 0x47,
// 0x54) the code is ((c >> 1) ^ (c >> 2)) & 3 = 0, 1, 2, 3, computed for the 4
// bytes of a word at once; the word is valid when the byte permute of "ACGT"
// by those codes gives back the 4 bytes (compared in the order 0, 2, 1, 3,
// the order in which c | c >> 12 lays the codes out as permute selectors);
// plane p's 4 bits are gathered by one multiply, ((c >> p) & 0x01010101) *
// 0x10204080 >> 28 (the partial products never overlap, so no carries).  A
// word with another byte takes the per-byte path: the first bad byte is
// recorded and bad bytes get code 0, as in pack_kernel.
__device__ __forceinline__ uint32_t dna_code_of(uint32_t b) {
    return b == 'A' ? 0u : b == 'C' ? 1u : b == 'G' ? 2u : b == 'T' ? 3u : 0xFFu;
}

__global__ void __launch_bounds__(256) pack_dna_kernel(const uint8_t *__restrict__ ascii, int64_t total,
                                                       uint8_t *__restrict__ codes, uint32_t *__restrict__ planes,
                                                       int64_t nwords, int32_t *err) {
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nwords;
         w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t base = w * 32;
        uint32_t x[8];
        const bool full = base + 32 <= total;
        if (full) {
            const uint4 *src = reinterpret_cast<const uint4 *>(ascii + base);
            const uint4 v0 = __ldg(src), v1 = __ldg(src + 1);
            x[0] = v0.x; x[1] = v0.y; x[2] = v0.z; x[3] = v0.w;
            x[4] = v1.x; x[5] = v1.y; x[6] = v1.z; x[7] = v1.w;
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                uint32_t v = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int64_t pos = base + 4 * i + k;
                    v |= (uint32_t)(pos < total ? ascii[pos] : 'A') << (8 * k);   // past the end: code 0
                }
                x[i] = v;
            }
        }
        uint32_t c[8], p0 = 0u, p1 = 0u;
        bool ok = true;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            c[i] = ((x[i] >> 1) ^ (x[i] >> 2)) & 0x03030303u;
            const uint32_t sel = c[i] | (c[i] >> 12);
            ok &= __byte_perm(0x54474341u, 0u, sel) == __byte_perm(x[i], 0u, 0x3120u);
        }
        if (!ok) {
            int badk = -1;
            uint32_t badb = 0u;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                uint32_t cc = 0u;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t b = (x[i] >> (8 * k)) & 0xFFu;
                    uint32_t v = dna_code_of(b);
                    if (v == 0xFFu) {
                        if (badk < 0) {
                            badk = 4 * i + k;
                            badb = b;
                        }
                        v = 0u;
                    }
                    cc |= v << (8 * k);
                }
                c[i] = cc;
            }
            if (badk >= 0) record_error(err, kErrSymbol, base + badk, badb);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            p0 |= ((c[i] & 0x01010101u) * 0x10204080u) >> 28 << (4 * i);
            p1 |= (((c[i] >> 1) & 0x01010101u) * 0x10204080u) >> 28 << (4 * i);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(codes + base);
        dst[0] = make_uint4(c[0], c[1], c[2], c[3]);
        dst[1] = make_uint4(c[4], c[5], c[6], c[7]);
        planes[w * 2] = p0;
        planes[w * 2 + 1] = p1;
    }
}

template <int B>
__global__ void __launch_bounds__(256) pack_kernel(const uint8_t *__restrict__ ascii, int64_t total,
                                                   uint8_t *__restrict__ codes,
                                                   uint32_t *__restrict__ planes, int64_t nwords,
                                                   int alphabet, int32_t *err) {
    __shared__ uint8_t lut[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        uint8_t v = 0xFF;
        if (alphabet == MSA_DNA) {
            const char *al = "ACGT";
            for (int k = 0; k < 4; ++k)
                if (i == al[k]) v = (uint8_t)k;
        } else {
            const char *al = "ACDEFGHIKLMNPQRSTVWY";
            for (int k = 0; k < 20; ++k)
                if (i == al[k]) v = (uint8_t)k;
        }
        lut[i] = v;
    }
    __syncthreads();
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nwords;
         w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t base = w * 32;
        uint8_t c[32];
        if (base + 32 <= total) {
            const uint4 *src = reinterpret_cast<const uint4 *>(ascii + base);
            uint4 v0 = __ldg(src), v1 = __ldg(src + 1);
            const uint8_t *b0 = reinterpret_cast<const uint8_t *>(&v0);
            const uint8_t *b1 = reinterpret_cast<const uint8_t *>(&v1);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                c[k] = lut[b0[k]];
                c[16 + k] = lut[b1[k]];
            }
        } else {
#pragma unroll
            for (int k = 0; k < 32; ++k) c[k] = (base + k < total) ? lut[ascii[base + k]] : 0;
        }
        uint32_t pl[B];
#pragma unroll
        for (int p = 0; p < B; ++p) pl[p] = 0;
        bool bad = false;
        int badk = 0;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            if (c[k] == 0xFF) {
                if (!bad) badk = k;
                bad = true;
                c[k] = 0;
            }
#pragma unroll
            for (int p = 0; p < B; ++p) pl[p] |= (uint32_t)((c[k] >> p) & 1) << k;
        }
        if (bad) record_error(err, kErrSymbol, base + badk, ascii[base + badk]);
        uint4 o0, o1;
        memcpy(&o0, c, 16);
        memcpy(&o1, c + 16, 16);
        uint4 *dst = reinterpret_cast<uint4 *>(codes + base);
        dst[0] = o0;
        dst[1] = o1;
#pragma unroll
        for (int p = 0; p < B; ++p) planes[w * B + p] = pl[p];
    }
    // the one padding word after the last arena word reads as zero
    if (blockIdx.x == 0 && threadIdx.x < B) planes[nwords * B + threadIdx.x] = 0;
}

__global__ void check_offsets_kernel(const int64_t *__restrict__ offs, int32_t n, int64_t total,
                                     int32_t max_len, int32_t *err) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = offs[s], b = offs[s + 1];
        if (a < 0 || b < a || b > total || b - a > max_len || (s == 0 && a != 0) ||
            (s == n - 1 && b != total))
            record_error(err, kErrLength, s, b - a);
    }
}

}  // namespace msa

using namespace msa;

extern "C" {

const char *msa_version(void) { return "msa-gb300 0.1 sm_103a"; }

int64_t msa_code_bytes(int64_t total) { return ((total + 31) / 32) * 32 + 32; }

int64_t msa_plane_words(int64_t total, int32_t alphabet) {
    return ((total + 31) / 32 + 1) * (alphabet == MSA_DNA ? 2 : 5);
}

msa_status msa_ctx_create(msa_ctx **out, int32_t device, int64_t workspace_bytes) {
    if (!out) return MSA_EINVAL;
    *out = nullptr;
    msa_ctx *ctx = new msa_ctx();
    ctx->device = device;
    msa_status st = cuda_check(ctx, cudaSetDevice(device), "cudaSetDevice");
    if (st) {
        delete ctx;
        return st;
    }
    cudaDeviceProp prop;
    if ((st = cuda_check(ctx, cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties"))) {
        delete ctx;
        return st;
    }
    if (prop.major < 10) {
        delete ctx;
        return MSA_EUNSUPPORTED;
    }
    ctx->sm_count = prop.multiProcessorCount;
    ctx->smem_optin = prop.sharedMemPerBlockOptin;
    ctx->ws_bytes = workspace_bytes > 0 ? workspace_bytes : (int64_t(1) << 30);
    if ((st = cuda_check(ctx, cudaMalloc(&ctx->ws, ctx->ws_bytes), "workspace cudaMalloc")) ||
        (st = cuda_check(ctx, cudaMalloc(&ctx->dev_err, kDeviceErrWords * sizeof(int32_t)),
                         "status cudaMalloc")) ||
        (st = cuda_check(ctx, cudaMemset(ctx->dev_err, 0, kDeviceErrWords * sizeof(int32_t)),
                         "status memset"))) {
        if (ctx->ws) cudaFree(ctx->ws);
        if (ctx->dev_err) cudaFree(ctx->dev_err);
        delete ctx;
        return st;
    }
    ctx->tune = create_tune();
    bool ok = cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < msa_ctx::kSide && ok; ++k)
        ok = cudaStreamCreateWithFlags(&ctx->side[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&ctx->join_ev[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        msa_ctx_destroy(ctx);
        return MSA_ECUDA;
    }
    *out = ctx;
    return MSA_OK;
}

void msa_ctx_destroy(msa_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    for (auto &ev : ctx->prof_events) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    for (int k = 0; k < msa_ctx::kSide; ++k) {
        if (ctx->side[k]) cudaStreamDestroy(ctx->side[k]);
        if (ctx->join_ev[k]) cudaEventDestroy(ctx->join_ev[k]);
    }
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->dev_err) cudaFree(ctx->dev_err);
    destroy_tune(ctx->tune);
    delete ctx;
}

const char *msa_last_error(const msa_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

msa_status msa_ctx_check(msa_ctx *ctx, void *stream) {
    if (!ctx) return MSA_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    msa_status rc = cuda_check(ctx, cudaStreamSynchronize(st), "cudaStreamSynchronize");
    if (rc) return rc;
    int32_t h[kDeviceErrWords];
    if ((rc = cuda_check(ctx, cudaMemcpy(h, ctx->dev_err, sizeof h, cudaMemcpyDeviceToHost),
                         "status read")))
        return rc;
    if (h[0] == 0) return MSA_OK;
    cudaMemset(ctx->dev_err, 0, sizeof h);
    long long d0 = (long long)(uint32_t)h[1] | ((long long)h[2] << 32);
    switch (h[0]) {
        case kErrIndex:
            return set_error(ctx, MSA_EDATA, "pair %lld refers to sequence %d outside the set", d0, h[3]);
        case kErrSymbol:
            return set_error(ctx, MSA_EDATA, "arena position %lld holds byte %d outside the alphabet", d0, h[3]);
        case kErrLength:
            return set_error(ctx, MSA_EDATA, "sequence %lld has bad offsets or length %d above max_len", d0, h[3]);
        case kErrTimeout:
            return set_error(ctx, MSA_ETIMEOUT, "bounded device wait ran out (site %lld)", d0);
        case kErrCapacity:
            return set_error(ctx, MSA_ENOMEM, "device capacity exceeded (site %lld, need %d)", d0, h[3]);
        default:
            return set_error(ctx, MSA_EDATA, "device error %d", h[0]);
    }
}

msa_status msa_pack(msa_ctx *ctx, const msa_seqset *s, void *stream) {
    if (!ctx || !s) return MSA_EINVAL;
    if (s->n_seqs < 0 || s->total < 0 || s->max_len < 0)
        return set_error(ctx, MSA_EINVAL, "msa_pack: negative size");
    if (s->alphabet != MSA_DNA && s->alphabet != MSA_PROTEIN)
        return set_error(ctx, MSA_EINVAL, "msa_pack: unknown alphabet %d", s->alphabet);
    if (s->n_seqs == 0) return MSA_OK;
    if (!s->ascii || !s->offs || !s->codes || !s->planes)
        return set_error(ctx, MSA_EINVAL, "msa_pack: null pointer");
    if (((uintptr_t)s->ascii & 15) || ((uintptr_t)s->codes & 15))
        return set_error(ctx, MSA_EINVAL, "msa_pack: ascii and codes must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nwords = (s->total + 31) / 32;
    ctx->launches += 2;
    check_offsets_kernel<<<(s->n_seqs + 255) / 256 < 1024 ? (s->n_seqs + 255) / 256 : 1024, 256, 0, st>>>(
        s->offs, s->n_seqs, s->total, s->max_len, ctx->dev_err);
    int64_t blocks = (nwords + 255) / 256;
    if (blocks > ctx->sm_count * 16) blocks = ctx->sm_count * 16;
    if (blocks < 1) blocks = 1;
    if (s->alphabet == MSA_DNA)
        pack_dna_kernel<<<(int)blocks, 256, 0, st>>>(s->ascii, s->total, s->codes, s->planes, nwords, ctx->dev_err);
    else
        pack_kernel<5><<<(int)blocks, 256, 0, st>>>(s->ascii, s->total, s->codes, s->planes, nwords,
                                                     s->alphabet, ctx->dev_err);
    return cuda_check(ctx, cudaGetLastError(), "msa_pack launch");
}

msa_status msa_prof_enable(msa_ctx *ctx, int32_t on) {
    if (!ctx) return MSA_EINVAL;
    ctx->prof = on != 0;
    return MSA_OK;
}

msa_status msa_prof_read(msa_ctx *ctx, double *dp_kernel_ms, int64_t *launches, int32_t reset) {
    if (!ctx) return MSA_EINVAL;
    for (auto &ev : ctx->prof_events) {
        cudaError_t e = cudaEventSynchronize(ev.second);
        if (e != cudaSuccess) return cuda_check(ctx, e, "msa_prof_read");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev.first, ev.second);
        ctx->prof_ms += ms;
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    ctx->prof_events.clear();
    if (dp_kernel_ms) *dp_kernel_ms = ctx->prof_ms;
    if (launches) *launches = ctx->launches;
    if (reset) {
        ctx->prof_ms = 0.0;
        ctx->launches = 0;
    }
    return MSA_OK;
}

}  // extern "C"
