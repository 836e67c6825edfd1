// Learned band proposer: 4-mer count profiles (A8), the MLP 256->128->64->1
// forward (A9) and its training step (A10), and msa_band_predict.
//
// The network maps the pair feature x = (c_a - c_b)^2 / ((len_a + len_b) / 2)
// over the 256 DNA 4-mer counts to y ~ f(a, b) / max(m, n).  Squared
// differences: if the k-mers that edits remove and add fall into the bins
// like independent Poisson draws, E (c_a - c_b)_i^2 is the number of changed
// windows in bin i, so the feature sum estimates the changed windows per
// residue whatever the length, where absolute differences cancel more in
// longer sequences (more changes share a bin).  Weights and
// activations are bf16, products accumulate in fp32 on the tensor cores
// (mma.sync m16n8k16 bf16); biases and the last layer are fp32.  The
// proposer only picks the starting band of msa_lev_banded_batch, whose
// certificate keeps every distance exact.
//
// Parameter layout (fp32, NP = 41217 floats), also used for the Adam moments
// and the gradient:  W1[128][256] (out-major), b1[128], W2[64][128], b2[64],
// W3[64], b3[1].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "msa_internal.cuh"

namespace msa {

constexpr int kF = 256, kH1 = 128, kH2 = 64;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH1 * kF, kOffW2 = kOffB1 + kH1, kOffB2 = kOffW2 + kH2 * kH1,
              kOffW3 = kOffB2 + kH2, kOffB3 = kOffW3 + kH2, kNP = kOffB3 + 1;
constexpr int kS1 = kF + 8, kS2 = kH1 + 8, kS3 = kH2 + 8;  // padded smem row strides (bf16 elements)
constexpr int kMlpWarps = 8;

// state buffer: params | m | v | grad (fp32, NP each) | bf16 weights (NP) |
// 64 spare | loss/aux (64) | band calibration (64)
struct MlpState {
    float *p, *m, *v, *g;
    __nv_bfloat16 *h;
    float *aux;   // [0] loss sum of the last step, [1] step count
    float *cal;   // [0] 1 when fitted, [1 .. kCalKnots] knots of c(yhat)
};

// Band calibration: knots of a monotone piecewise-linear map at yhat =
// 0, 1/32, ..., 1 (the table is this library's addition to the band policy).
constexpr int kCalKnots = 33;
constexpr int kCalMinPairs = 16;
constexpr int kCalFloats = 64;

__host__ __device__ inline int64_t np_round(int64_t x) { return (x + 63) / 64 * 64; }

static MlpState state_of(void *base) {
    MlpState s;
    float *f = reinterpret_cast<float *>(base);
    const int64_t R = np_round(kNP);
    s.p = f;
    s.m = f + R;
    s.v = f + 2 * R;
    s.g = f + 3 * R;
    s.h = reinterpret_cast<__nv_bfloat16 *>(f + 4 * R);
    s.aux = f + 4 * R + R / 2 + 64;
    s.cal = s.aux + 64;
    return s;
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// A fragment of a row-major 16 x 16 tile at A (stride lda elements).
__device__ __forceinline__ void frag_a(uint32_t (&a)[4], const __nv_bfloat16 *A, int lda, int lane) {
    const int g = lane >> 2, t = lane & 3;
    a[0] = ld32(A + g * lda + 2 * t);
    a[1] = ld32(A + (g + 8) * lda + 2 * t);
    a[2] = ld32(A + g * lda + 2 * t + 8);
    a[3] = ld32(A + (g + 8) * lda + 2 * t + 8);
}

// B fragment of a 16(k) x 8(n) tile stored as Bt[n][k] (k contiguous, stride ldb).
__device__ __forceinline__ void frag_b(uint32_t (&b)[2], const __nv_bfloat16 *Bt, int ldb, int lane) {
    const int g = lane >> 2, t = lane & 3;
    b[0] = ld32(Bt + g * ldb + 2 * t);
    b[1] = ld32(Bt + g * ldb + 2 * t + 8);
}

// ---------------------------------------------------------------------------
// A8: 4-mer counts.  One warp per sequence, counts in shared memory.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) kmer_kernel(const uint8_t *__restrict__ codes, const int64_t *__restrict__ offs,
                                                   int32_t n, int64_t total, uint16_t *__restrict__ prof,
                                                   int32_t *err) {
    __shared__ uint32_t cnt[8][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t s = (int64_t)blockIdx.x * 8 + w; s < n; s += (int64_t)gridDim.x * 8) {
        for (int k = lane; k < 256; k += 32) cnt[w][k] = 0;
        __syncwarp();
        const int64_t a = offs[s], b = offs[s + 1];
        if (a < 0 || b < a || b > total || b - a > 65535) {
            if (lane == 0) record_error(err, kErrLength, s, b - a);
        } else {
            const uint8_t *c = codes + a;
            const int L = (int)(b - a);
            for (int i = lane; i + 3 < L; i += 32) {
                const int v = ((c[i] & 3) << 6) | ((c[i + 1] & 3) << 4) | ((c[i + 2] & 3) << 2) | (c[i + 3] & 3);
                atomicAdd(&cnt[w][v], 1u);
            }
        }
        __syncwarp();
        for (int k = lane; k < 256; k += 32) prof[s * 256 + k] = (uint16_t)cnt[w][k];
        __syncwarp();
    }
}

// Pair features of 16 pairs into a warp's shared tile X[16][kS1] (bf16).
__device__ __forceinline__ void features_tile(__nv_bfloat16 *X, const uint16_t *__restrict__ prof,
                                              const int64_t *__restrict__ offs, const int32_t *__restrict__ pairs,
                                              int64_t row0, int64_t P, int32_t n, int lane) {
    for (int r = 0; r < 16; ++r) {
        const int64_t p = row0 + r;
        const int a = p < P ? pairs[2 * p] : -1, b = p < P ? pairs[2 * p + 1] : -1;
        if (a >= 0 && a < n && b >= 0 && b < n) {
            const float den0 = 0.5f * (float)((offs[a + 1] - offs[a]) + (offs[b + 1] - offs[b]));
            const float den = den0 > 0.f ? den0 : 1.f;
            const uint16_t *ca = prof + (int64_t)a * 256, *cb = prof + (int64_t)b * 256;
#pragma unroll
            for (int k = lane * 8; k < lane * 8 + 8; ++k) {
                const float d = fabsf((float)ca[k] - (float)cb[k]);
                X[r * kS1 + k] = __float2bfloat16_rn(d * d / den);
            }
        } else {
#pragma unroll
            for (int k = lane * 8; k < lane * 8 + 8; ++k) X[r * kS1 + k] = __float2bfloat16_rn(0.f);
        }
    }
}

// Pair features to global memory: one warp per pair, 8 features per lane.
__global__ void __launch_bounds__(256) features_kernel(const uint16_t *__restrict__ prof, const int64_t *__restrict__ offs,
                                                       int32_t n, const int32_t *__restrict__ pairs, int64_t P,
                                                       __nv_bfloat16 *__restrict__ X, int32_t *err) {
    const int lane = threadIdx.x & 31;
    for (int64_t p = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); p < P; p += (int64_t)gridDim.x * 8) {
        const int a = pairs[2 * p], b = pairs[2 * p + 1];
        if (a < 0 || a >= n || b < 0 || b >= n) {
            if (lane == 0) record_error(err, kErrIndex, p, a);
            continue;
        }
        const float den0 = 0.5f * (float)((offs[a + 1] - offs[a]) + (offs[b + 1] - offs[b]));
        const float den = den0 > 0.f ? den0 : 1.f;
        const uint16_t *ca = prof + (int64_t)a * 256, *cb = prof + (int64_t)b * 256;
#pragma unroll
        for (int k = lane * 8; k < lane * 8 + 8; ++k) {
            const float d = fabsf((float)ca[k] - (float)cb[k]);
            X[p * 256 + k] = __float2bfloat16_rn(d * d / den);
        }
    }
}

// Loads the bf16 weights and fp32 biases into shared memory.
__device__ __forceinline__ void load_weights(__nv_bfloat16 *W1s, __nv_bfloat16 *W2s, float *bias, const MlpState st) {
    for (int i = threadIdx.x; i < kH1 * kF; i += blockDim.x) W1s[(i / kF) * kS1 + (i % kF)] = st.h[kOffW1 + i];
    for (int i = threadIdx.x; i < kH2 * kH1; i += blockDim.x) W2s[(i / kH1) * kS2 + (i % kH1)] = st.h[kOffW2 + i];
    for (int i = threadIdx.x; i < kH1 + kH2 + kH2 + 1; i += blockDim.x) {
        float v;
        if (i < kH1) v = st.p[kOffB1 + i];
        else if (i < kH1 + kH2) v = st.p[kOffB2 + i - kH1];
        else if (i < kH1 + 2 * kH2) v = __bfloat162float(st.h[kOffW3 + i - kH1 - kH2]);
        else v = st.p[kOffB3];
        bias[i] = v;
    }
}

// Forward of a 16-row tile.  X (bf16 [16][kS1]) -> H1 (bf16 [16][kS2]),
// H2 (bf16 [16][kS3]) and y for rows g and g+8 (returned in y0, y1 on lanes
// with (lane & 3) == 0).
__device__ __forceinline__ void forward_tile(const __nv_bfloat16 *X, __nv_bfloat16 *H1, __nv_bfloat16 *H2,
                                             const __nv_bfloat16 *W1s, const __nv_bfloat16 *W2s, const float *bias,
                                             int lane, float &y0, float &y1) {
    const int g = lane >> 2, t = lane & 3;
    {
        float acc[16][4];
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll 4
        for (int k0 = 0; k0 < kF; k0 += 16) {
            uint32_t a[4];
            frag_a(a, X + k0, kS1, lane);
#pragma unroll
            for (int nt = 0; nt < 16; ++nt) {
                uint32_t b[2];
                frag_b(b, W1s + nt * 8 * kS1 + k0, kS1, lane);
                mma16816(acc[nt], a, b);
            }
        }
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            const int c = nt * 8 + 2 * t;
            const float b0 = bias[c], b1 = bias[c + 1];
            H1[g * kS2 + c] = __float2bfloat16_rn(fmaxf(acc[nt][0] + b0, 0.f));
            H1[g * kS2 + c + 1] = __float2bfloat16_rn(fmaxf(acc[nt][1] + b1, 0.f));
            H1[(g + 8) * kS2 + c] = __float2bfloat16_rn(fmaxf(acc[nt][2] + b0, 0.f));
            H1[(g + 8) * kS2 + c + 1] = __float2bfloat16_rn(fmaxf(acc[nt][3] + b1, 0.f));
        }
    }
    __syncwarp();
    float s0 = 0.f, s1 = 0.f;
    {
        float acc[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
        for (int k0 = 0; k0 < kH1; k0 += 16) {
            uint32_t a[4];
            frag_a(a, H1 + k0, kS2, lane);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                uint32_t b[2];
                frag_b(b, W2s + nt * 8 * kS2 + k0, kS2, lane);
                mma16816(acc[nt], a, b);
            }
        }
        const float *b2 = bias + kH1;
        const float *w3 = bias + kH1 + kH2;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int c = nt * 8 + 2 * t;
            const __nv_bfloat16 h00 = __float2bfloat16_rn(fmaxf(acc[nt][0] + b2[c], 0.f));
            const __nv_bfloat16 h01 = __float2bfloat16_rn(fmaxf(acc[nt][1] + b2[c + 1], 0.f));
            const __nv_bfloat16 h10 = __float2bfloat16_rn(fmaxf(acc[nt][2] + b2[c], 0.f));
            const __nv_bfloat16 h11 = __float2bfloat16_rn(fmaxf(acc[nt][3] + b2[c + 1], 0.f));
            H2[g * kS3 + c] = h00;
            H2[g * kS3 + c + 1] = h01;
            H2[(g + 8) * kS3 + c] = h10;
            H2[(g + 8) * kS3 + c + 1] = h11;
            s0 += __bfloat162float(h00) * w3[c] + __bfloat162float(h01) * w3[c + 1];
            s1 += __bfloat162float(h10) * w3[c] + __bfloat162float(h11) * w3[c + 1];
        }
    }
    s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
    s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
    const float b3 = bias[kH1 + 2 * kH2];
    y0 = s0 + b3;
    y1 = s1 + b3;
    __syncwarp();
}

constexpr size_t kMlpSmem = (size_t)(kH1 * kS1 + kH2 * kS2) * 2 + (kH1 + 2 * kH2 + 1 + 3) * 4 +
                            (size_t)kMlpWarps * (16 * kS1 + 16 * kS2 + 16 * kS3) * 2;

struct FwdArgs {
    MlpState st;
    const __nv_bfloat16 *X;      // [P][256] bf16 (forward from features given)
    const uint16_t *prof;        // or profiles + pairs (fused band predictor)
    const int64_t *offs;
    const int32_t *pairs;
    int64_t P;
    int32_t n_seqs;
    float *yhat;                 // [P]
    int32_t *k_out;              // [P] band, or null
    float gamma;
    int32_t margin;
};

// c(yhat): the calibration knots interpolated at clamp(yhat, 0, 1) * 32,
// each operation rounded on its own (no fused multiply-add), so a float32
// restatement reproduces it bit for bit.
__device__ __forceinline__ float band_cal(const float *knots, float y) {
    const float x = __fmul_rn(fminf(fmaxf(y, 0.f), 1.f), 32.f);
    const int i = min((int)x, kCalKnots - 2);
    const float f = __fsub_rn(x, (float)i);
    const float k0 = knots[i], k1 = knots[i + 1];
    return __fadd_rn(k0, __fmul_rn(f, __fsub_rn(k1, k0)));
}

// Forward over P rows; with k_out also the band policy
//   k = max(|m - n|, ceil((1 + gamma) * c * max(m, n)) + margin),
// c = max(yhat, 0), or c(yhat) once the state holds a calibration.
__global__ void __launch_bounds__(kMlpWarps * 32) mlp_forward_kernel(FwdArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16 *W1s = reinterpret_cast<__nv_bfloat16 *>(smem_raw);
    __nv_bfloat16 *W2s = W1s + kH1 * kS1;
    float *bias = reinterpret_cast<float *>(W2s + kH2 * kS2);
    __nv_bfloat16 *tiles = reinterpret_cast<__nv_bfloat16 *>(bias + kH1 + 2 * kH2 + 1 + 3);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __nv_bfloat16 *X = tiles + w * (16 * kS1 + 16 * kS2 + 16 * kS3);
    __nv_bfloat16 *H1 = X + 16 * kS1;
    __nv_bfloat16 *H2 = H1 + 16 * kS2;
    load_weights(W1s, W2s, bias, a.st);
    __syncthreads();
    const int64_t ntiles = (a.P + 15) / 16;
    for (int64_t tile = (int64_t)blockIdx.x * kMlpWarps + w; tile < ntiles; tile += (int64_t)gridDim.x * kMlpWarps) {
        const int64_t row0 = tile * 16;
        if (a.X) {
            for (int r = 0; r < 16; ++r) {
                const int64_t p = row0 + r;
                for (int k = lane * 8; k < lane * 8 + 8; ++k)
                    X[r * kS1 + k] = p < a.P ? a.X[p * kF + k] : __float2bfloat16_rn(0.f);
            }
        } else {
            features_tile(X, a.prof, a.offs, a.pairs, row0, a.P, a.n_seqs, lane);
        }
        __syncwarp();
        float y0, y1;
        forward_tile(X, H1, H2, W1s, W2s, bias, lane, y0, y1);
        if ((lane & 3) == 0) {
            const int g = lane >> 2;
            for (int h = 0; h < 2; ++h) {
                const int64_t p = row0 + g + 8 * h;
                if (p >= a.P) continue;
                const float y = h ? y1 : y0;
                a.yhat[p] = y;
                if (a.k_out) {
                    const int x = a.pairs[2 * p], z = a.pairs[2 * p + 1];
                    if (x < 0 || x >= a.n_seqs || z < 0 || z >= a.n_seqs) {
                        a.k_out[p] = 0;
                        continue;
                    }
                    const int lx = (int)(a.offs[x + 1] - a.offs[x]), lz = (int)(a.offs[z + 1] - a.offs[z]);
                    const int mx = max(lx, lz);
                    const float c = a.st.cal[0] != 0.f ? band_cal(a.st.cal + 1, y) : fmaxf(y, 0.f);
                    const float kf = ceilf(__fmul_rn(__fmul_rn(1.f + a.gamma, c), (float)mx));
                    const int kk = (int)fminf(kf, 2.0e9f) + a.margin;
                    a.k_out[p] = max(abs(lx - lz), kk);
                }
            }
        }
    }
}

// Calibration fit, one block: for each knot i, the tau-quantile of the
// clamped y over the pairs whose yhat rounds to i / 32 (smallest v with
// #{y <= v} >= ceil(tau n)), found by a radix select on the float bits (y in
// [0, 1] orders like its bits), 8 bits per pass; bins with fewer than
// kCalMinPairs pairs keep the identity; a running maximum makes the map
// monotone.  4 passes over the inputs per knot.
__device__ __forceinline__ int cal_bin(float yh) {
    const float x = fminf(fmaxf(__fadd_rn(__fmul_rn(yh, 32.f), 0.5f), 0.f), 32.f);
    return (int)x;
}

__global__ void __launch_bounds__(1024) band_calibrate_kernel(const float *__restrict__ yhat,
                                                              const float *__restrict__ y, int64_t N, double tau,
                                                              float *cal) {
    __shared__ uint32_t hist[256];
    __shared__ unsigned long long s_cnt;
    __shared__ uint32_t s_prefix;
    __shared__ long long s_rank;
    __shared__ float s_knot[kCalKnots];
    const int tid = threadIdx.x;
    for (int b = 0; b < kCalKnots; ++b) {
        if (tid == 0) s_cnt = 0ull;
        __syncthreads();
        unsigned long long c = 0;
        for (int64_t j = tid; j < N; j += blockDim.x) c += cal_bin(yhat[j]) == b;
        atomicAdd(&s_cnt, c);
        __syncthreads();
        const long long nb = (long long)s_cnt;
        if (nb < kCalMinPairs) {
            if (tid == 0) s_knot[b] = -1.f;
            __syncthreads();
            continue;
        }
        long long r = (long long)ceil(tau * (double)nb);
        r = r < 1 ? 1 : (r > nb ? nb : r);
        uint32_t prefix = 0;
        for (int shift = 24; shift >= 0; shift -= 8) {
            for (int i = tid; i < 256; i += blockDim.x) hist[i] = 0;
            __syncthreads();
            for (int64_t j = tid; j < N; j += blockDim.x) {
                if (cal_bin(yhat[j]) != b) continue;
                const uint32_t bits = __float_as_uint(fminf(fmaxf(y[j], 0.f), 1.f));
                if (shift == 24 || (bits >> (shift + 8)) == prefix) atomicAdd(&hist[(bits >> shift) & 255u], 1u);
            }
            __syncthreads();
            if (tid == 0) {
                long long cum = 0;
                int dg = 0;
                for (; dg < 255; ++dg) {
                    if (cum + (long long)hist[dg] >= r) break;
                    cum += hist[dg];
                }
                s_rank = r - cum;
                s_prefix = (prefix << 8) | (uint32_t)dg;
            }
            __syncthreads();
            prefix = s_prefix;
            r = s_rank;
            __syncthreads();
        }
        if (tid == 0) s_knot[b] = __uint_as_float(prefix);
        __syncthreads();
    }
    if (tid == 0) {
        float run = 0.f;
        for (int b = 0; b < kCalKnots; ++b) {
            const float k = s_knot[b] < 0.f ? (float)b / 32.f : s_knot[b];
            run = fmaxf(run, k);
            cal[1 + b] = run;
        }
        cal[0] = 1.f;
    }
}

// ---------------------------------------------------------------------------
// A10: training step.  K1 per 16-row tile: forward, pinball gradient, dh2,
// dh1 = (dh2 W2) * [z1 > 0]; writes the transposed bf16 operands of the
// weight-gradient GEMMs and the bias gradients.  K2: dW1 = dh1^T X and
// dW2 = dh2^T h1 over the batch on the tensor cores, dW3 = dy^T h2.
// K3: Adam on fp32 master weights and the bf16 refresh.
// ---------------------------------------------------------------------------
struct TrainArgs {
    MlpState st;
    const __nv_bfloat16 *Xall;   // [N][256]
    const float *yall;           // [N]
    const int32_t *idx;          // [B] rows of this minibatch
    int64_t N;                   // rows of Xall / yall
    int32_t B, Bp;               // batch and its padded stride (multiple of 16)
    float tau;
    __nv_bfloat16 *XT;           // [256][Bp]
    __nv_bfloat16 *H1T;          // [128][Bp]
    __nv_bfloat16 *H2T;          // [64][Bp]
    __nv_bfloat16 *D1T;          // [128][Bp]
    __nv_bfloat16 *D2T;          // [64][Bp]
    float *dy;                   // [Bp]
};

__global__ void __launch_bounds__(kMlpWarps * 32) train_fwd_bwd_kernel(TrainArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16 *W1s = reinterpret_cast<__nv_bfloat16 *>(smem_raw);
    __nv_bfloat16 *W2s = W1s + kH1 * kS1;
    float *bias = reinterpret_cast<float *>(W2s + kH2 * kS2);
    __nv_bfloat16 *tiles = reinterpret_cast<__nv_bfloat16 *>(bias + kH1 + 2 * kH2 + 1 + 3);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    __nv_bfloat16 *X = tiles + w * (16 * kS1 + 16 * kS2 + 16 * kS3);
    __nv_bfloat16 *H1 = X + 16 * kS1;
    __nv_bfloat16 *H2 = H1 + 16 * kS2;
    load_weights(W1s, W2s, bias, a.st);
    __syncthreads();
    const float *w3 = bias + kH1 + kH2;
    const int ntiles = (a.B + 15) / 16;
    for (int tile = blockIdx.x * kMlpWarps + w; tile < ntiles; tile += gridDim.x * kMlpWarps) {
        const int row0 = tile * 16;
        for (int r = 0; r < 16; ++r) {
            const int b = row0 + r;
            int64_t src = b < a.B ? (int64_t)a.idx[b] : -1;
            if (src >= a.N) src = -1;
            for (int k = lane * 8; k < lane * 8 + 8; ++k) {
                const __nv_bfloat16 v = src >= 0 ? a.Xall[src * kF + k] : __float2bfloat16_rn(0.f);
                X[r * kS1 + k] = v;
                a.XT[(int64_t)k * a.Bp + b] = v;
            }
        }
        __syncwarp();
        float y0, y1;
        forward_tile(X, H1, H2, W1s, W2s, bias, lane, y0, y1);
        // dL/dy for rows g and g + 8 (identical on the 4 lanes of a group)
        float dy[2] = {0.f, 0.f};
        float loss = 0.f;
        for (int h = 0; h < 2; ++h) {
            const int b = row0 + g + 8 * h;
            if (b < a.B) {
                const int64_t src = a.idx[b];
                const float r = (src >= 0 && src < a.N ? a.yall[src] : 0.f) - (h ? y1 : y0);
                dy[h] = (r > 0.f ? -a.tau : 1.f - a.tau) / (float)a.B;
                loss += (r > 0.f ? a.tau * r : (a.tau - 1.f) * r) / (float)a.B;
            }
        }
        float sdy = 0.f;
        if (t == 0) {
            for (int h = 0; h < 2; ++h) {
                const int b = row0 + g + 8 * h;
                a.dy[b] = dy[h];
                sdy += dy[h];
            }
        } else {
            loss = 0.f;
        }
        for (int o = 16; o > 0; o >>= 1) {
            sdy += __shfl_xor_sync(0xffffffffu, sdy, o);
            loss += __shfl_xor_sync(0xffffffffu, loss, o);
        }
        if (lane == 0) {
            atomicAdd(&a.st.g[kOffB3], sdy);
            atomicAdd(&a.st.aux[0], loss);
        }
        // dh2 = dy * w3 * [h2 > 0]; each lane owns columns 2t, 2t+1 of every 8-block
        __nv_bfloat16 *D2 = X;             // reuse the X tile as dh2 [16][kS3] (X is saved in XT)
        for (int c = 2 * t; c < kH2; c += 8) {
            for (int e = 0; e < 2; ++e) {
                const int cc = c + e;
                for (int h = 0; h < 2; ++h) {
                    const int r = g + 8 * h;
                    const float hv = __bfloat162float(H2[r * kS3 + cc]);
                    const float d = hv > 0.f ? dy[h] * w3[cc] : 0.f;
                    D2[r * kS3 + cc] = __float2bfloat16_rn(d);
                }
            }
        }
        __syncwarp();
        // bias gradient of layer 2 and the transposed copies
        for (int c = lane; c < kH2; c += 32) {
            float sb = 0.f;
            for (int r = 0; r < 16; ++r) {
                const int b = row0 + r;
                const __nv_bfloat16 dv = D2[r * kS3 + c];
                if (b < a.B) sb += __bfloat162float(dv);
                a.D2T[(int64_t)c * a.Bp + b] = dv;
                a.H2T[(int64_t)c * a.Bp + b] = H2[r * kS3 + c];
            }
            atomicAdd(&a.st.g[kOffB2 + c], sb);
        }
        for (int c = lane; c < kH1; c += 32)
            for (int r = 0; r < 16; ++r) a.H1T[(int64_t)c * a.Bp + row0 + r] = H1[r * kS2 + c];
        // dh1 = dh2 [16 x 64] . W2 [64 x 128], masked by h1 > 0
        {
            float acc[16][4];
#pragma unroll
            for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
            for (int k0 = 0; k0 < kH2; k0 += 16) {
                uint32_t af[4];
                frag_a(af, D2 + k0, kS3, lane);
#pragma unroll
                for (int nt = 0; nt < 16; ++nt) {
                    // B[k = out][n = in] = W2[out][in]: two rows of W2s per register
                    const int n = nt * 8 + g, k = k0 + 2 * t;
                    uint32_t bf[2];
                    bf[0] = pack2(W2s[k * kS2 + n], W2s[(k + 1) * kS2 + n]);
                    bf[1] = pack2(W2s[(k + 8) * kS2 + n], W2s[(k + 9) * kS2 + n]);
                    mma16816(acc[nt], af, bf);
                }
            }
            __syncwarp();
            __nv_bfloat16 *D1 = X;         // dh1 [16][kS2] over the (consumed) dh2 tile area
#pragma unroll
            for (int nt = 0; nt < 16; ++nt) {
                const int c = nt * 8 + 2 * t;
                for (int e = 0; e < 2; ++e)
                    for (int h = 0; h < 2; ++h) {
                        const int r = g + 8 * h;
                        const float hv = __bfloat162float(H1[r * kS2 + c + e]);
                        D1[r * kS2 + c + e] = __float2bfloat16_rn(hv > 0.f ? acc[nt][2 * h + e] : 0.f);
                    }
            }
            __syncwarp();
            for (int c = lane; c < kH1; c += 32) {
                float sb = 0.f;
                for (int r = 0; r < 16; ++r) {
                    const int b = row0 + r;
                    const __nv_bfloat16 dv = D1[r * kS2 + c];
                    if (b < a.B) sb += __bfloat162float(dv);
                    a.D1T[(int64_t)c * a.Bp + b] = dv;
                }
                atomicAdd(&a.st.g[kOffB1 + c], sb);
            }
        }
        __syncwarp();
    }
}

// C[M][N] += A[M][K] . B[N][K]^T over the batch (both operands K-contiguous),
// one warp per 16 x 64 output tile and K chunk; fp32 atomics into C.
__global__ void __launch_bounds__(128) wgrad_kernel(const __nv_bfloat16 *__restrict__ A, const __nv_bfloat16 *__restrict__ Bm,
                                                    int M, int N, int K, int ld, int kchunk, float *C) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * 4 + (threadIdx.x >> 5);
    const int mt = M / 16, nt4 = N / 64, kc = (K + kchunk - 1) / kchunk;
    if (gw >= mt * nt4 * kc) return;
    const int m0 = (gw % mt) * 16, n0 = ((gw / mt) % nt4) * 64, kb = (gw / (mt * nt4)) * kchunk;
    const int ke = min(K, kb + kchunk);
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    for (int k0 = kb; k0 < ke; k0 += 16) {
        uint32_t af[4];
        frag_a(af, A + (int64_t)m0 * ld + k0, ld, lane);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            uint32_t bf[2];
            frag_b(bf, Bm + (int64_t)(n0 + 8 * j) * ld + k0, ld, lane);
            mma16816(acc[j], af, bf);
        }
    }
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = n0 + 8 * j + 2 * t;
        atomicAdd(&C[(m0 + g) * N + c], acc[j][0]);
        atomicAdd(&C[(m0 + g) * N + c + 1], acc[j][1]);
        atomicAdd(&C[(m0 + g + 8) * N + c], acc[j][2]);
        atomicAdd(&C[(m0 + g + 8) * N + c + 1], acc[j][3]);
    }
}

// dW3[k] = sum_b dy[b] h2[b][k]
__global__ void w3grad_kernel(const __nv_bfloat16 *__restrict__ H2T, const float *__restrict__ dy, int B, int ld,
                              float *g) {
    const int c = blockIdx.x;
    float s = 0.f;
    for (int b = threadIdx.x; b < B; b += blockDim.x) s += dy[b] * __bfloat162float(H2T[(int64_t)c * ld + b]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += part[i];
        g[c] = tot;
    }
}

__global__ void adam_kernel(MlpState st, float lr, float beta1, float beta2, float eps) {
    const float t = st.aux[1] + 1.f;
    const float c1 = 1.f - powf(beta1, t), c2 = 1.f - powf(beta2, t);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNP; i += gridDim.x * blockDim.x) {
        const float g = st.g[i];
        const float m = beta1 * st.m[i] + (1.f - beta1) * g;
        const float v = beta2 * st.v[i] + (1.f - beta2) * g * g;
        st.m[i] = m;
        st.v[i] = v;
        const float p = st.p[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
        st.p[i] = p;
        st.h[i] = __float2bfloat16_rn(p);
        st.g[i] = 0.f;
    }
}

__global__ void step_count_kernel(MlpState st) { st.aux[1] += 1.f; }

__global__ void sync_kernel(MlpState st) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNP; i += gridDim.x * blockDim.x) {
        st.h[i] = __float2bfloat16_rn(st.p[i]);
        st.m[i] = 0.f;
        st.v[i] = 0.f;
        st.g[i] = 0.f;
    }
    if (blockIdx.x == 0 && threadIdx.x < 2) st.aux[threadIdx.x] = 0.f;
}

static msa_status ensure_mlp_smem(msa_ctx *ctx) {
    if (ctx->mlp_smem_set) return MSA_OK;
    cudaError_t e = cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMlpSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(train_fwd_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMlpSmem);
    if (e != cudaSuccess) return cuda_check(ctx, e, "mlp smem attribute");
    ctx->mlp_smem_set = true;
    return MSA_OK;
}

}  // namespace msa

using namespace msa;

extern "C" {

int32_t msa_mlp_num_params(void) { return kNP; }

int64_t msa_mlp_state_bytes(void) { return (4 * np_round(kNP) + np_round(kNP) / 2 + 64 + 64 + kCalFloats) * 4; }

msa_status msa_band_calibrate(msa_ctx *ctx, void *state, const float *yhat, const float *y, int64_t N, float tau,
                              void *stream) {
    if (!ctx || !state) return MSA_EINVAL;
    if (N < 0) return set_error(ctx, MSA_EINVAL, "msa_band_calibrate: N < 0");
    if (!(tau > 0.f && tau <= 1.f)) return set_error(ctx, MSA_EINVAL, "msa_band_calibrate: tau %g not in (0, 1]", tau);
    const cudaStream_t st = (cudaStream_t)stream;
    MlpState S = state_of(state);
    if (N == 0) return cuda_check(ctx, cudaMemsetAsync(S.cal, 0, sizeof(float), st), "msa_band_calibrate reset");
    if (!yhat || !y) return set_error(ctx, MSA_EINVAL, "msa_band_calibrate: null pointer");
    band_calibrate_kernel<<<1, 1024, 0, st>>>(yhat, y, N, (double)tau, S.cal);
    ++ctx->launches;
    return cuda_check(ctx, cudaGetLastError(), "msa_band_calibrate");
}

msa_status msa_mlp_sync(msa_ctx *ctx, void *state, void *stream) {
    if (!ctx || !state) return MSA_EINVAL;
    sync_kernel<<<64, 256, 0, (cudaStream_t)stream>>>(state_of(state));
    ++ctx->launches;
    return cuda_check(ctx, cudaGetLastError(), "msa_mlp_sync");
}

msa_status msa_kmer_profile(msa_ctx *ctx, const msa_seqset *s, uint16_t *prof, void *stream) {
    if (!ctx || !s) return MSA_EINVAL;
    if (s->n_seqs == 0) return MSA_OK;
    if (!prof || !s->codes || !s->offs) return set_error(ctx, MSA_EINVAL, "msa_kmer_profile: null pointer");
    if (s->alphabet != MSA_DNA) return set_error(ctx, MSA_EUNSUPPORTED, "msa_kmer_profile: DNA only");
    const int blocks = (int)std::min<int64_t>((s->n_seqs + 7) / 8, ctx->sm_count * 8);
    kmer_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(s->codes, s->offs, s->n_seqs, s->total, prof, ctx->dev_err);
    ++ctx->launches;
    return cuda_check(ctx, cudaGetLastError(), "msa_kmer_profile");
}

msa_status msa_pair_features(msa_ctx *ctx, const msa_seqset *s, const uint16_t *prof, const int32_t *pairs,
                             int64_t P, uint16_t *X, void *stream) {
    if (!ctx || !s) return MSA_EINVAL;
    if (P < 0) return set_error(ctx, MSA_EINVAL, "msa_pair_features: P < 0");
    if (P == 0) return MSA_OK;
    if (!prof || !pairs || !X || !s->offs) return set_error(ctx, MSA_EINVAL, "msa_pair_features: null pointer");
    const int blocks = (int)std::min<int64_t>((P + 7) / 8, ctx->sm_count * 16);
    features_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(prof, s->offs, s->n_seqs, pairs, P,
                                                              reinterpret_cast<__nv_bfloat16 *>(X), ctx->dev_err);
    ++ctx->launches;
    return cuda_check(ctx, cudaGetLastError(), "msa_pair_features");
}

msa_status msa_mlp_forward(msa_ctx *ctx, const void *state, const uint16_t *X, int64_t P, float *yhat, void *stream) {
    if (!ctx || !state) return MSA_EINVAL;
    if (P < 0) return set_error(ctx, MSA_EINVAL, "msa_mlp_forward: P < 0");
    if (P == 0) return MSA_OK;
    if (!X || !yhat) return set_error(ctx, MSA_EINVAL, "msa_mlp_forward: null pointer");
    msa_status rc = ensure_mlp_smem(ctx);
    if (rc) return rc;
    FwdArgs a{state_of(const_cast<void *>(state)), reinterpret_cast<const __nv_bfloat16 *>(X), nullptr, nullptr,
              nullptr, P, 0, yhat, nullptr, 0.f, 0};
    const int blocks = (int)std::min<int64_t>((P + 16 * kMlpWarps - 1) / (16 * kMlpWarps), ctx->sm_count);
    mlp_forward_kernel<<<blocks, kMlpWarps * 32, kMlpSmem, (cudaStream_t)stream>>>(a);
    ++ctx->launches;
    return cuda_check(ctx, cudaGetLastError(), "msa_mlp_forward");
}

msa_status msa_band_predict(msa_ctx *ctx, const void *state, const msa_seqset *s, const uint16_t *prof,
                            const int32_t *pairs, int64_t P, float gamma, int32_t margin, float *yhat,
                            int32_t *k_out, void *stream) {
    if (!ctx || !state || !s) return MSA_EINVAL;
    if (P < 0) return set_error(ctx, MSA_EINVAL, "msa_band_predict: P < 0");
    if (P == 0) return MSA_OK;
    if (!prof || !pairs || !yhat || !k_out || !s->offs)
        return set_error(ctx, MSA_EINVAL, "msa_band_predict: null pointer");
    msa_status rc = ensure_mlp_smem(ctx);
    if (rc) return rc;
    FwdArgs a{state_of(const_cast<void *>(state)), nullptr, prof, s->offs, pairs, P, s->n_seqs, yhat, k_out, gamma,
              margin};
    const int blocks = (int)std::min<int64_t>((P + 16 * kMlpWarps - 1) / (16 * kMlpWarps), ctx->sm_count);
    ProfScope prof_scope(ctx, (cudaStream_t)stream);
    mlp_forward_kernel<<<blocks, kMlpWarps * 32, kMlpSmem, (cudaStream_t)stream>>>(a);
    ++ctx->launches;
    return cuda_check(ctx, cudaGetLastError(), "msa_band_predict");
}

int64_t msa_mlp_train_workspace_bytes(int32_t B) {
    const int64_t Bp = (B + 15) / 16 * 16;
    return ((int64_t)(kF + kH1 + kH2 + kH1 + kH2) * Bp * 2 + Bp * 4 + 4096);
}

msa_status msa_mlp_train_step(msa_ctx *ctx, void *state, const uint16_t *X, const float *y, int64_t N,
                              const int32_t *idx, int32_t B, float lr, float tau, float *loss_out, void *stream) {
    if (!ctx || !state) return MSA_EINVAL;
    if (B <= 0 || !X || !y || !idx) return set_error(ctx, MSA_EINVAL, "msa_mlp_train_step: bad batch");
    msa_status rc = ensure_mlp_smem(ctx);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int Bp = (B + 15) / 16 * 16;
    Arena ar{ctx->ws, ctx->ws_bytes};
    TrainArgs a{};
    a.st = state_of(state);
    a.Xall = reinterpret_cast<const __nv_bfloat16 *>(X);
    a.yall = y;
    a.idx = idx;
    a.N = N;
    a.B = B;
    a.Bp = Bp;
    a.tau = tau;
    a.XT = ar.take<__nv_bfloat16>((int64_t)kF * Bp);
    a.H1T = ar.take<__nv_bfloat16>((int64_t)kH1 * Bp);
    a.H2T = ar.take<__nv_bfloat16>((int64_t)kH2 * Bp);
    a.D1T = ar.take<__nv_bfloat16>((int64_t)kH1 * Bp);
    a.D2T = ar.take<__nv_bfloat16>((int64_t)kH2 * Bp);
    a.dy = ar.take<float>(Bp);
    if (!a.dy) return set_error(ctx, MSA_ENOMEM, "msa_mlp_train_step: workspace too small for B=%d", B);
    cudaError_t e = cudaMemsetAsync(a.st.aux, 0, sizeof(float), st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "train memset");
    const int tiles = Bp / 16;
    const int blocks = std::max(1, std::min((tiles + kMlpWarps - 1) / kMlpWarps, ctx->sm_count));
    train_fwd_bwd_kernel<<<blocks, kMlpWarps * 32, kMlpSmem, st>>>(a);
    const int kchunk = 512;
    const int kc = (Bp + kchunk - 1) / kchunk;
    const int w1 = (kH1 / 16) * (kF / 64) * kc, w2 = (kH2 / 16) * (kH1 / 64) * kc;
    wgrad_kernel<<<(w1 + 3) / 4, 128, 0, st>>>(a.D1T, a.XT, kH1, kF, Bp, Bp, kchunk, a.st.g + kOffW1);
    wgrad_kernel<<<(w2 + 3) / 4, 128, 0, st>>>(a.D2T, a.H1T, kH2, kH1, Bp, Bp, kchunk, a.st.g + kOffW2);
    w3grad_kernel<<<kH2, 256, 0, st>>>(a.H2T, a.dy, B, Bp, a.st.g + kOffW3);
    if (loss_out) {
        e = cudaMemcpyAsync(loss_out, a.st.aux, sizeof(float), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_check(ctx, e, "train loss copy");
    }
    if (lr != 0.f) {
        adam_kernel<<<64, 256, 0, st>>>(a.st, lr, 0.9f, 0.999f, 1e-8f);
        step_count_kernel<<<1, 1, 0, st>>>(a.st);
        ctx->launches += 2;
    }
    ctx->launches += 4;
    return cuda_check(ctx, cudaGetLastError(), "msa_mlp_train_step");
}

}  // extern "C"

extern "C" msa_status msa_mlp_read_grad(msa_ctx *ctx, void *state, float *grad_out, void *stream) {
    if (!ctx || !state || !grad_out) return MSA_EINVAL;
    MlpState st = state_of(state);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(grad_out, st.g, kNP * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(st.g, 0, kNP * sizeof(float), s);
    return cuda_check(ctx, e, "msa_mlp_read_grad");
}
