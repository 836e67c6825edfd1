// Bit-parallel Needleman-Wunsch with traceback for the unit cost model
// (match 0, mismatch = gap > 0), the model of the merges (A5 fill, A6
// traceback): with these costs D[i][j] / gap is the edit distance, so the
// column recurrence of the Levenshtein kernels computes the fill 32 rows per
// integer operation, and the moves of the traceback follow from bit vectors
// that recurrence already forms.  With D0 the rows where
// D[i][j] = D[i-1][j-1] (Hyyro: D0 = (((Eq & Pv) + Pv) ^ Pv) | Eq | Mv of the
// previous column):
//   diagonal attains D[i][j]  iff  a_i = b_j, or D[i][j] = D[i-1][j-1] + 1,
//                             iff  (Eq | ~D0)[i];
//   up attains D[i][j]        iff  D[i][j] = D[i-1][j] + 1  iff  Pv[i] of column j;
//   otherwise left attains it.
// So one 2-bit move per cell, (Eq | ~D0, Pv), is written per column with the
// same preference as the plain DP (diagonal, then up, then left), and the
// walk back from (m, n) reproduces its edit script exactly.
//
// One warp per pair (persistent, pairs pulled from an atomic counter).  Rows
// are cut into tiles of 32 lanes x kBvWpl words (2,048 rows); lane l holds
// words l*kBvWpl .. of the tile and works on column j at step j + l, taking
// the Ph bit and the carry (= Mh bit) of the row above from lane l - 1 by
// __shfl_up_sync, and lane 31 leaves them per column for the next tile.  The
// match masks are built per pair over the distinct bytes of a (at most 32;
// pairs with more go to the plain DP kernel), in shared memory [word][symbol]
// [lane].  Moves are stored per warp at [tile][step][lane][word] (2 bits a
// cell), laid out by pipeline step so that every step's stores coalesce.
// The traceback runs on the whole warp: the lanes load the moves of
// 64 columns x 96 rows around the current cell, and the walk reads them by
// shuffles until it leaves that window.
#include <cuda_runtime.h>

#include "carry_chain.cuh"
#include "msa_internal.cuh"

namespace msa {

constexpr int kBvWpl = 2;                    // words per lane
constexpr int kBvTileWords = 32 * kBvWpl;    // words per tile
constexpr int kBvTileRows = 32 * kBvTileWords;
constexpr int kBvWarps = 4;
static_assert(kBvWarps * 32 == kBvThreads, "nw_bv_kernel block size");
constexpr uint32_t kBvFull = 0xffffffffu;

// Two columns per pipeline step: lane l computes columns 2q - 1 and 2q at
// step q + l, so the shuffle and the loop are paid once per two columns.
// Moves of one pair: uint2 {diagonal plane, up plane} per (tile, step, lane,
// column of the step, word): the 32 lanes of one step write one contiguous
// 1 KB run.
__host__ __device__ inline int64_t nw_bv_steps(int max_len) { return ((int64_t)max_len + 1) / 2 + 32; }
__host__ __device__ inline int64_t nw_bv_move_bytes(int max_len) {
    const int64_t tiles = (max_len + kBvTileRows - 1) / kBvTileRows;
    return tiles * nw_bv_steps(max_len) * 32 * 2 * kBvWpl * 8;
}
// index (in uint2) of the moves of word W (over all rows) at column j >= 1
__device__ __forceinline__ int64_t nw_bv_move_index(int W, int j, int max_len) {
    const int T = W / kBvTileWords, L = (W % kBvTileWords) / kBvWpl, w = W % kBvWpl;
    const int q = (j + 1) >> 1, c = (j - 1) & 1;
    return ((T * nw_bv_steps(max_len) + q + L) * 32 + L) * (2 * kBvWpl) + c * kBvWpl + w;
}

// One column over the lane's words; returns the Ph bit and carry sent down
// and writes the column's move planes.
__device__ __forceinline__ uint32_t nw_bv_column(const uint32_t (&eq)[kBvWpl], uint32_t (&Pv)[kBvWpl],
                                                 uint32_t (&Mv)[kBvWpl], uint32_t bits, uint2 *dst) {
    const uint32_t ph_in = bits & 1u, cin = (bits >> 1) & 1u;
    uint32_t u[kBvWpl], sum[kBvWpl], pv[kBvWpl];
#pragma unroll
    for (int w = 0; w < kBvWpl; ++w) {
        pv[w] = Pv[w];
        u[w] = eq[w] & pv[w];
    }
    const uint32_t cout = CarryChainIn<kBvWpl>::add(sum, u, pv, cin);
    uint32_t php = ph_in << 31;
    uint2 mvw[kBvWpl];
#pragma unroll
    for (int w = 0; w < kBvWpl; ++w) {
        const uint32_t mhs = sum[w] ^ u[w] ^ pv[w];
        const uint32_t ph = Mv[w] | ~(sum[w] | pv[w] | eq[w]);
        const uint32_t phs = __funnelshift_l(php, ph, 1);
        php = ph;
        const uint32_t xv = eq[w] | Mv[w];
        const uint32_t diag = eq[w] | ~((sum[w] ^ pv[w]) | Mv[w]);
        Pv[w] = mhs | ~(xv | phs);
        Mv[w] = phs & xv;
        mvw[w] = make_uint2(diag, Pv[w]);
    }
#pragma unroll
    for (int w = 0; w < kBvWpl; ++w) dst[w] = mvw[w];
    return (php >> 31) | (cout << 1);
}

struct NwBvArgs {
    const uint8_t *codes;
    const int64_t *offs;
    int32_t n_seqs;
    int64_t total;
    const int32_t *pairs;
    int64_t P;
    int32_t gap;
    int32_t *score;
    uint8_t *ops;
    const int64_t *ops_off;
    int32_t *ops_len;
    char *slabs;            // per-warp scratch
    int64_t slab_bytes;
    int32_t max_len;
    int32_t *counter;
    int32_t *fb_list;       // pairs left to the plain DP (more than 32 distinct bytes in a)
    int32_t *fb_count;
    int32_t *err;
};

__global__ void __launch_bounds__(kBvWarps * 32) nw_bv_kernel(NwBvArgs a) {
    const unsigned FULL = 0xffffffffu;
    __shared__ uint32_t sPeq[kBvWarps][kBvWpl][32][32];
    __shared__ uint8_t sLut[kBvWarps][256];
    __shared__ uint32_t sSeen[kBvWarps][8];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int gw = blockIdx.x * kBvWarps + wid;
    char *slab = a.slabs + (int64_t)gw * a.slab_bytes;
    uint8_t *brow = reinterpret_cast<uint8_t *>(slab);
    uint2 *moves = reinterpret_cast<uint2 *>(slab + ((int64_t)a.max_len + 1 + 255) / 256 * 256);
    uint8_t *lut = sLut[wid];
    uint32_t *seen = sSeen[wid];

    while (true) {
        int p = 0;
        if (lane == 0) p = atomicAdd(a.counter, 1);
        p = __shfl_sync(FULL, p, 0);
        if (p >= a.P) break;
        const int x = a.pairs[2 * p], y = a.pairs[2 * p + 1];
        bool ok = x >= 0 && x < a.n_seqs && y >= 0 && y < a.n_seqs;
        int64_t xa = 0, xb = 0, ya = 0, yb = 0;
        if (ok) {
            xa = a.offs[x], xb = a.offs[x + 1], ya = a.offs[y], yb = a.offs[y + 1];
            ok = xa >= 0 && xa <= xb && xb <= a.total && ya >= 0 && ya <= yb && yb <= a.total;
        }
        if (!ok) {
            if (lane == 0) record_error(a.err, kErrIndex, p, x);
            continue;
        }
        const int m = (int)(xb - xa), n = (int)(yb - ya);
        const uint8_t *A = a.codes + xa;
        const uint8_t *Bq = a.codes + ya;
        const int64_t o0 = a.ops_off[p];
        if (a.ops_off[p + 1] - o0 < (int64_t)m + n) {
            if (lane == 0) record_error(a.err, kErrCapacity, p, m + n);
            continue;
        }
        if (m > a.max_len || n > a.max_len) {
            if (lane == 0) record_error(a.err, kErrLength, p, max(m, n));
            continue;
        }
        uint8_t *ops = a.ops + o0;
        if (m == 0 || n == 0) {
            for (int k = lane; k < m + n; k += 32) ops[k] = m == 0 ? MSA_OP_INS : MSA_OP_DEL;
            if (lane == 0) {
                a.score[p] = (m + n) * a.gap;
                a.ops_len[p] = m + n;
            }
            continue;
        }

        // ---- alphabet of a: distinct bytes -> match-mask index -------------
        if (lane < 8) seen[lane] = 0u;
        __syncwarp();
        for (int k = lane; k < m; k += 32) atomicOr(&seen[A[k] >> 5], 1u << (A[k] & 31));
        __syncwarp();
        int distinct = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) distinct += __popc(seen[w]);
        if (distinct > 32) {
            if (lane == 0) a.fb_list[atomicAdd(a.fb_count, 1)] = p;
            continue;
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int v = lane * 8 + t, w = v >> 5, bit = v & 31;
            int below = __popc(seen[w] & ((1u << bit) - 1u));
            for (int u = 0; u < w; ++u) below += __popc(seen[u]);
            lut[v] = ((seen[w] >> bit) & 1u) ? (uint8_t)below : (uint8_t)0xFF;
        }
        __syncwarp();

        // ---- fill, tile by tile -------------------------------------------
        const int ntiles = (m + kBvTileRows - 1) / kBvTileRows;
        int part = 0;                       // this lane's vertical deltas at column n, rows <= m
        for (int t = 0; t < ntiles; ++t) {
            const int row0 = t * kBvTileRows + lane * kBvWpl * 32;   // rows row0 + 1 ..
#pragma unroll
            for (int w = 0; w < kBvWpl; ++w)
                for (int c = 0; c < 32; ++c) sPeq[wid][w][c][lane] = 0u;
            uint32_t maskw[kBvWpl];
#pragma unroll
            for (int w = 0; w < kBvWpl; ++w) {
                const int rem = m - (row0 + 32 * w);
                maskw[w] = rem >= 32 ? kBvFull : (rem <= 0 ? 0u : ((1u << rem) - 1u));
                // the word's 32 row bytes are loaded first, all at once
                int ab[32];
#pragma unroll
                for (int r = 0; r < 32; ++r) ab[r] = r < rem ? (int)__ldg(A + row0 + 32 * w + r) : -1;
#pragma unroll
                for (int r = 0; r < 32; ++r)
                    if (ab[r] >= 0) sPeq[wid][w][lut[ab[r]]][lane] |= 1u << r;
            }
            __syncwarp();
            uint32_t Pv[kBvWpl], Mv[kBvWpl];
#pragma unroll
            for (int w = 0; w < kBvWpl; ++w) {
                Pv[w] = kBvFull;
                Mv[w] = 0u;
            }
            uint2 *mv_tile = moves + (int64_t)t * nw_bv_steps(a.max_len) * 32 * 2 * kBvWpl;
            // lanes whose rows all lie past m feed nobody: they idle
            const bool live = row0 < m;
            // masks of the next step's two columns are read one step ahead
            // (their bytes two steps ahead), off the carry chain's critical path
            auto masks = [&](int byte, uint32_t (&e)[kBvWpl]) {
                const int ci = lut[byte];
#pragma unroll
                for (int w = 0; w < kBvWpl; ++w) {
                    const uint32_t v = sPeq[wid][w][ci & 31][lane];     // index kept in range
                    e[w] = ci == 0xFF ? 0u : v;
                }
            };
            uint32_t eqA[kBvWpl], eqB[kBvWpl];
            masks(Bq[0], eqA);
            masks(n > 1 ? (int)Bq[1] : 0, eqB);
            int bA = n > 2 ? (int)__ldg(Bq + 2) : 0, bB = n > 3 ? (int)__ldg(Bq + 3) : 0;
            const int nq = (n + 1) / 2;
            uint32_t out = 0u;
            for (int s = 1; s <= nq + 31; ++s) {
                const uint32_t in = __shfl_up_sync(FULL, out, 1);
                const int q = s - lane;
                if (live && q >= 1 && q <= nq) {
                    const int j1 = 2 * q - 1, j2 = 2 * q;          // j2 may be n + 1: computed, never read
                    uint32_t bits = in;
                    if (lane == 0) bits = t == 0 ? 5u : ((uint32_t)brow[j1] | (j2 <= n ? (uint32_t)brow[j2] << 2 : 0u));
                    uint32_t e1[kBvWpl], e2[kBvWpl];
#pragma unroll
                    for (int w = 0; w < kBvWpl; ++w) {
                        e1[w] = eqA[w];
                        e2[w] = eqB[w];
                    }
                    if (q < nq) {
                        masks(bA, eqA);
                        masks(bB, eqB);
                        bA = j2 + 2 < n ? (int)__ldg(Bq + j2 + 2) : 0;
                        bB = j2 + 3 < n ? (int)__ldg(Bq + j2 + 3) : 0;
                    }
                    uint2 *dst = mv_tile + ((int64_t)s * 32 + lane) * (2 * kBvWpl);   // s = q + lane
                    const uint32_t o1 = nw_bv_column(e1, Pv, Mv, bits, dst);
                    if (j1 == n) {
#pragma unroll
                        for (int w = 0; w < kBvWpl; ++w) part += __popc(Pv[w] & maskw[w]) - __popc(Mv[w] & maskw[w]);
                    }
                    const uint32_t o2 = nw_bv_column(e2, Pv, Mv, bits >> 2, dst + kBvWpl);
                    if (j2 == n) {
#pragma unroll
                        for (int w = 0; w < kBvWpl; ++w) part += __popc(Pv[w] & maskw[w]) - __popc(Mv[w] & maskw[w]);
                    }
                    out = o1 | (o2 << 2);
                    if (lane == 31) {
                        brow[j1] = (uint8_t)o1;
                        if (j2 <= n) brow[j2] = (uint8_t)o2;
                    }
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
        if (lane == 0) a.score[p] = (n + part) * a.gap;

        // ---- traceback on the whole warp -------------------------------------
        // script written backwards from o0 + m + n - 1
        int i = m, j = n;
        int64_t wpos = (int64_t)m + n - 1;
        while (i > 0 && j > 0) {
            // window: columns jb - 63 .. jb (lane k holds jb - k and jb - 32 - k)
            // and rows rl .. ib (the words Wi - 2 .. Wi)
            const int jb = j, ib = i;
            const int Wi = (ib - 1) >> 5;
            const int rl = Wi >= 2 ? 32 * (Wi - 2) + 1 : 1;
            uint2 c00 = make_uint2(0u, 0u), c01 = c00, c02 = c00, c10 = c00, c11 = c00, c12 = c00;
            int bw0 = 0, bw1 = 0;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int jc = jb - 32 * hh - lane;
                if (jc >= 1) {
                    uint2 v[3];
#pragma unroll
                    for (int ww = 0; ww < 3; ++ww) {
                        const int W = Wi - ww;
                        v[ww] = make_uint2(0u, 0u);
                        if (W >= 0) v[ww] = moves[nw_bv_move_index(W, jc, a.max_len)];
                    }
                    const int bv = (int)Bq[jc - 1];
                    if (hh == 0) {
                        c00 = v[0]; c01 = v[1]; c02 = v[2]; bw0 = bv;
                    } else {
                        c10 = v[0]; c11 = v[1]; c12 = v[2]; bw1 = bv;
                    }
                }
            }
            int aw0 = 0, aw1 = 0, aw2 = 0;
            {
                const int r0 = rl - 1 + lane, r1 = r0 + 32, r2 = r0 + 64;
                if (r0 < m) aw0 = (int)A[r0];
                if (r1 < m) aw1 = (int)A[r1];
                if (r2 < m) aw2 = (int)A[r2];
            }
            while (i > 0 && j > 0 && j > jb - 64 && i >= rl) {
                const int k = jb - j, kl = k & 31;
                const bool h1 = k >= 32;
                const int ww = Wi - ((i - 1) >> 5);
                const uint2 cw = ww == 0 ? (h1 ? c10 : c00) : (ww == 1 ? (h1 ? c11 : c01) : (h1 ? c12 : c02));
                const uint32_t dpl = __shfl_sync(FULL, cw.x, kl);
                const uint32_t upl = __shfl_sync(FULL, cw.y, kl);
                const int bit = (i - 1) & 31;
                uint8_t op;
                if ((dpl >> bit) & 1u) {
                    const int o = i - rl;
                    const int ao = o < 32 ? aw0 : (o < 64 ? aw1 : aw2);
                    const int av = __shfl_sync(FULL, ao, o & 31);
                    const int bv = __shfl_sync(FULL, h1 ? bw1 : bw0, kl);
                    op = av == bv ? MSA_OP_MATCH : MSA_OP_MISMATCH;
                    --i;
                    --j;
                } else if ((upl >> bit) & 1u) {
                    op = MSA_OP_DEL;
                    --i;
                } else {
                    op = MSA_OP_INS;
                    --j;
                }
                if (lane == 0) ops[wpos] = op;
                --wpos;
            }
        }
        for (int k = lane; k < i; k += 32) ops[wpos - k] = MSA_OP_DEL;
        wpos -= i;
        for (int k = lane; k < j; k += 32) ops[wpos - k] = MSA_OP_INS;
        wpos -= j;
        const int L = (int)((int64_t)m + n - 1 - wpos);
        if (lane == 0) a.ops_len[p] = L;
        __syncwarp();
        // move the script to the front (forward order), in chunks that never
        // overlap their own source
        const int shift = m + n - L;
        if (shift > 0) {
            for (int base = 0; base < L; base += 32) {
                const int k = base + lane;
                uint8_t v = 0;
                if (k < L) v = ops[shift + k];
                __syncwarp();
                if (k < L) ops[k] = v;
                __syncwarp();
            }
        }
    }
}

int64_t nw_bv_slab_bytes(int max_len) {
    return ((int64_t)max_len + 1 + 255) / 256 * 256 + (nw_bv_move_bytes(max_len) + 255) / 256 * 256;
}

cudaError_t nw_bv_launch(msa_ctx *ctx, const uint8_t *codes, const int64_t *offs, int32_t n_seqs, int64_t total,
                         int32_t max_len, const int32_t *pairs, int64_t P, int32_t gap, int32_t *score,
                         uint8_t *ops, const int64_t *ops_off, int32_t *ops_len, char *slabs, int64_t slab_bytes,
                         int64_t warps, int32_t *counter, int32_t *fb_list, int32_t *fb_count, cudaStream_t st) {
    NwBvArgs a{codes, offs, n_seqs, total, pairs, P, gap, score, ops, ops_off, ops_len, slabs, slab_bytes, max_len,
               counter, fb_list, fb_count, ctx->dev_err};
    nw_bv_kernel<<<(int)(warps / kBvWarps), kBvWarps * 32, 0, st>>>(a);
    ++ctx->launches;
    return cudaGetLastError();
}

const void *nw_bv_kernel_fn() { return (const void *)nw_bv_kernel; }

}  // namespace msa
