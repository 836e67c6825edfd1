// Needleman-Wunsch with traceback (A5 fill, A6 device traceback) and the
// C entry point msa_nw_align_batch.
//
// Minimum-cost global alignment with a flat cost model (match, mismatch,
// gap): D[i][0] = i*gap, D[0][j] = j*gap,
//   D[i][j] = min(D[i-1][j-1] + cost(a_i, b_j), D[i-1][j] + gap, D[i][j-1] + gap).
// Each cell also records which move attains D[i][j], preferring diagonal,
// then up (a_i against a gap), then left (b_j against a gap); the traceback
// from (m, n) follows those codes, so it returns the same alignment as the
// plain rule "take the first of diagonal, up, left that attains D".
//
// One warp per pair (persistent, pairs pulled from an atomic counter).  Rows
// are cut into tiles of 32 lanes x 16 rows; lane l holds rows
// tile*512 + 16l + 1 .. +16 and works on column j at step j + l, taking the
// value of the row above its first row from lane l-1 by __shfl_up_sync.  The
// bottom row of a tile is kept in the warp's slab for the next tile.  The 16
// two-bit codes of a lane's rows in one column form one 32-bit word, stored
// in the warp's slab at [tile][lane][column]; lane 0 then walks back from
// (m, n) through those words and emits the edit script.
#include <cuda_runtime.h>

#include <algorithm>

#include "msa_internal.cuh"

namespace msa {

constexpr int kNwR = 16;                 // rows per lane
constexpr int kNwTile = 32 * kNwR;       // rows per tile
constexpr int kNwWarps = 4;              // warps per block

struct NwArgs {
    const uint8_t *codes;
    const int64_t *offs;
    int32_t n_seqs;
    int64_t total;
    const int32_t *pairs;
    int64_t P;
    int32_t match, mismatch, gap;
    int32_t *score;
    uint8_t *ops;
    const int64_t *ops_off;
    int32_t *ops_len;
    char *slabs;            // per-warp scratch
    int64_t slab_bytes;
    int32_t max_len;        // slab capacity in rows / columns
    int32_t *counter;
    const int32_t *plist;   // optional pair ids (count at *pcount); all pairs when null
    const int32_t *pcount;
    int32_t *err;
    const int32_t *sub;     // optional substitution costs [nsym][nsym] by code (affine kernel)
    int32_t nsym;
};

// substitution table in shared memory: stride kSubStride > kSubMax so that the
// rows a warp reads fall on different banks
constexpr int kSubMax = 32;
constexpr int kSubStride = 33;

__device__ __forceinline__ int64_t nw_tb_words(int max_len) {
    return (int64_t)((max_len + kNwTile - 1) / kNwTile) * 32 * max_len;
}

__global__ void __launch_bounds__(kNwWarps * 32) nw_kernel(NwArgs a) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kNwWarps + (threadIdx.x >> 5);
    char *slab = a.slabs + (int64_t)gw * a.slab_bytes;
    int32_t *brow = reinterpret_cast<int32_t *>(slab);
    uint32_t *tb = reinterpret_cast<uint32_t *>(slab + (((int64_t)a.max_len + 1) * 4 + 255) / 256 * 256);
    const int gap = a.gap, match = a.match, mismatch = a.mismatch;

    const int64_t count = a.plist ? (int64_t)*a.pcount : a.P;
    while (true) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(a.counter, 1);
        idx = __shfl_sync(FULL, idx, 0);
        if (idx >= count) break;
        const int p = a.plist ? a.plist[idx] : idx;
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
            for (int k = lane; k < m + n; k += 32) ops[k] = m == 0 ? 'I' : 'D';
            if (lane == 0) {
                a.score[p] = (m + n) * gap;
                a.ops_len[p] = m + n;
            }
            continue;
        }

        // ---- fill -------------------------------------------------------
        for (int j = lane; j <= n; j += 32) brow[j] = j * gap;
        __syncwarp();
        const int ntiles = (m + kNwTile - 1) / kNwTile;
        int32_t H[kNwR];
        for (int t = 0; t < ntiles; ++t) {
            const int i_first = t * kNwTile + lane * kNwR + 1;     // first row of this lane
            int ac[kNwR];
#pragma unroll
            for (int r = 0; r < kNwR; ++r) {
                const int i = i_first + r;
                ac[r] = i <= m ? (int)A[i - 1] : -1;
                H[r] = i * gap;                                      // column 0
            }
            int prev_top = (i_first - 1) * gap;                      // D[i_first-1][0]
            int last = H[kNwR - 1];
            uint32_t *tbl = tb + ((int64_t)t * 32 + lane) * n;
            for (int s = 1; s <= n + 31; ++s) {
                const int up_in = __shfl_up_sync(FULL, last, 1);
                const int j = s - lane;
                if (j >= 1 && j <= n) {
                    const int top = lane == 0 ? brow[j] : up_in;
                    const int bj = Bq[j - 1];
                    int diag = prev_top, up = top;
                    uint32_t code = 0;
#pragma unroll
                    for (int r = 0; r < kNwR; ++r) {
                        const int dg = diag + (ac[r] == bj ? match : mismatch);
                        // two-way minima with their "first argument won" flag:
                        // up <= left keeps up, then diagonal <= that keeps diagonal
                        bool up_wins, diag_wins;
                        const int m1 = __vibmin_s32(up + gap, H[r] + gap, &up_wins);
                        const int d = __vibmin_s32(dg, m1, &diag_wins);
                        const uint32_t c = diag_wins ? 0u : (up_wins ? 1u : 2u);
                        code |= c << (2 * r);
                        diag = H[r];
                        H[r] = d;
                        up = d;
                    }
                    prev_top = top;
                    last = H[kNwR - 1];
                    tbl[j - 1] = code;
                    if (lane == 31) brow[j] = last;
                }
            }
            __syncwarp();
        }
        // D[m][n]: lane holding row m, after the last column
        {
            const int lm = ((m - 1) % kNwTile) / kNwR, rm = (m - 1) % kNwR;
            if (lane == lm) {
                int v = 0;
#pragma unroll
                for (int r = 0; r < kNwR; ++r)
                    if (r == rm) v = H[r];
                a.score[p] = v;
            }
        }
        __syncwarp();

        // ---- traceback (lane 0), script written backwards from o0 + m + n - 1
        int L = 0;
        if (lane == 0) {
            int i = m, j = n;
            int64_t w = (int64_t)m + n - 1;
            while (i > 0 && j > 0) {
                const int t = (i - 1) / kNwTile, l = ((i - 1) % kNwTile) / kNwR, r = (i - 1) % kNwR;
                const uint32_t c = (tb[((int64_t)t * 32 + l) * n + (j - 1)] >> (2 * r)) & 3u;
                if (c == 0) {
                    ops[w--] = A[i - 1] == Bq[j - 1] ? 'M' : 'X';
                    --i;
                    --j;
                } else if (c == 1) {
                    ops[w--] = 'D';
                    --i;
                } else {
                    ops[w--] = 'I';
                    --j;
                }
            }
            while (i > 0) {
                ops[w--] = 'D';
                --i;
            }
            while (j > 0) {
                ops[w--] = 'I';
                --j;
            }
            L = (int)((int64_t)m + n - 1 - w);
            a.ops_len[p] = L;
        }
        L = __shfl_sync(FULL, L, 0);
        __syncwarp();
        // move the script to the front (forward order), 32 lanes, in chunks
        // that never overlap their own source
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

// ---------------------------------------------------------------------------
// Affine gap costs (Gotoh): a run of L gap positions costs open + L * ext.
// Per cell H (best), F (best ending with an up move) and E (best ending with
// a left move):
//   F[i][j] = min(F[i-1][j] + ext, H[i-1][j] + open + ext)
//   E[i][j] = min(E[i][j-1] + ext, H[i][j-1] + open + ext)
//   H[i][j] = min(H[i-1][j-1] + c(a_i, b_j), F[i][j], E[i][j])
// with H[i][0] = F[i][0] = open + i ext, H[0][j] = E[0][j] = open + j ext.
// Same layout as nw_kernel (warp per pair, 16 rows per lane, skew across
// lanes); H and F of the row above come from the lane above, E and H of the
// previous column stay in registers.  Four bits per cell: H's move (0
// diagonal, 1 F, 2 E, preferred in that order), whether F opened from H and
// whether E opened from H (opening preferred when it attains); the traceback
// runs the three-state walk from (m, n) in state H.
// ---------------------------------------------------------------------------
constexpr int32_t kNwInf = 1 << 29;

template <bool kSub>
__global__ void __launch_bounds__(kNwWarps * 32) nw_affine_kernel(NwArgs a, int32_t open, int32_t ext) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    __shared__ int32_t sSub[kSub ? kSubMax * kSubStride : 1];
    if constexpr (kSub) {
        for (int i = threadIdx.x; i < a.nsym * a.nsym; i += blockDim.x)
            sSub[(i / a.nsym) * kSubStride + i % a.nsym] = a.sub[i];
        __syncthreads();
    }
    const int gw = blockIdx.x * kNwWarps + (threadIdx.x >> 5);
    char *slab = a.slabs + (int64_t)gw * a.slab_bytes;
    int32_t *bH = reinterpret_cast<int32_t *>(slab);
    int32_t *bF = bH + (a.max_len + 1);
    uint2 *tb = reinterpret_cast<uint2 *>(slab + (((int64_t)a.max_len + 1) * 8 + 255) / 256 * 256);
    const int match = a.match, mismatch = a.mismatch;
    const int oe = open + ext;

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
        if constexpr (kSub) {
            // every code must index the table
            bool bad = false;
            for (int k = lane; k < m; k += 32) bad |= A[k] >= a.nsym;
            for (int k = lane; k < n; k += 32) bad |= Bq[k] >= a.nsym;
            if (__any_sync(FULL, bad)) {
                if (lane == 0) record_error(a.err, kErrSymbol, p, a.nsym);
                continue;
            }
        }
        if (m == 0 || n == 0) {
            for (int k = lane; k < m + n; k += 32) ops[k] = m == 0 ? 'I' : 'D';
            if (lane == 0) {
                a.score[p] = m + n > 0 ? open + (m + n) * ext : 0;
                a.ops_len[p] = m + n;
            }
            continue;
        }

        // ---- fill -------------------------------------------------------
        // row 0: H = E = open + j ext (H[0][0] = 0), F = inf
        for (int j = lane; j <= n; j += 32) {
            bH[j] = j == 0 ? 0 : open + j * ext;
            bF[j] = kNwInf;
        }
        __syncwarp();
        const int ntiles = (m + kNwTile - 1) / kNwTile;
        int32_t H[kNwR], E[kNwR];
        for (int t = 0; t < ntiles; ++t) {
            const int i_first = t * kNwTile + lane * kNwR + 1;
            int ac[kNwR];
#pragma unroll
            for (int r = 0; r < kNwR; ++r) {
                const int i = i_first + r;
                ac[r] = i <= m ? (int)A[i - 1] : -1;
                H[r] = open + i * ext;                      // column 0
                E[r] = kNwInf;
            }
            int prev_top = i_first - 1 == 0 ? 0 : open + (i_first - 1) * ext;   // H[i_first-1][0]
            int lastH = H[kNwR - 1], lastF = kNwInf;
            uint2 *tbl = tb + ((int64_t)t * 32 + lane) * n;
            for (int s = 1; s <= n + 31; ++s) {
                const int upH_in = __shfl_up_sync(FULL, lastH, 1);
                const int upF_in = __shfl_up_sync(FULL, lastF, 1);
                const int j = s - lane;
                if (j >= 1 && j <= n) {
                    const int topH = lane == 0 ? bH[j] : upH_in;
                    const int topF = lane == 0 ? bF[j] : upF_in;
                    const int bj = Bq[j - 1];
                    int diag = prev_top, upH = topH, upF = topF;
                    uint32_t c0 = 0u, c1 = 0u;
#pragma unroll
                    for (int r = 0; r < kNwR; ++r) {
                        const int fx = upF + ext, fo = upH + oe;
                        const int Fn = min(fx, fo);
                        const int ex = E[r] + ext, eo = H[r] + oe;
                        const int En = min(ex, eo);
                        // rows past m (ac = -1) read any entry: never used
                        const int dg = diag + (kSub ? sSub[(ac[r] & (kSubMax - 1)) * kSubStride + bj]
                                                    : (ac[r] == bj ? match : mismatch));
                        const int Hn = min(dg, min(Fn, En));
                        const uint32_t hs = dg == Hn ? 0u : (Fn == Hn ? 1u : 2u);
                        const uint32_t code = hs | ((uint32_t)(fo <= fx) << 2) | ((uint32_t)(eo <= ex) << 3);
                        if (r < 8) c0 |= code << (4 * r);
                        else c1 |= code << (4 * (r - 8));
                        diag = H[r];
                        H[r] = Hn;
                        E[r] = En;
                        upH = Hn;
                        upF = Fn;
                    }
                    prev_top = topH;
                    lastH = upH;
                    lastF = upF;
                    tbl[j - 1] = make_uint2(c0, c1);
                    if (lane == 31) {
                        bH[j] = lastH;
                        bF[j] = lastF;
                    }
                }
            }
            __syncwarp();
        }
        {
            const int lm = ((m - 1) % kNwTile) / kNwR, rm = (m - 1) % kNwR;
            if (lane == lm) {
                int v = 0;
#pragma unroll
                for (int r = 0; r < kNwR; ++r)
                    if (r == rm) v = H[r];
                a.score[p] = v;
            }
        }
        __syncwarp();

        // ---- traceback (lane 0): three-state walk, script written backwards
        int L = 0;
        if (lane == 0) {
            int i = m, j = n, state = 0;
            int64_t w = (int64_t)m + n - 1;
            while (i > 0 && j > 0) {
                const int t = (i - 1) / kNwTile, l = ((i - 1) % kNwTile) / kNwR, r = (i - 1) % kNwR;
                const uint2 cw = tb[((int64_t)t * 32 + l) * n + (j - 1)];
                const uint32_t c = ((r < 8 ? cw.x : cw.y) >> (4 * (r & 7))) & 15u;
                if (state == 0) {
                    const uint32_t hs = c & 3u;
                    if (hs == 0u) {
                        ops[w--] = A[i - 1] == Bq[j - 1] ? 'M' : 'X';
                        --i;
                        --j;
                    } else {
                        state = hs == 1u ? 1 : 2;
                    }
                } else if (state == 1) {
                    ops[w--] = 'D';
                    if (c & 4u) state = 0;
                    --i;
                } else {
                    ops[w--] = 'I';
                    if (c & 8u) state = 0;
                    --j;
                }
            }
            while (i > 0) {
                ops[w--] = 'D';
                --i;
            }
            while (j > 0) {
                ops[w--] = 'I';
                --j;
            }
            L = (int)((int64_t)m + n - 1 - w);
            a.ops_len[p] = L;
        }
        L = __shfl_sync(FULL, L, 0);
        __syncwarp();
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

int64_t nw_affine_slab_bytes(int max_len) {
    const int64_t brow = (((int64_t)max_len + 1) * 8 + 255) / 256 * 256;
    const int64_t tiles = (max_len + kNwTile - 1) / kNwTile;
    const int64_t tbw = tiles * 32 * (int64_t)std::max(max_len, 1) * 8;
    return brow + (tbw + 255) / 256 * 256;
}

msa_status nw_affine_run(msa_ctx *ctx, Arena &ar, const uint8_t *codes, const int64_t *offs, int32_t n_seqs,
                         int64_t total, int32_t max_len, const int32_t *pairs, int64_t P, int32_t match,
                         int32_t mismatch, int32_t open, int32_t ext, int32_t *score_out, uint8_t *ops_out,
                         const int64_t *ops_off, int32_t *ops_len_out, cudaStream_t st, const int32_t *sub,
                         int32_t nsym) {
    if (sub && (nsym < 1 || nsym > kSubMax))
        return set_error(ctx, MSA_EINVAL, "msa_nw_align_batch_affine_sub: table size %d outside 1..%d", nsym, kSubMax);
    if (P < 0 || P >= (int64_t(1) << 31) || n_seqs < 0 || max_len < 0 || total < 0)
        return set_error(ctx, MSA_EINVAL, "msa_nw_align_batch_affine: negative or oversized count");
    if (open < 0 || ext < 1)
        return set_error(ctx, MSA_EINVAL, "msa_nw_align_batch_affine: needs gap_open >= 0 and gap_ext >= 1");
    if (P == 0) return MSA_OK;
    if (!codes || !offs || !pairs || !score_out || !ops_out || !ops_off || !ops_len_out)
        return set_error(ctx, MSA_EINVAL, "msa_nw_align_batch_affine: null pointer");
    const void *fn = sub ? (const void *)nw_affine_kernel<true> : (const void *)nw_affine_kernel<false>;
    int occ = 1;
    if (msa_status rc = occupancy(ctx, fn, kNwWarps * 32, 0, &occ)) return rc;
    int32_t *counter = ar.take<int32_t>(64);
    const int64_t slab = nw_affine_slab_bytes(max_len);
    const int64_t avail = counter ? ar.cap - ar.used : 0;
    int64_t warps = std::min<int64_t>((int64_t)ctx->sm_count * occ * kNwWarps, avail / slab);
    warps = std::min<int64_t>(warps, ((P + kNwWarps - 1) / kNwWarps) * kNwWarps);
    warps = warps / kNwWarps * kNwWarps;
    if (warps < kNwWarps)
        return set_error(ctx, MSA_ENOMEM,
                         "msa_nw_align_batch_affine: max_len %d needs %lld workspace bytes per warp group", max_len,
                         (long long)(slab * kNwWarps + 256));
    char *slabs = ar.take<char>(warps * slab);
    cudaError_t e = cudaMemsetAsync(counter, 0, 4, st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "nw memset");
    NwArgs a{codes, offs, n_seqs, total, pairs, P, match, mismatch, 0, score_out, ops_out, ops_off,
             ops_len_out, slabs, slab, max_len, counter, nullptr, nullptr, ctx->dev_err, sub, nsym};
    ProfScope prof(ctx, st);
    if (sub)
        nw_affine_kernel<true><<<(int)(warps / kNwWarps), kNwWarps * 32, 0, st>>>(a, open, ext);
    else
        nw_affine_kernel<false><<<(int)(warps / kNwWarps), kNwWarps * 32, 0, st>>>(a, open, ext);
    ++ctx->launches;
    return cuda_check(ctx, cudaGetLastError(), "nw affine launch");
}

// Per-warp scratch, large enough for either kernel (the bit-parallel one for
// the unit cost model, the plain DP for the rest); the two run one after the
// other on the same slabs.
int64_t nw_slab_bytes(int max_len) {
    const int64_t brow = (((int64_t)max_len + 1) * 4 + 255) / 256 * 256;
    const int64_t tiles = (max_len + kNwTile - 1) / kNwTile;
    const int64_t tbw = tiles * 32 * (int64_t)std::max(max_len, 1) * 4;
    return std::max(brow + (tbw + 255) / 256 * 256, nw_bv_slab_bytes(max_len));
}

msa_status nw_run(msa_ctx *ctx, Arena &ar, const uint8_t *codes, const int64_t *offs, int32_t n_seqs, int64_t total,
                  int32_t max_len, const int32_t *pairs, int64_t P, int32_t match, int32_t mismatch, int32_t gap,
                  int32_t *score_out, uint8_t *ops_out, const int64_t *ops_off, int32_t *ops_len_out,
                  cudaStream_t st) {
    if (P < 0 || P >= (int64_t(1) << 31) || n_seqs < 0 || max_len < 0 || total < 0)
        return set_error(ctx, MSA_EINVAL, "msa_nw_align_batch: negative or oversized count");
    if (P == 0) return MSA_OK;
    if (!codes || !offs || !pairs || !score_out || !ops_out || !ops_off || !ops_len_out)
        return set_error(ctx, MSA_EINVAL, "msa_nw_align_batch: null pointer");
    int occ = 1, occ_bv = 1;
    if (msa_status rc = occupancy(ctx, (const void *)nw_kernel, kNwWarps * 32, 0, &occ)) return rc;
    if (msa_status rc = occupancy(ctx, nw_bv_kernel_fn(), kBvThreads, 0, &occ_bv)) return rc;
    // unit costs (match 0, mismatch = gap > 0): the bit-parallel kernel, with
    // the plain DP for the pairs it hands back
    const bool unit = match == 0 && mismatch == gap && gap > 0;
    int32_t *counter = ar.take<int32_t>(64);
    int32_t *fb_list = unit ? ar.take<int32_t>(P) : nullptr;
    const int64_t slab = nw_slab_bytes(max_len);
    const int64_t avail = counter && (!unit || fb_list) ? ar.cap - ar.used : 0;
    const int64_t want = (int64_t)ctx->sm_count * std::max(occ, unit ? occ_bv : 0) * kNwWarps;
    int64_t warps = std::min<int64_t>(want, avail / slab);
    warps = std::min<int64_t>(warps, ((P + kNwWarps - 1) / kNwWarps) * kNwWarps);
    warps = warps / kNwWarps * kNwWarps;
    if (warps < kNwWarps)
        return set_error(ctx, MSA_ENOMEM, "msa_nw_align_batch: max_len %d needs %lld workspace bytes per warp group",
                         max_len, (long long)(slab * kNwWarps + 256 + (unit ? 4 * P : 0)));
    char *slabs = ar.take<char>(warps * slab);
    cudaError_t e = cudaMemsetAsync(counter, 0, 4 * 64, st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "nw memset");
    ProfScope prof(ctx, st);
    NwArgs a{codes, offs, n_seqs, total, pairs, P, match, mismatch, gap, score_out, ops_out, ops_off,
             ops_len_out, slabs, slab, max_len, counter, nullptr, nullptr, ctx->dev_err};
    if (unit) {
        const int64_t wbv = std::min<int64_t>(warps, (int64_t)ctx->sm_count * occ_bv * kNwWarps) / kNwWarps * kNwWarps;
        e = nw_bv_launch(ctx, codes, offs, n_seqs, total, max_len, pairs, P, gap, score_out, ops_out, ops_off,
                         ops_len_out, slabs, slab, std::max<int64_t>(wbv, kNwWarps), counter, fb_list, counter + 32, st);
        if (e != cudaSuccess) return cuda_check(ctx, e, "nw launch");
        a.counter = counter + 1;
        a.plist = fb_list;
        a.pcount = counter + 32;
    }
    const int64_t wdp = std::min<int64_t>(warps, (int64_t)ctx->sm_count * occ * kNwWarps) / kNwWarps * kNwWarps;
    nw_kernel<<<(int)(std::max<int64_t>(wdp, kNwWarps) / kNwWarps), kNwWarps * 32, 0, st>>>(a);
    ++ctx->launches;
    return cuda_check(ctx, cudaGetLastError(), "nw launch");
}

}  // namespace msa

using namespace msa;

extern "C" {

int64_t msa_nw_workspace_bytes(int32_t max_len, int32_t warps) {
    return 256 + (int64_t)warps * nw_slab_bytes(max_len);
}

msa_status msa_nw_align_batch_affine(msa_ctx *ctx, const uint8_t *codes, const int64_t *offs, int32_t n_seqs,
                                     int64_t total, int32_t max_len, const int32_t *pairs, int64_t P, int32_t match,
                                     int32_t mismatch, int32_t gap_open, int32_t gap_ext, int32_t *score_out,
                                     uint8_t *ops_out, const int64_t *ops_off, int32_t *ops_len_out, void *stream) {
    if (!ctx) return MSA_EINVAL;
    Arena ar{ctx->ws, ctx->ws_bytes};
    return nw_affine_run(ctx, ar, codes, offs, n_seqs, total, max_len, pairs, P, match, mismatch, gap_open, gap_ext,
                         score_out, ops_out, ops_off, ops_len_out, (cudaStream_t)stream);
}

msa_status msa_nw_align_batch_affine_sub(msa_ctx *ctx, const uint8_t *codes, const int64_t *offs, int32_t n_seqs,
                                         int64_t total, int32_t max_len, const int32_t *pairs, int64_t P,
                                         const int32_t *sub, int32_t nsym, int32_t gap_open, int32_t gap_ext,
                                         int32_t *score_out, uint8_t *ops_out, const int64_t *ops_off,
                                         int32_t *ops_len_out, void *stream) {
    if (!ctx) return MSA_EINVAL;
    if (!sub) return set_error(ctx, MSA_EINVAL, "msa_nw_align_batch_affine_sub: null table");
    Arena ar{ctx->ws, ctx->ws_bytes};
    return nw_affine_run(ctx, ar, codes, offs, n_seqs, total, max_len, pairs, P, 0, 0, gap_open, gap_ext, score_out,
                         ops_out, ops_off, ops_len_out, (cudaStream_t)stream, sub, nsym);
}

msa_status msa_nw_align_batch(msa_ctx *ctx, const uint8_t *codes, const int64_t *offs, int32_t n_seqs,
                              int64_t total, int32_t max_len, const int32_t *pairs, int64_t P, int32_t match,
                              int32_t mismatch, int32_t gap, int32_t *score_out, uint8_t *ops_out,
                              const int64_t *ops_off, int32_t *ops_len_out, void *stream) {
    if (!ctx) return MSA_EINVAL;
    Arena ar{ctx->ws, ctx->ws_bytes};
    return nw_run(ctx, ar, codes, offs, n_seqs, total, max_len, pairs, P, match, mismatch, gap, score_out, ops_out,
                  ops_off, ops_len_out, (cudaStream_t)stream);
}

}  // extern "C"
