// Needleman-Wunsch split at k-mer anchors (the paper names splitting long
// alignments at k-mer anchors as future work for length scaling, section
// "Discussion and Future Work", without fixing a method -- the steps below
// are this library's definition):
//   1. anchors: every (i, j) where the k-mer a[i .. i+k) occurs exactly once
//      in a and exactly once in b, and b[j .. j+k) is that k-mer;
//   2. chain: the longest chain of anchors increasing in i and j, by patience
//      sorting over the anchors in i order (each anchor replaces the first
//      tail whose j is >= its own and links to the tail before it; the chain
//      is read back from the last tail);
//   3. blocks, left to right over the chain: an anchor on the current
//      block's diagonal that starts inside or right after it extends the
//      block to its own end, one that starts at or after the block's end in
//      both sequences starts a new block, any other is dropped;
//   4. each block is aligned as a run of matches and every segment between
//      blocks (and before the first and after the last) by the library's NW
//      (msa_nw_align_batch's costs and tie-break); the scripts are joined.
// The cost is an upper bound of the optimal NW cost, equal to it when an
// optimal alignment passes through every block.
//
// Device steps: anchor_chain_kernel (one block per pair: a hash table of
// a's k-mers with occurrence counts in both sequences, the anchors marked by
// their i, the chain and the blocks by one thread), scans of the segment
// counts and bytes, one read-back of the two totals, seg_build_kernel (the
// segments' bytes into an arena of their own), nw_run on the segments, and
// assemble_kernel (one warp per pair joins the scripts and adds the costs).
#include <cuda_runtime.h>

#include <algorithm>

#include "msa_internal.cuh"

namespace msa {

constexpr int kAnchorThreads = 256;
constexpr int kMaxK = 256;

// One distinct k-mer of a: rep is the position in a of the occurrence that
// claimed the slot (-1 = empty); k-mers are compared byte by byte, so any
// byte values and any k up to kMaxK work.
struct KmerSlot {
    int32_t rep;
    int32_t ca, cb;     // occurrences in a, in b
    int32_t pa, pb;     // a position in a, in b (the only one when the count is 1)
};

struct AnchorArgs {
    const uint8_t *codes;
    const int64_t *offs;
    int32_t n_seqs;
    int64_t total;
    const int32_t *pairs;
    int32_t P;
    int32_t k;
    int32_t match;
    int32_t max_len;
    int32_t tbits;            // log2 of the table size (>= 2 max_len entries)
    char *slabs;              // per-block scratch
    int64_t slab_bytes;
    int3 *blocks;             // [P][bcap]: start in a, start in b, length
    int32_t bcap;
    int32_t *nblocks;         // [P]
    int32_t *seg_count;       // [P] segments (blocks + 1)
    int64_t *seg_bytes;       // [P] bytes outside the blocks (m + n - 2 sum of lengths)
    int32_t *counter;         // [0] pair claims, [1] longest segment
    int32_t *err;
};

// Multiplicative hash of the k bytes at s (a polynomial in an odd 64-bit
// base, then Fibonacci hashing to tbits bits).
__device__ __forceinline__ uint32_t kmer_hash(const uint8_t *s, int k, int tbits) {
    unsigned long long h = 0;
    for (int t = 0; t < k; ++t) h = h * 0x100000001B3ull + (unsigned long long)s[t] + 1ull;
    return (uint32_t)((h * 0x9E3779B97F4A7C15ull) >> (64 - tbits));
}

__device__ __forceinline__ bool same_kmer(const uint8_t *x, const uint8_t *y, int k) {
    for (int t = 0; t < k; ++t)
        if (x[t] != y[t]) return false;
    return true;
}

__global__ void __launch_bounds__(kAnchorThreads) anchor_chain_kernel(AnchorArgs a) {
    __shared__ int32_t s_pair;
    char *slab = a.slabs + (int64_t)blockIdx.x * a.slab_bytes;
    const int64_t tsize = int64_t(1) << a.tbits;
    KmerSlot *table = reinterpret_cast<KmerSlot *>(slab);
    int32_t *aj = reinterpret_cast<int32_t *>(slab + tsize * sizeof(KmerSlot));
    int32_t *tails = aj + a.max_len;
    int32_t *tidx = tails + a.max_len;
    int32_t *prev = tidx + a.max_len;
    const int k = a.k;
    while (true) {
        if (threadIdx.x == 0) s_pair = atomicAdd(a.counter, 1);
        __syncthreads();
        const int p = s_pair;
        __syncthreads();
        if (p >= a.P) break;
        const int x = a.pairs[2 * p], y = a.pairs[2 * p + 1];
        bool ok = x >= 0 && x < a.n_seqs && y >= 0 && y < a.n_seqs;
        int64_t xa = 0, xb = 0, ya = 0, yb = 0;
        if (ok) {
            xa = a.offs[x], xb = a.offs[x + 1], ya = a.offs[y], yb = a.offs[y + 1];
            ok = xa >= 0 && xa <= xb && xb <= a.total && ya >= 0 && ya <= yb && yb <= a.total;
        }
        const int m = ok ? (int)(xb - xa) : 0, n = ok ? (int)(yb - ya) : 0;
        if (ok && (m > a.max_len || n > a.max_len)) ok = false;
        if (!ok) {
            if (threadIdx.x == 0) {
                record_error(a.err, kErrIndex, p, x);
                a.nblocks[p] = 0;
                a.seg_count[p] = 0;
                a.seg_bytes[p] = 0;
            }
            continue;
        }
        const uint8_t *A = a.codes + xa, *B = a.codes + ya;
        // the table of a's k-mers, sized to at least twice their number
        int tb = 4;
        while ((int64_t(1) << tb) < 2 * (int64_t)max(m, 1)) ++tb;
        const uint32_t tmask = (1u << tb) - 1u;
        for (int64_t t = threadIdx.x; t < (int64_t(1) << tb); t += blockDim.x) {
            table[t].rep = -1;
            table[t].ca = table[t].cb = 0;
        }
        for (int i = threadIdx.x; i < m; i += blockDim.x) aj[i] = -1;
        __syncthreads();
        for (int i = threadIdx.x; i + k <= m; i += blockDim.x) {
            uint32_t h = kmer_hash(A + i, k, tb);
            while (true) {
                const int old = atomicCAS(&table[h].rep, -1, i);
                if (old < 0 || same_kmer(A + old, A + i, k)) break;
                h = (h + 1) & tmask;
            }
            atomicAdd(&table[h].ca, 1);
            table[h].pa = i;
        }
        __syncthreads();
        for (int j = threadIdx.x; j + k <= n; j += blockDim.x) {
            uint32_t h = kmer_hash(B + j, k, tb);
            while (true) {
                const int cur = table[h].rep;
                if (cur < 0) break;                // not in a: never an anchor
                if (same_kmer(A + cur, B + j, k)) {
                    atomicAdd(&table[h].cb, 1);
                    table[h].pb = j;
                    break;
                }
                h = (h + 1) & tmask;
            }
        }
        __syncthreads();
        for (int64_t t = threadIdx.x; t < (int64_t(1) << tb); t += blockDim.x)
            if (table[t].ca == 1 && table[t].cb == 1) aj[table[t].pa] = table[t].pb;
        __syncthreads();
        // chain and blocks: one thread
        if (threadIdx.x == 0) {
            int len = 0;
            for (int i = 0; i < m; ++i) {
                const int j = aj[i];
                if (j < 0) continue;
                int lo = 0, hi = len;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (tails[mid] < j) lo = mid + 1;
                    else hi = mid;
                }
                tails[lo] = j;
                tidx[lo] = i;
                prev[i] = lo > 0 ? tidx[lo - 1] : -1;
                if (lo == len) ++len;
            }
            // the chain back to front into tails[] as anchor i's (front first)
            int c = len;
            for (int i = len ? tidx[len - 1] : -1; i >= 0; i = prev[i]) tails[--c] = i;
            int3 *bl = a.blocks + (int64_t)p * a.bcap;
            int nb = 0;
            int64_t matched = 0;
            for (int t = 0; t < len; ++t) {
                const int i = tails[t], j = aj[i];
                if (nb) {
                    int3 &cur = bl[nb - 1];
                    if (j - i == cur.y - cur.x && i <= cur.x + cur.z) {
                        const int nl = max(cur.z, i + k - cur.x);
                        matched += nl - cur.z;
                        cur.z = nl;
                        continue;
                    }
                    if (i < cur.x + cur.z || j < cur.y + cur.z) continue;
                }
                if (nb == a.bcap) {          // cannot happen for blocks of >= k residues in a
                    record_error(a.err, kErrCapacity, p, nb);
                    break;
                }
                bl[nb++] = make_int3(i, j, k);
                matched += k;
            }
            int ia = 0, ib = 0, longest = 0;
            for (int t = 0; t <= nb; ++t) {
                const int sa = t < nb ? bl[t].x : m, sb = t < nb ? bl[t].y : n;
                longest = max(longest, max(sa - ia, sb - ib));
                if (t < nb) ia = sa + bl[t].z, ib = sb + bl[t].z;
            }
            atomicMax(a.counter + 1, longest);
            a.nblocks[p] = nb;
            a.seg_count[p] = nb + 1;
            a.seg_bytes[p] = (int64_t)m + n - 2 * matched;
        }
        __syncthreads();
    }
}

// Writes the segments of every pair: their bytes into the segment arena
// (a-part then b-part), the pseudo-sequence offsets and the pseudo pairs.
__global__ void __launch_bounds__(kAnchorThreads) seg_build_kernel(
    const uint8_t *__restrict__ codes, const int64_t *__restrict__ offs, const int32_t *__restrict__ pairs, int32_t P,
    const int3 *__restrict__ blocks, int32_t bcap, const int32_t *__restrict__ nblocks,
    const int32_t *__restrict__ seg_start, const int64_t *__restrict__ byte_start, uint8_t *__restrict__ seg_codes,
    int64_t *__restrict__ seg_offs, int32_t *__restrict__ seg_pairs) {
    for (int p = blockIdx.x; p < P; p += gridDim.x) {
        const int nb = nblocks[p];
        if (seg_start[p + 1] == seg_start[p]) continue;   // a rejected pair
        const int64_t xa = offs[pairs[2 * p]], ya = offs[pairs[2 * p + 1]];
        const int m = (int)(offs[pairs[2 * p] + 1] - xa), n = (int)(offs[pairs[2 * p + 1] + 1] - ya);
        const int3 *bl = blocks + (int64_t)p * bcap;
        int ia = 0, ib = 0;
        int64_t w = byte_start[p];
        for (int s = 0; s <= nb; ++s) {
            const int sa = s < nb ? bl[s].x : m, sb = s < nb ? bl[s].y : n;
            const int g = seg_start[p] + s;
            const int la = sa - ia, lb = sb - ib;
            for (int t = threadIdx.x; t < la; t += blockDim.x) seg_codes[w + t] = codes[xa + ia + t];
            for (int t = threadIdx.x; t < lb; t += blockDim.x) seg_codes[w + la + t] = codes[ya + ib + t];
            if (threadIdx.x == 0) {
                seg_offs[2 * g] = w;
                seg_offs[2 * g + 1] = w + la;
                seg_offs[2 * g + 2] = w + la + lb;
                seg_pairs[2 * g] = 2 * g;
                seg_pairs[2 * g + 1] = 2 * g + 1;
            }
            w += la + lb;
            if (s < nb) {
                ia = sa + bl[s].z;
                ib = sb + bl[s].z;
            }
        }
    }
}

// One warp per pair: the segments' scripts with each block's run of matches
// between them, and the total cost.
__global__ void assemble_kernel(int32_t P, const int3 *__restrict__ blocks, int32_t bcap,
                                const int32_t *__restrict__ nblocks, const int32_t *__restrict__ seg_start,
                                const int32_t *__restrict__ seg_score, const uint8_t *__restrict__ seg_ops,
                                const int64_t *__restrict__ seg_ops_off, const int32_t *__restrict__ seg_ops_len,
                                int32_t match, int32_t *__restrict__ score_out, uint8_t *__restrict__ ops_out,
                                const int64_t *__restrict__ ops_off, int32_t *__restrict__ ops_len_out) {
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < P; p += warps) {
        if (seg_start[p + 1] == seg_start[p]) continue;   // a rejected pair (error recorded)
        const int nb = nblocks[p];
        const int3 *bl = blocks + (int64_t)p * bcap;
        int64_t w = ops_off[p];
        int score = 0;
        for (int s = 0; s <= nb; ++s) {
            const int g = seg_start[p] + s;
            const int L = seg_ops_len[g];
            const uint8_t *src = seg_ops + seg_ops_off[g];
            for (int t = lane; t < L; t += 32) ops_out[w + t] = src[t];
            w += L;
            score += seg_score[g];
            if (s < nb) {
                const int z = bl[s].z;
                for (int t = lane; t < z; t += 32) ops_out[w + t] = 'M';
                w += z;
                score += z * match;
            }
        }
        if (lane == 0) {
            score_out[p] = score;
            ops_len_out[p] = (int32_t)(w - ops_off[p]);
        }
    }
}

}  // namespace msa

using namespace msa;

extern "C" {

msa_status msa_nw_align_batch_anchored(msa_ctx *ctx, const uint8_t *codes, const int64_t *offs, int32_t n_seqs,
                                       int64_t total, int32_t max_len, const int32_t *pairs, int64_t P, int32_t k,
                                       int32_t match, int32_t mismatch, int32_t gap, int32_t *score_out,
                                       uint8_t *ops_out, const int64_t *ops_off, int32_t *ops_len_out, void *stream) {
    if (!ctx) return MSA_EINVAL;
    if (P < 0 || P >= (int64_t(1) << 30) || n_seqs < 0 || max_len < 0 || total < 0)
        return set_error(ctx, MSA_EINVAL, "msa_nw_align_batch_anchored: negative or oversized count");
    if (k < 1 || k > kMaxK)
        return set_error(ctx, MSA_EINVAL, "msa_nw_align_batch_anchored: k %d outside 1..%d", k, kMaxK);
    if (P == 0) return MSA_OK;
    if (!codes || !offs || !pairs || !score_out || !ops_out || !ops_off || !ops_len_out)
        return set_error(ctx, MSA_EINVAL, "msa_nw_align_batch_anchored: null pointer");
    cudaStream_t st = (cudaStream_t)stream;
    const int Pi = (int)P;
    int tbits = 4;
    while ((int64_t(1) << tbits) < 2 * (int64_t)std::max(max_len, 1)) ++tbits;
    const int64_t slab = ((int64_t(1) << tbits) * (int64_t)sizeof(KmerSlot) + 4 * (int64_t)max_len * 4 + 255) / 256 * 256;
    const int32_t bcap = max_len / k + 1;
    Arena ar{ctx->ws, ctx->ws_bytes};
    int3 *blocks = ar.take<int3>((int64_t)Pi * bcap);
    int32_t *nblocks = ar.take<int32_t>(Pi);
    int32_t *seg_count = ar.take<int32_t>(Pi + 1);
    int64_t *seg_bytes = ar.take<int64_t>(Pi + 1);
    int32_t *seg_start = ar.take<int32_t>(Pi + 1);
    int64_t *byte_start = ar.take<int64_t>(Pi + 1);
    int32_t *tsum = ar.take<int32_t>(scan_tiles(Pi + 1));
    int64_t *tsum64 = ar.take<int64_t>(scan_tiles(Pi + 1));
    int32_t *counter = ar.take<int32_t>(64);
    if (!counter) return set_error(ctx, MSA_ENOMEM, "msa_nw_align_batch_anchored: workspace too small for the blocks");
    const int64_t nblk = std::min<int64_t>({(int64_t)ctx->sm_count * 4, (ar.cap - ar.used) / slab, (int64_t)Pi});
    if (nblk < 1)
        return set_error(ctx, MSA_ENOMEM, "msa_nw_align_batch_anchored: max_len %d needs %lld workspace bytes",
                         max_len, (long long)(slab + ar.used));
    Arena slabs_ar = ar;
    char *slabs = slabs_ar.take<char>(nblk * slab);
    cudaError_t e = cudaMemsetAsync(counter, 0, 8, st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "anchored memset");
    AnchorArgs aa{codes, offs, n_seqs, total, pairs, Pi, k, match, max_len, tbits, slabs, slab, blocks, bcap,
                  nblocks, seg_count, seg_bytes, counter, ctx->dev_err};
    anchor_chain_kernel<<<(int)nblk, kAnchorThreads, 0, st>>>(aa);
    exclusive_scan(seg_count, Pi, seg_start, tsum, st);
    exclusive_scan64(seg_bytes, Pi, byte_start, tsum64, st);
    ctx->launches += 5;
    // the totals and the longest segment size the segment batch: one read-back
    int32_t S = 0, seg_max = 0;
    int64_t bytes = 0;
    if ((e = cudaMemcpyAsync(&S, seg_start + Pi, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&bytes, byte_start + Pi, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&seg_max, counter + 1, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_check(ctx, e, "anchored totals");
    // the blocks and scans stay where they are; the segments follow them
    uint8_t *seg_codes = ar.take<uint8_t>(bytes + 64);
    int64_t *seg_offs = ar.take<int64_t>(2 * (int64_t)S + 1);
    int32_t *seg_pairs = ar.take<int32_t>(2 * (int64_t)S);
    int32_t *seg_score = ar.take<int32_t>(S);
    int32_t *seg_ops_len = ar.take<int32_t>(S);
    uint8_t *seg_ops = ar.take<uint8_t>(bytes + 64);
    if (!seg_ops) return set_error(ctx, MSA_ENOMEM, "msa_nw_align_batch_anchored: workspace too small for the segments");
    if (S == 0) return cuda_check(ctx, cudaGetLastError(), "anchored");
    seg_build_kernel<<<std::min(Pi, 65535), kAnchorThreads, 0, st>>>(codes, offs, pairs, Pi, blocks, bcap, nblocks,
                                                                      seg_start, byte_start, seg_codes, seg_offs,
                                                                      seg_pairs);
    ++ctx->launches;
    // a segment's script holds at most its two lengths: the offsets of its
    // bytes are its script offsets (every second pseudo-sequence offset)
    int64_t *seg_ops_off = ar.take<int64_t>((int64_t)S + 1);
    if (!seg_ops_off) return set_error(ctx, MSA_ENOMEM, "msa_nw_align_batch_anchored: workspace too small");
    if ((e = cudaMemcpy2DAsync(seg_ops_off, sizeof(int64_t), seg_offs, 2 * sizeof(int64_t), sizeof(int64_t), S + 1,
                               cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return cuda_check(ctx, e, "anchored script offsets");
    if (msa_status rc = nw_run(ctx, ar, seg_codes, seg_offs, 2 * S, bytes, seg_max, seg_pairs, S, match, mismatch, gap,
                               seg_score, seg_ops, seg_ops_off, seg_ops_len, st))
        return rc;
    assemble_kernel<<<std::max(1, std::min((Pi + 3) / 4, 65535)), 128, 0, st>>>(
        Pi, blocks, bcap, nblocks, seg_start, seg_score, seg_ops, seg_ops_off, seg_ops_len, match, score_out, ops_out,
        ops_off, ops_len_out);
    ++ctx->launches;
    return cuda_check(ctx, cudaGetLastError(), "anchored assemble");
}

}  // extern "C"
