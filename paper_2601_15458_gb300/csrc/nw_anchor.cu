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
// their i, the chain and the blocks by one warp in 32-anchor steps), scans
// of the segment counts and bytes, one read-back of the two totals and the
// longest segment, seg_build_kernel (the segments' bytes into an arena of
// their own, one warp per segment), nw_run on the segments, and
// assemble_kernel (a block scan of the segments' script lengths places
// them; the costs are added up).
#include <cuda_runtime.h>

#include <algorithm>

#include "msa_internal.cuh"

namespace msa {

constexpr int kAnchorThreads = 256;
constexpr int kMaxK = 256;
constexpr int64_t kSeqSmemMax = 64 * 1024;   // shared bytes for a pair's two sequences

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
    int32_t seq_smem;         // bytes of shared memory per sequence (0: read from global)
    char *slabs;              // per-block scratch
    int64_t slab_bytes;
    int4 *blocks;             // [P][bcap]: start in a, start in b, length, matched before
    int32_t bcap;
    int32_t *nblocks;         // [P]
    int32_t *seg_count;       // [P] segments (blocks + 1)
    int64_t *seg_bytes;       // [P] bytes outside the blocks (m + n - 2 sum of lengths)
    int32_t *counter;         // [0] pair claims, [1] longest segment
    int32_t *err;
};

// Multiplicative hash of the k bytes at s (a polynomial in an odd 64-bit
// base, then Fibonacci hashing to tbits bits); bytes are read 8 at a time
// so that the loads of a group are in flight together.
__device__ __forceinline__ uint32_t kmer_hash(const uint8_t *s, int k, int tbits) {
    unsigned long long h = 0;
    for (int t0 = 0; t0 < k; t0 += 8) {
        uint32_t c[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) c[u] = t0 + u < k ? s[t0 + u] : 0u;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (t0 + u < k) h = h * 0x100000001B3ull + (unsigned long long)c[u] + 1ull;
    }
    return (uint32_t)((h * 0x9E3779B97F4A7C15ull) >> (64 - tbits));
}

__device__ __forceinline__ bool same_kmer(const uint8_t *x, const uint8_t *y, int k) {
    for (int t0 = 0; t0 < k; t0 += 8) {
        uint32_t diff = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (t0 + u < k) diff |= (uint32_t)(x[t0 + u] ^ y[t0 + u]);
        if (diff) return false;
    }
    return true;
}

__global__ void __launch_bounds__(kAnchorThreads) anchor_chain_kernel(AnchorArgs a) {
    // chunks of the per-position arrays staged by the whole block, so the
    // sequential chain passes of warp 0 read shared memory, not global
    constexpr int kChunk = 2048;
    __shared__ int32_t s_a[kChunk], s_b[kChunk];
    __shared__ int32_t s_pair, s_len, s_last, s_want;
    // the pair's two sequences, when they fit (a.seq_smem: bytes per side)
    extern __shared__ uint8_t s_seq[];
    char *slab = a.slabs + (int64_t)blockIdx.x * a.slab_bytes;
    const int64_t tsize = int64_t(1) << a.tbits;
    KmerSlot *table = reinterpret_cast<KmerSlot *>(slab);
    // per position of a: its anchor's j (-1: none) and its chain level;
    // the patience tails; the chain (positions in a, in b)
    const int64_t L4 = ((int64_t)a.max_len + 3) & ~int64_t(3);
    int32_t *aj = reinterpret_cast<int32_t *>(slab + tsize * sizeof(KmerSlot));
    int32_t *level = aj + L4;
    int32_t *tails = level + L4;
    int32_t *cj = tails + L4;
    int32_t *ci = tails;          // written over the tails once they are done
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
        if (a.seq_smem) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) s_seq[i] = A[i];
            for (int j = threadIdx.x; j < n; j += blockDim.x) s_seq[a.seq_smem + j] = B[j];
            A = s_seq;
            B = s_seq + a.seq_smem;
        }
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
        // Chain and blocks: warp 0 over chunks the block stages.  Patience
        // sorting in a's order; level[i] = the chain length ending at anchor
        // i, minus one.  A window of 32 positions whose anchors all lie past
        // the last tail and increase (most windows when the pair is related)
        // appends them in one step; any other window is done one anchor at a
        // time by lane 0, exactly as the definition reads.
        const int lane = threadIdx.x & 31;
        const unsigned lt_mask = (1u << lane) - 1u;
        int len = 0, last_j = -1, last_i = -1;
        for (int c0 = 0; c0 < m; c0 += kChunk) {
            const int cn = min(kChunk, m - c0);
            for (int t = threadIdx.x; t < cn; t += blockDim.x) s_a[t] = aj[c0 + t];
            __syncthreads();
            if (threadIdx.x < 32) {
                for (int w0 = 0; w0 < cn; w0 += 32) {
                    const int t = w0 + lane;
                    const int j = t < cn ? s_a[t] : -1;
                    const unsigned amask = __ballot_sync(0xffffffffu, j >= 0);
                    if (!amask) continue;
                    int pm = j;                              // running max of j (non-anchors: -1)
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int v = __shfl_up_sync(0xffffffffu, pm, o);
                        if (lane >= o) pm = max(pm, v);
                    }
                    int before = __shfl_up_sync(0xffffffffu, pm, 1);
                    before = lane == 0 ? last_j : max(before, last_j);
                    if (__all_sync(0xffffffffu, j < 0 || j > before)) {
                        const int r = __popc(amask & lt_mask);
                        if (j >= 0) {
                            tails[len + r] = j;
                            s_b[t] = len + r;
                        }
                        const int top = 31 - __clz(amask);
                        last_j = __shfl_sync(0xffffffffu, j, top);
                        last_i = c0 + w0 + top;
                        len += __popc(amask);
                    } else {
                        if (lane == 0) {
                            for (int u = 0; u < 32 && w0 + u < cn; ++u) {
                                const int jj = s_a[w0 + u];
                                if (jj < 0) continue;
                                int lo = len;
                                if (jj < last_j) {       // first tail >= jj lies in [0, len - 1]
                                    int lo2 = 0, hi = len - 1;
                                    while (lo2 < hi) {
                                        const int mid = (lo2 + hi) >> 1;
                                        if (tails[mid] < jj) lo2 = mid + 1;
                                        else hi = mid;
                                    }
                                    lo = lo2;
                                }
                                tails[lo] = jj;
                                s_b[w0 + u] = lo;
                                if (lo == len) ++len;
                                if (lo == len - 1) {
                                    last_j = jj;
                                    last_i = c0 + w0 + u;
                                }
                            }
                        }
                        len = __shfl_sync(0xffffffffu, len, 0);
                        last_j = __shfl_sync(0xffffffffu, last_j, 0);
                        last_i = __shfl_sync(0xffffffffu, last_i, 0);
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
            for (int t = threadIdx.x; t < cn; t += blockDim.x)
                if (s_a[t] >= 0) level[c0 + t] = s_b[t];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            s_len = len;
            s_last = last_i;
            s_want = len - 1;
        }
        __syncthreads();
        len = s_len;
        last_i = s_last;
        // the chain, back to front: the anchor that set the last tail, then
        // before each chain anchor the nearest anchor one level lower (the
        // one whose tail it linked to when it was placed).  Warp 0 takes 32
        // positions at a time, lane 0 the highest: when the window's anchors
        // read want, want - 1, ... from the top they are all taken at once,
        // otherwise one at a time (the highest anchor at level want below the
        // last one taken).
        int c = len, want = len - 1;
        for (int hi = last_i + 1; hi > 0 && s_want >= 0; hi -= kChunk) {
            const int lo = max(0, hi - kChunk), cn = hi - lo;
            for (int t = threadIdx.x; t < cn; t += blockDim.x) {
                s_a[t] = aj[lo + t];
                s_b[t] = level[lo + t];
            }
            __syncthreads();
            if (threadIdx.x < 32) {
                for (int top = cn - 1; top >= 0 && want >= 0; top -= 32) {
                    const int t = top - lane;
                    const int j = t >= 0 ? s_a[t] : -1;
                    const int lev = j >= 0 ? s_b[t] : -1;
                    const unsigned amask = __ballot_sync(0xffffffffu, j >= 0);
                    if (!amask) continue;
                    const int r = __popc(amask & lt_mask);
                    if (__all_sync(0xffffffffu, j < 0 || lev == want - r)) {
                        if (j >= 0) {
                            ci[c - 1 - r] = lo + t;
                            cj[c - 1 - r] = j;
                        }
                        c -= __popc(amask);
                        want -= __popc(amask);
                    } else {
                        int from = 0;                    // lanes below `from` are above the last taken
                        while (want >= 0) {
                            const unsigned hit =
                                __ballot_sync(0xffffffffu, j >= 0 && lev == want && lane >= from);
                            if (!hit) break;
                            const int h = __ffs(hit) - 1;
                            if (lane == h) {
                                ci[c - 1] = lo + t;
                                cj[c - 1] = j;
                            }
                            --c;
                            --want;
                            from = h + 1;
                        }
                    }
                    __syncwarp();
                }
                if (lane == 0) s_want = want;
            }
            __syncthreads();
        }
        // blocks along the chain, the open one held by every lane of warp 0;
        // each block records the matched length before it (for the segment
        // offsets).  A run of chain anchors on the open block's diagonal,
        // each starting inside or right after the block as extended by the
        // ones before it, extends it in one step; the anchor that ends such
        // a run is taken alone.
        int4 *bl = a.blocks + (int64_t)p * a.bcap;
        int nb = 0, bx = -1, by = 0, bz = 0, ia = 0, ib = 0, longest = 0;
        int64_t matched = 0;
        bool full = false;
        auto close_block = [&]() {
            if (nb == a.bcap) {                  // cannot happen: blocks are >= k residues of a apart
                full = true;
                return;
            }
            if (lane == 0) bl[nb] = make_int4(bx, by, bz, (int)(matched - bz));
            ++nb;
            longest = max(longest, max(bx - ia, by - ib));
            ia = bx + bz;
            ib = by + bz;
        };
        for (int c0 = 0; c0 < len; c0 += kChunk) {
            const int cn = min(kChunk, len - c0);
            for (int t = threadIdx.x; t < cn; t += blockDim.x) {
                s_a[t] = ci[c0 + t];
                s_b[t] = cj[c0 + t];
            }
            __syncthreads();
            if (threadIdx.x < 32) {
                for (int w0 = 0; w0 < cn && !full; w0 += 32) {
                    const int wn = min(32, cn - w0);
                    const int i = lane < wn ? s_a[w0 + lane] : 0, j = lane < wn ? s_b[w0 + lane] : 0;
                    const int prev_i = __shfl_up_sync(0xffffffffu, i, 1);
                    int start = 0;
                    while (start < wn && !full) {
                        const int end_before = lane == start ? bx + bz : max(bx + bz, prev_i + k);
                        const bool in = lane >= start && lane < wn;
                        const bool ok = !in || (bx >= 0 && j - i == by - bx && i <= end_before);
                        const unsigned bad = __ballot_sync(0xffffffffu, !ok);
                        const int f = bad ? __ffs(bad) - 1 : wn;
                        if (f > start) {
                            const int iend = __shfl_sync(0xffffffffu, i, f - 1);
                            const int nl = max(bz, iend + k - bx);
                            matched += nl - bz;
                            bz = nl;
                        }
                        if (f >= wn) break;
                        const int fi = __shfl_sync(0xffffffffu, i, f), fj = __shfl_sync(0xffffffffu, j, f);
                        start = f + 1;
                        if (bx >= 0) {
                            if (fi < bx + bz || fj < by + bz) continue;   // dropped
                            close_block();
                            if (full) break;
                        }
                        bx = fi;
                        by = fj;
                        bz = k;
                        matched += k;
                    }
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (bx >= 0 && !full) close_block();
            if (full) record_error(a.err, kErrCapacity, p, nb);
            longest = max(longest, max(m - ia, n - ib));
            atomicMax(a.counter + 1, longest);
            a.nblocks[p] = nb;
            a.seg_count[p] = nb + 1;
            a.seg_bytes[p] = (int64_t)m + n - 2 * matched;
        }
        __syncthreads();
    }
}

// Exclusive scan of one value per thread over the block (kAnchorThreads);
// returns the thread's prefix and leaves the block total in *total.
__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_sums, int *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < kAnchorThreads / 32; ++w) {
            const int t = warp_sums[w];
            warp_sums[w] = run;
            run += t;
        }
        *total = run;
    }
    __syncthreads();
    return warp_sums[wid] + incl - v;
}

// Segment s of a pair runs from the end of block s - 1 (or the start) to the
// start of block s (or the end) in both sequences; blocks[.].w is the
// matched length before the block, so the bytes of the pair's earlier
// segments are (start in a + start in b - 2 x matched before).
struct SegSpan {
    int ia, ib, sa, sb, cum;
};

__device__ __forceinline__ SegSpan seg_span(const int4 *bl, int nb, int s, int m, int n) {
    SegSpan r{0, 0, m, n, 0};
    if (s > 0) {
        const int4 b = bl[s - 1];
        r.ia = b.x + b.z;
        r.ib = b.y + b.z;
        r.cum = b.w + b.z;
    }
    if (s < nb) {
        const int4 b = bl[s];
        r.sa = b.x;
        r.sb = b.y;
    }
    return r;
}

// Writes the segments of every pair: their bytes into the segment arena
// (a-part then b-part), the pseudo-sequence offsets and the pseudo pairs.
// One block per pair, one warp per segment.
__global__ void __launch_bounds__(kAnchorThreads) seg_build_kernel(
    const uint8_t *__restrict__ codes, const int64_t *__restrict__ offs, const int32_t *__restrict__ pairs, int32_t P,
    const int4 *__restrict__ blocks, int32_t bcap, const int32_t *__restrict__ nblocks,
    const int32_t *__restrict__ seg_start, const int64_t *__restrict__ byte_start, uint8_t *__restrict__ seg_codes,
    int64_t *__restrict__ seg_offs, int32_t *__restrict__ seg_pairs) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int p = blockIdx.x; p < P; p += gridDim.x) {
        if (seg_start[p + 1] == seg_start[p]) continue;   // a rejected pair
        const int nb = nblocks[p];
        const int64_t xa = offs[pairs[2 * p]], ya = offs[pairs[2 * p + 1]];
        const int m = (int)(offs[pairs[2 * p] + 1] - xa), n = (int)(offs[pairs[2 * p + 1] + 1] - ya);
        const int4 *bl = blocks + (int64_t)p * bcap;
        const int g0 = seg_start[p];
        const int64_t w0 = byte_start[p];
        for (int sg = wid; sg <= nb; sg += kAnchorThreads / 32) {
            const SegSpan sp = seg_span(bl, nb, sg, m, n);
            const int la = sp.sa - sp.ia, lb = sp.sb - sp.ib;
            const int64_t w = w0 + sp.ia + sp.ib - 2 * (int64_t)sp.cum;
            for (int t = lane; t < la; t += 32) seg_codes[w + t] = codes[xa + sp.ia + t];
            for (int t = lane; t < lb; t += 32) seg_codes[w + la + t] = codes[ya + sp.ib + t];
            if (lane == 0) {
                const int g = g0 + sg;
                seg_offs[2 * g] = w;
                seg_offs[2 * g + 1] = w + la;
                seg_offs[2 * g + 2] = w + la + lb;
                seg_pairs[2 * g] = 2 * g;
                seg_pairs[2 * g + 1] = 2 * g + 1;
            }
        }
    }
}

// Joins the segments' scripts with each block's run of matches between
// them and adds up the cost.  One block per pair: a block scan of the
// segments' script lengths places each segment, then one warp per segment
// copies its script and the block after it.
__global__ void __launch_bounds__(kAnchorThreads) assemble_kernel(
    int32_t P, const int4 *__restrict__ blocks, int32_t bcap, const int32_t *__restrict__ nblocks,
    const int32_t *__restrict__ seg_start, const int32_t *__restrict__ seg_score, const uint8_t *__restrict__ seg_ops,
    const int64_t *__restrict__ seg_ops_off, const int32_t *__restrict__ seg_ops_len, int32_t match,
    const uint8_t *__restrict__ codes, const int64_t *__restrict__ offs, const int32_t *__restrict__ pairs,
    const int32_t *__restrict__ sub, int32_t nsym, int32_t *err, int32_t *__restrict__ score_out,
    uint8_t *__restrict__ ops_out, const int64_t *__restrict__ ops_off, int32_t *__restrict__ ops_len_out) {
    __shared__ int warp_sums[kAnchorThreads / 32];
    __shared__ int s_total, s_score;
    __shared__ int64_t s_pos[kAnchorThreads];
    __shared__ int s_len[kAnchorThreads];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int p = blockIdx.x; p < P; p += gridDim.x) {
        if (seg_start[p + 1] == seg_start[p]) continue;   // a rejected pair (error recorded)
        const int nb = nblocks[p];
        const int4 *bl = blocks + (int64_t)p * bcap;
        const int g0 = seg_start[p];
        const int64_t base = ops_off[p];
        if (threadIdx.x == 0) s_score = 0;
        int64_t carry = 0;                                  // script bytes of earlier chunks
        for (int s0 = 0; s0 <= nb; s0 += kAnchorThreads) {
            const int sg = s0 + threadIdx.x;
            const bool live = sg <= nb;
            const int L = live ? seg_ops_len[g0 + sg] : 0;
            const int excl = block_exclusive_scan(L, warp_sums, &s_total);
            if (live) {
                const int cum = sg > 0 ? bl[sg - 1].w + bl[sg - 1].z : 0;
                s_pos[threadIdx.x] = base + carry + excl + cum;
                s_len[threadIdx.x] = L;
                atomicAdd(&s_score, seg_score[g0 + sg]);
            }
            __syncthreads();
            const int cnt = min(kAnchorThreads, nb + 1 - s0);
            for (int t = wid; t < cnt; t += kAnchorThreads / 32) {
                const int g = g0 + s0 + t;
                const uint8_t *src = seg_ops + seg_ops_off[g];
                const int64_t pos = s_pos[t];
                const int len = s_len[t];
                for (int u = lane; u < len; u += 32) ops_out[pos + u] = src[u];
                if (s0 + t < nb) {
                    const int z = bl[s0 + t].z;
                    for (int u = lane; u < z; u += 32) ops_out[pos + len + u] = 'M';
                    if (sub) {                     // a block residue costs the table's diagonal
                        const uint8_t *A = codes + offs[pairs[2 * p]] + bl[s0 + t].x;
                        int v = 0;
                        for (int u = lane; u < z; u += 32) {
                            const int c = A[u];
                            if (c < nsym) v += sub[c * nsym + c];
                            else record_error(err, kErrSymbol, p, c);
                        }
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                        if (lane == 0) atomicAdd(&s_score, v);
                    }
                }
            }
            carry += s_total;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const int matched = nb > 0 ? bl[nb - 1].w + bl[nb - 1].z : 0;
            score_out[p] = s_score + (sub ? 0 : matched * match);
            ops_len_out[p] = (int32_t)(carry + matched);
        }
        __syncthreads();
    }
}

// The anchored split with linear gaps (gap_open < 0: segments by nw_run) or
// affine gaps (segments by nw_affine_run, with the table when sub is given).
static msa_status anchored_run(msa_ctx *ctx, const uint8_t *codes, const int64_t *offs, int32_t n_seqs, int64_t total,
                               int32_t max_len, const int32_t *pairs, int64_t P, int32_t k, int32_t match,
                               int32_t mismatch, int32_t gap, int32_t gap_open, const int32_t *sub, int32_t nsym,
                               int32_t *score_out, uint8_t *ops_out, const int64_t *ops_off, int32_t *ops_len_out,
                               void *stream) {
    if (!ctx) return MSA_EINVAL;
    if (sub && (nsym < 1 || nsym > 32))
        return set_error(ctx, MSA_EINVAL, "msa_nw_align_batch_anchored: table of %d symbols outside 1..32", nsym);
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
    const int64_t slab = ((int64_t(1) << tbits) * (int64_t)sizeof(KmerSlot) + 4 * (((int64_t)max_len + 3) & ~int64_t(3)) * 4 + 255) / 256 * 256;
    const int32_t bcap = max_len / k + 1;
    Arena ar{ctx->ws, ctx->ws_bytes};
    int4 *blocks = ar.take<int4>((int64_t)Pi * bcap);
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
    // the pair's sequences go to shared memory when both fit in kSeqSmemMax
    const int32_t seq_smem = 2 * (((int64_t)max_len + 15) & ~int64_t(15)) <= kSeqSmemMax ? (max_len + 15) & ~15 : 0;
    if (seq_smem && (e = cudaFuncSetAttribute(anchor_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              2 * seq_smem)) != cudaSuccess)
        return cuda_check(ctx, e, "anchored smem attribute");
    AnchorArgs aa{codes, offs, n_seqs, total, pairs, Pi, k, match, max_len, tbits, seq_smem, slabs, slab, blocks, bcap,
                  nblocks, seg_count, seg_bytes, counter, ctx->dev_err};
    anchor_chain_kernel<<<(int)nblk, kAnchorThreads, 2 * seq_smem, st>>>(aa);
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
    if (msa_status rc = gap_open < 0
                            ? nw_run(ctx, ar, seg_codes, seg_offs, 2 * S, bytes, seg_max, seg_pairs, S, match,
                                     mismatch, gap, seg_score, seg_ops, seg_ops_off, seg_ops_len, st)
                            : nw_affine_run(ctx, ar, seg_codes, seg_offs, 2 * S, bytes, seg_max, seg_pairs, S, match,
                                            mismatch, gap_open, gap, seg_score, seg_ops, seg_ops_off, seg_ops_len, st,
                                            sub, nsym))
        return rc;
    assemble_kernel<<<std::min(Pi, 65535), kAnchorThreads, 0, st>>>(
        Pi, blocks, bcap, nblocks, seg_start, seg_score, seg_ops, seg_ops_off, seg_ops_len, match, codes, offs, pairs,
        sub, nsym, ctx->dev_err, score_out, ops_out, ops_off, ops_len_out);
    ++ctx->launches;
    return cuda_check(ctx, cudaGetLastError(), "anchored assemble");
}

}  // namespace msa

using namespace msa;

extern "C" {

msa_status msa_nw_align_batch_anchored(msa_ctx *ctx, const uint8_t *codes, const int64_t *offs, int32_t n_seqs,
                                       int64_t total, int32_t max_len, const int32_t *pairs, int64_t P, int32_t k,
                                       int32_t match, int32_t mismatch, int32_t gap, int32_t *score_out,
                                       uint8_t *ops_out, const int64_t *ops_off, int32_t *ops_len_out, void *stream) {
    return anchored_run(ctx, codes, offs, n_seqs, total, max_len, pairs, P, k, match, mismatch, gap, -1, nullptr, 0,
                        score_out, ops_out, ops_off, ops_len_out, stream);
}

msa_status msa_nw_align_batch_anchored_affine(msa_ctx *ctx, const uint8_t *codes, const int64_t *offs,
                                              int32_t n_seqs, int64_t total, int32_t max_len, const int32_t *pairs,
                                              int64_t P, int32_t k, int32_t match, int32_t mismatch, int32_t gap_open,
                                              int32_t gap_ext, int32_t *score_out, uint8_t *ops_out,
                                              const int64_t *ops_off, int32_t *ops_len_out, void *stream) {
    if (ctx && gap_open < 0)
        return set_error(ctx, MSA_EINVAL, "msa_nw_align_batch_anchored_affine: negative gap_open %d", gap_open);
    return anchored_run(ctx, codes, offs, n_seqs, total, max_len, pairs, P, k, match, mismatch, gap_ext, gap_open,
                        nullptr, 0, score_out, ops_out, ops_off, ops_len_out, stream);
}

msa_status msa_nw_align_batch_anchored_affine_sub(msa_ctx *ctx, const uint8_t *codes, const int64_t *offs,
                                                  int32_t n_seqs, int64_t total, int32_t max_len, const int32_t *pairs,
                                                  int64_t P, int32_t k, const int32_t *sub, int32_t nsym,
                                                  int32_t gap_open, int32_t gap_ext, int32_t *score_out,
                                                  uint8_t *ops_out, const int64_t *ops_off, int32_t *ops_len_out,
                                                  void *stream) {
    if (ctx && (gap_open < 0 || !sub))
        return set_error(ctx, MSA_EINVAL, "msa_nw_align_batch_anchored_affine_sub: negative gap_open or null table");
    return anchored_run(ctx, codes, offs, n_seqs, total, max_len, pairs, P, k, 0, 0, gap_ext, gap_open, sub, nsym,
                        score_out, ops_out, ops_off, ops_len_out, stream);
}

}  // extern "C"
