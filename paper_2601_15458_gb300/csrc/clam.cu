// Guide tree by Alg. 1 "Partition" (A11) and the bottom-up merge of section
// "Merging" (A12): C entry points msa_clam_partition, msa_merge_tree and
// msa_msa_rows.
//
// Partition, level by level (all clusters of one depth at once):
//   centre c = geometric median over the candidates S of the cluster (all of
//     C when |C| <= 256, else the 256 members at positions floor(k|C|/256)
//     of C sorted by index): one batch of all unordered pairs within S,
//     row sums, argmin (ties: smallest index);
//   l = argmax f(c, x), r = argmax f(l, x) over C (ties: smallest index):
//     one-to-many batches;
//   L = {x : f(l, x) <= f(r, x)}, R = the rest: a stable partition of the
//     cluster's contiguous range in `order`, so every cluster stays sorted by
//     index and occupies one range.
// The host keeps the node table and reads back only the left sizes once per
// level; all distances, reductions and the partition run on the device.  A
// cluster of at most 256 members keeps its medoid batch as a distance
// matrix, from which it and all its descendants read every later distance
// (the same values the DP would give, so the tree is unchanged).
//
// Merge, height by height (all merges of one height at once): every
// sequence s keeps pos_s[k], the column of its k-th residue in the MSA of the
// cluster that currently holds it (so the MSA itself is never stored).  A
// merge builds the gapped rows of both children's centres from pos, aligns
// them with NW (the gap symbol is an ordinary symbol), turns the edit script
// into two monotone column maps (child column -> parent column) and applies
// them to pos of every member of each child.  The parent's rows are the left
// child's rows followed by the right child's, which is `order` restricted to
// the parent's range.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "msa_internal.cuh"

namespace msa {

constexpr int kMedoidSample = 256;

// ---------------------------------------------------------------------------
// partition kernels
// ---------------------------------------------------------------------------

// Candidate j of node k sits at range position lo + floor(j * size / s_k)
// (s_k = min(size, 256)).
__device__ __forceinline__ int cand_pos(int lo, int size, int s, int j) {
    return size <= kMedoidSample ? lo + j : lo + (int)(((int64_t)j * size) / kMedoidSample);
}

// Distance matrices of small clusters.  A cluster of at most 256 members
// computes all its unordered pairs for its medoid; they are kept as a
// |C| x |C| matrix in a pool, and every distance the cluster and all its
// descendants need later (c, l and r against the members, the medoids of
// the sub-clusters) is read from it instead of being computed again.
// base[k] < 0: cluster k has no matrix.
struct MatView {
    const int64_t *base;    // [A] offset of the cluster's matrix in the pool
    const int32_t *stride;  // [A] its row length (the size of the cluster that made it)
    const int32_t *local;   // [N] a sequence's row in its matrix
    const int32_t *pool;
    __device__ __forceinline__ bool has(int k) const { return base[k] >= 0; }
    __device__ __forceinline__ int32_t d(int k, int x, int y) const {
        return pool[base[k] + (int64_t)local[x] * stride[k] + local[y]];
    }
};

// Pair t of a medoid batch over s candidates: candidate i with i + d (mod s)
// for d = 1..h, h = (s - 1) / 2, and for even s also i + s/2 for i < s/2.
__device__ __forceinline__ void medoid_pair(int64_t t, int s, int &i, int &j) {
    const int h = (s - 1) / 2;
    if (t < (int64_t)s * h) {
        i = (int)(t / h);
        j = (i + (int)(t % h) + 1) % s;
    } else {
        i = (int)(t - (int64_t)s * h);
        j = i + s / 2;
    }
}

// Medoid pairs of the nodes whose medoid is computed (poff[k + 1] > poff[k]).
__global__ void medoid_pairs_kernel(const int32_t *__restrict__ order, const int32_t *__restrict__ nlo,
                                    const int32_t *__restrict__ nsize, const int64_t *__restrict__ poff, int A,
                                    int32_t *__restrict__ pairs) {
    for (int k = blockIdx.x; k < A; k += gridDim.x) {
        const int lo = nlo[k], size = nsize[k];
        const int s = min(size, kMedoidSample);
        const int64_t base = poff[k], cnt = poff[k + 1] - poff[k];
        for (int64_t t = threadIdx.x; t < cnt; t += blockDim.x) {
            int i, j;
            medoid_pair(t, s, i, j);
            pairs[2 * (base + t)] = order[cand_pos(lo, size, s, i)];
            pairs[2 * (base + t) + 1] = order[cand_pos(lo, size, s, j)];
        }
    }
}

// The matrices of the nodes that make one at this level (fresh[k]): their
// medoid distances in both orders, zeros on the diagonal, and each member's
// row.
__global__ void build_matrix_kernel(const int32_t *__restrict__ order, const int32_t *__restrict__ nlo,
                                    const int32_t *__restrict__ nsize, const int64_t *__restrict__ poff, int A,
                                    const int32_t *__restrict__ fresh, const int64_t *__restrict__ mbase,
                                    const int32_t *__restrict__ d, int32_t *__restrict__ pool,
                                    int32_t *__restrict__ local) {
    for (int k = blockIdx.x; k < A; k += gridDim.x) {
        if (!fresh[k]) continue;
        const int lo = nlo[k], s = nsize[k];
        const int64_t base = mbase[k], cnt = poff[k + 1] - poff[k];
        for (int i = threadIdx.x; i < s; i += blockDim.x) {
            local[order[lo + i]] = i;
            pool[base + (int64_t)i * s + i] = 0;
        }
        for (int64_t t = threadIdx.x; t < cnt; t += blockDim.x) {
            int i, j;
            medoid_pair(t, s, i, j);
            const int32_t v = d[poff[k] + t];
            pool[base + (int64_t)i * s + j] = v;
            pool[base + (int64_t)j * s + i] = v;
        }
    }
}

__global__ void medoid_sums_kernel(const int32_t *__restrict__ order, const int32_t *__restrict__ nlo,
                                   const int32_t *__restrict__ nsize, const int64_t *__restrict__ poff,
                                   const int64_t *__restrict__ soff, int A, const int32_t *__restrict__ d, MatView M,
                                   unsigned long long *__restrict__ sums) {
    for (int k = blockIdx.x; k < A; k += gridDim.x) {
        const int lo = nlo[k];
        const int s = min(nsize[k], kMedoidSample);
        const bool mat = M.has(k);                 // then the candidates are all s members
        const int64_t cnt = (int64_t)s * (s - 1) / 2;
        for (int64_t t = threadIdx.x; t < cnt; t += blockDim.x) {
            int i, j;
            medoid_pair(t, s, i, j);
            const unsigned long long v =
                (unsigned long long)(mat ? M.d(k, order[lo + i], order[lo + j]) : d[poff[k] + t]);
            atomicAdd(sums + soff[k] + i, v);
            atomicAdd(sums + soff[k] + j, v);
        }
    }
}

// centre of node k: argmin over candidates of (row sum, index)
__global__ void medoid_argmin_kernel(const int32_t *__restrict__ order, const int32_t *__restrict__ nlo,
                                     const int32_t *__restrict__ nsize, const int64_t *__restrict__ soff, int A,
                                     const unsigned long long *__restrict__ sums, int32_t *__restrict__ center) {
    __shared__ unsigned long long best[32];
    for (int k = blockIdx.x; k < A; k += gridDim.x) {
        const int lo = nlo[k], size = nsize[k];
        const int s = min(size, kMedoidSample);
        unsigned long long b = ~0ull;
        for (int i = threadIdx.x; i < s; i += blockDim.x) {
            const int idx = order[cand_pos(lo, size, s, i)];
            // sums < 2^31 for any realistic input: key = sum << 32 | index
            const unsigned long long key = (sums[soff[k] + i] << 32) | (unsigned)idx;
            b = key < b ? key : b;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long x = __shfl_xor_sync(0xffffffffu, b, o);
            b = x < b ? x : b;
        }
        if ((threadIdx.x & 31) == 0) best[threadIdx.x >> 5] = b;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long m = ~0ull;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = best[w] < m ? best[w] : m;
            center[k] = (int32_t)(m & 0xffffffffu);
        }
        __syncthreads();
    }
}

// one-to-many pairs (q_k, order[i]) for i in node k's range, for the nodes
// whose distances are computed (moff[k + 1] > moff[k])
__global__ void one_to_many_kernel(const int32_t *__restrict__ order, const int32_t *__restrict__ nlo,
                                   const int64_t *__restrict__ moff, int A, const int32_t *__restrict__ q,
                                   int32_t *__restrict__ pairs) {
    for (int k = blockIdx.x; k < A; k += gridDim.x) {
        const int lo = nlo[k];
        const int cnt = (int)(moff[k + 1] - moff[k]);
        const int qk = q[k];
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            pairs[2 * (moff[k] + i)] = qk;
            pairs[2 * (moff[k] + i) + 1] = order[lo + i];
        }
    }
}

// argmax over (distance from q_k, -index) per node
__global__ void argmax_kernel(const int32_t *__restrict__ order, const int32_t *__restrict__ nlo,
                              const int32_t *__restrict__ nsize, const int64_t *__restrict__ moff, int A,
                              const int32_t *__restrict__ d, const int32_t *__restrict__ q, MatView M,
                              int32_t *__restrict__ out) {
    __shared__ unsigned long long best[32];
    for (int k = blockIdx.x; k < A; k += gridDim.x) {
        const int lo = nlo[k], size = nsize[k];
        const bool mat = M.has(k);
        const int qk = q[k];
        unsigned long long b = 0;
        for (int i = threadIdx.x; i < size; i += blockDim.x) {
            const int x = order[lo + i];
            const unsigned dist = (unsigned)(mat ? M.d(k, qk, x) : d[moff[k] + i]);
            const unsigned long long key = ((unsigned long long)dist << 32) | (0xffffffffu - (unsigned)x);
            b = key > b ? key : b;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long x = __shfl_xor_sync(0xffffffffu, b, o);
            b = x > b ? x : b;
        }
        if ((threadIdx.x & 31) == 0) best[threadIdx.x >> 5] = b;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long m = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = best[w] > m ? best[w] : m;
            out[k] = (int32_t)(0xffffffffu - (unsigned)(m & 0xffffffffu));
        }
        __syncthreads();
    }
}

// stable partition of each node's range: L = {x : f(l,x) <= f(r,x)} first.
// One block per node: block-wide scans over the range in chunks.
__global__ void __launch_bounds__(1024) split_kernel(const int32_t *__restrict__ order, int32_t *__restrict__ order_out,
                                                     const int32_t *__restrict__ nlo, const int32_t *__restrict__ nsize,
                                                     const int64_t *__restrict__ moff, int A,
                                                     const int32_t *__restrict__ dl, const int32_t *__restrict__ dr,
                                                     const int32_t *__restrict__ ql, const int32_t *__restrict__ qr,
                                                     MatView M, int32_t *__restrict__ nleft) {
    __shared__ int32_t wsum[32];
    __shared__ int32_t base_l;
    for (int k = blockIdx.x; k < A; k += gridDim.x) {
        const int lo = nlo[k], size = nsize[k];
        const bool mat = M.has(k);
        const int lk = ql[k], rk = qr[k];
        // x goes left when f(l, x) <= f(r, x)
        auto goes_left = [&](int i) {
            if (mat) {
                const int x = order[lo + i];
                return M.d(k, lk, x) <= M.d(k, rk, x);
            }
            return dl[moff[k] + i] <= dr[moff[k] + i];
        };
        // pass 1: count lefts
        int c = 0;
        for (int i = threadIdx.x; i < size; i += blockDim.x) c += goes_left(i);
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
            base_l = t;
            nleft[k] = t;
        }
        __syncthreads();
        const int nl = base_l;
        // pass 2: chunked stable scatter
        int run_l = 0, run_r = 0;
        for (int c0 = 0; c0 < size; c0 += blockDim.x) {
            const int i = c0 + threadIdx.x;
            const int f = i < size ? (int)goes_left(i) : 0;
            const int valid = i < size;
            // block exclusive scan of f
            const unsigned mask = __ballot_sync(0xffffffffu, f);
            const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
            const int wpre = __popc(mask & ((1u << lane) - 1u));
            __syncthreads();
            if (lane == 0) wsum[w] = __popc(mask);
            __syncthreads();
            int before = 0, tot = 0;
            for (int x = 0; x < (int)(blockDim.x >> 5); ++x) {
                if (x < w) before += wsum[x];
                tot += wsum[x];
            }
            const int pl = run_l + before + wpre;
            const int nvalid = min((int)blockDim.x, size - c0);
            if (valid) {
                const int v = order[lo + i];
                if (f)
                    order_out[lo + pl] = v;
                else
                    order_out[lo + nl + run_r + (threadIdx.x - (before + wpre))] = v;
            }
            run_l += tot;
            run_r += nvalid - tot;
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// merge kernels
// ---------------------------------------------------------------------------

// gapped centre rows: row m*2 = centre of the left child, m*2+1 = right child
__global__ void center_rows_kernel(const uint8_t *__restrict__ codes, const int64_t *__restrict__ offs,
                                   const int32_t *__restrict__ pos, const int32_t *__restrict__ rc,
                                   const int64_t *__restrict__ roff, int nrows, uint8_t gap_code,
                                   uint8_t *__restrict__ rows) {
    for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int64_t o = roff[r], w = roff[r + 1] - o;
        for (int64_t c = threadIdx.x; c < w; c += blockDim.x) rows[o + c] = gap_code;
        __syncthreads();
        const int s = rc[r];
        const int64_t a = offs[s], L = offs[s + 1] - a;
        for (int64_t k = threadIdx.x; k < L; k += blockDim.x) {
            const int c = pos[a + k];
            if (c >= 0 && c < w) rows[o + c] = codes[a + k];
        }
        __syncthreads();
    }
}

// column maps from the edit scripts: one thread per merge
__global__ void column_maps_kernel(const uint8_t *__restrict__ ops, const int64_t *__restrict__ ops_off,
                                   const int32_t *__restrict__ ops_len, const int64_t *__restrict__ roff, int M,
                                   int32_t *__restrict__ maps) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const uint8_t *o = ops + ops_off[m];
    int32_t *mapL = maps + roff[2 * m];
    int32_t *mapR = maps + roff[2 * m + 1];
    const int64_t wl = roff[2 * m + 1] - roff[2 * m], wr = roff[2 * m + 2] - roff[2 * m + 1];
    int64_t il = 0, ir = 0;
    const int L = ops_len[m];
    for (int t = 0; t < L; ++t) {
        const uint8_t op = o[t];
        if (op != 'I' && il < wl) mapL[il++] = t;     // M, X, D consume the left row
        if (op != 'D' && ir < wr) mapR[ir++] = t;     // M, X, I consume the right row
    }
}

// pos <- map[pos] for every member of every merged child: one warp per sequence
__global__ void apply_maps_kernel(const int32_t *__restrict__ order, const int64_t *__restrict__ offs,
                                  const int32_t *__restrict__ seg_lo, const int32_t *__restrict__ seg_hi,
                                  const int64_t *__restrict__ seg_map, int nseg, int32_t total_members,
                                  const int64_t *__restrict__ seg_start, const int32_t *__restrict__ maps,
                                  int32_t *__restrict__ pos) {
    const int lane = threadIdx.x & 31;
    for (int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < total_members;
         g += (int64_t)gridDim.x * (blockDim.x >> 5)) {
        // find the segment of member g (segments are in order of seg_start)
        int lo = 0, hi = nseg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (seg_start[mid] <= g) lo = mid; else hi = mid - 1;
        }
        const int s = order[seg_lo[lo] + (int)(g - seg_start[lo])];
        const int32_t *map = maps + seg_map[lo];
        const int64_t a = offs[s], L = offs[s + 1] - a;
        for (int64_t k = lane; k < L; k += 32) pos[a + k] = map[pos[a + k]];
    }
}

__global__ void init_pos_kernel(const int64_t *__restrict__ offs, int n, int32_t *__restrict__ pos) {
    for (int64_t s = blockIdx.x; s < n; s += gridDim.x) {
        const int64_t a = offs[s], L = offs[s + 1] - a;
        for (int64_t k = threadIdx.x; k < L; k += blockDim.x) pos[a + k] = (int32_t)k;
    }
}

__global__ void rows_kernel(const uint8_t *__restrict__ ascii, const int64_t *__restrict__ offs,
                            const int32_t *__restrict__ order, const int32_t *__restrict__ pos, int n, int W,
                            uint8_t *__restrict__ out) {
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        uint8_t *row = out + r * (int64_t)W;
        for (int c = threadIdx.x; c < W; c += blockDim.x) row[c] = '-';
        __syncthreads();
        const int s = order[r];
        const int64_t a = offs[s], L = offs[s + 1] - a;
        for (int64_t k = threadIdx.x; k < L; k += blockDim.x) {
            const int c = pos[a + k];
            if (c >= 0 && c < W) row[c] = ascii[a + k];
        }
        __syncthreads();
    }
}

template <class T>
static msa_status h2d(msa_ctx *ctx, T *dst, const std::vector<T> &src, cudaStream_t st) {
    if (src.empty()) return MSA_OK;
    return cuda_check(ctx, cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st),
                      "host to device copy");
}

// Starting bands of the distance batches from the band network (nullptr:
// every batch runs the full DP).
struct PartitionBand {
    const void *state;
    const uint16_t *prof;
    float gamma;
    int32_t margin;
};

static msa_status clam_partition_run(msa_ctx *ctx, const msa_seqset *s, const PartitionBand *band, int32_t *order,
                                     int32_t *lo, int32_t *hi, int32_t *center, int32_t *left, int32_t *right,
                                     int32_t *parent, int32_t *n_nodes, void *stream) {
    msa_status rc = lev_validate(ctx, s, order, 1, order, "msa_clam_partition");
    if (rc) return rc;
    if (!lo || !hi || !center || !left || !right || !parent || !n_nodes)
        return set_error(ctx, MSA_EINVAL, "msa_clam_partition: null pointer");
    const int N = s->n_seqs;
    *n_nodes = 0;
    if (N == 0) return MSA_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // node table (host)
    int nn = 1;
    lo[0] = 0;
    hi[0] = N;
    parent[0] = -1;
    left[0] = right[0] = -1;
    center[0] = N == 1 ? 0 : -1;
    {
        std::vector<int32_t> iota(N);
        for (int i = 0; i < N; ++i) iota[i] = i;
        if ((rc = h2d(ctx, order, iota, st))) return rc;
    }
    std::vector<int32_t> active = N > 1 ? std::vector<int32_t>{0} : std::vector<int32_t>{};
    Arena base{ctx->ws, ctx->ws_bytes};
    int32_t *order_tmp = base.take<int32_t>(N);
    int32_t *mlocal = base.take<int32_t>(N);
    if (!mlocal) return set_error(ctx, MSA_ENOMEM, "msa_clam_partition: workspace");
    // the matrix pool: at most 256 N entries are ever needed (the clusters
    // that make matrices are disjoint and have at most 256 members); a
    // quarter of the free workspace at most, and a cluster that does not fit
    // computes its distances as a large one does
    const int64_t pool_cap = std::min<int64_t>((int64_t)kMedoidSample * N, (base.cap - base.used) / 16);
    int32_t *pool = base.take<int32_t>(std::max<int64_t>(pool_cap, 1));
    if (!pool) return set_error(ctx, MSA_ENOMEM, "msa_clam_partition: workspace");
    int64_t pool_used = 0;
    // per node: its matrix (offset in the pool, -1: none) and row length
    std::vector<int64_t> node_mbase(2 * (size_t)N, -1);
    std::vector<int32_t> node_mstride(2 * (size_t)N, 0);
    // order_tmp mirrors order: each level's split rewrites the active ranges
    // in order_tmp and one copy of the whole array brings them back (ranges
    // that are no longer active are equal in both)
    {
        cudaError_t e = cudaMemcpyAsync(order_tmp, order, N * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_check(ctx, e, "partition order copy");
    }
    while (!active.empty()) {
        const int A = (int)active.size();
        std::vector<int32_t> hlo(A), hsz(A), hfresh(A, 0), hstride(A, 0);
        std::vector<int64_t> poff(A + 1), soff(A + 1), moff(A + 1), hmbase(A, -1);
        poff[0] = soff[0] = moff[0] = 0;
        for (int k = 0; k < A; ++k) {
            const int nd = active[k];
            hlo[k] = lo[nd];
            hsz[k] = hi[nd] - lo[nd];
            const int64_t sk = std::min(hsz[k], kMedoidSample);
            // a cluster of at most 256 members without a matrix makes one
            // from its medoid batch, if the pool has room
            if (node_mbase[nd] < 0 && hsz[k] <= kMedoidSample &&
                pool_used + (int64_t)hsz[k] * hsz[k] <= pool_cap) {
                node_mbase[nd] = pool_used;
                node_mstride[nd] = hsz[k];
                pool_used += (int64_t)hsz[k] * hsz[k];
                hfresh[k] = 1;
            }
            hmbase[k] = node_mbase[nd];
            hstride[k] = node_mstride[nd];
            const bool mat = hmbase[k] >= 0;
            // computed: the medoid batch unless an ancestor's matrix holds it,
            // the one-to-many batches unless the cluster has a matrix
            poff[k + 1] = poff[k] + (mat && !hfresh[k] ? 0 : sk * (sk - 1) / 2);
            soff[k + 1] = soff[k] + sk;
            moff[k + 1] = moff[k] + (mat ? 0 : hsz[k]);
        }
        const int64_t PM = poff[A], PC = moff[A];
        Arena ar = base;
        int32_t *d_lo = ar.take<int32_t>(A), *d_sz = ar.take<int32_t>(A);
        int64_t *d_poff = ar.take<int64_t>(A + 1), *d_soff = ar.take<int64_t>(A + 1), *d_moff = ar.take<int64_t>(A + 1);
        int32_t *d_c = ar.take<int32_t>(A), *d_l = ar.take<int32_t>(A), *d_r = ar.take<int32_t>(A),
                *d_nl = ar.take<int32_t>(A);
        int64_t *d_mbase = ar.take<int64_t>(A);
        int32_t *d_stride = ar.take<int32_t>(A), *d_fresh = ar.take<int32_t>(A);
        unsigned long long *sums = ar.take<unsigned long long>(soff[A]);
        int32_t *pairs = ar.take<int32_t>(2 * std::max(PM, PC));
        int32_t *dm = ar.take<int32_t>(PM), *dc = ar.take<int32_t>(PC), *dl = ar.take<int32_t>(PC),
                *dr = ar.take<int32_t>(PC);
        const int64_t PX = std::max(PM, PC);
        const int64_t need = band ? msa_lev_banded_workspace_bytes(PX, N) + 3 * ((4 * PX + 255) / 256 * 256)
                                  : lev_workspace(PX, N);
        if (!dr || ar.cap - ar.used < need)
            return set_error(ctx, MSA_ENOMEM, "msa_clam_partition: workspace too small for a level of %d clusters", A);
        // one distance batch: the full DP, or the network's band and the
        // certified banded DP (exact either way)
        // The network's bands serve the medoid batches only: c, l and r are
        // far from most of the cluster (l and r are argmaxes), their bands
        // cover most of each matrix, and the full DP's lane kernel does such
        // batches faster than the band kernels (measured on 50,000 16S-like
        // sequences: 2.5 ms against 4-5 ms per one-to-many batch).
        auto dist = [&](const int32_t *pr, int64_t np, int32_t *out, bool banded) -> msa_status {
            Arena tmp = ar;
            if (!band || !banded) return lev_run(ctx, s, pr, np, out, st, nullptr, nullptr, &tmp);
            float *yhat = tmp.take<float>(np);
            int32_t *k0 = tmp.take<int32_t>(np), *ku = tmp.take<int32_t>(np);
            if (!ku) return set_error(ctx, MSA_ENOMEM, "msa_clam_partition_banded: workspace");
            msa_status r2 = msa_band_predict(ctx, band->state, s, band->prof, pr, np, band->gamma, band->margin,
                                             yhat, k0, st);
            if (r2) return r2;
            return lev_banded_run(ctx, s, pr, np, k0, out, ku, st, tmp);
        };
        if ((rc = h2d(ctx, d_lo, hlo, st)) || (rc = h2d(ctx, d_sz, hsz, st)) || (rc = h2d(ctx, d_poff, poff, st)) ||
            (rc = h2d(ctx, d_soff, soff, st)) || (rc = h2d(ctx, d_moff, moff, st)) ||
            (rc = h2d(ctx, d_mbase, hmbase, st)) || (rc = h2d(ctx, d_stride, hstride, st)) ||
            (rc = h2d(ctx, d_fresh, hfresh, st)))
            return rc;
        const MatView M{d_mbase, d_stride, mlocal, pool};
        cudaError_t e = cudaMemsetAsync(sums, 0, soff[A] * sizeof(unsigned long long), st);
        if (e != cudaSuccess) return cuda_check(ctx, e, "partition memset");
        const int g = std::min(A, 65535);
        medoid_pairs_kernel<<<g, 256, 0, st>>>(order, d_lo, d_sz, d_poff, A, pairs);
        if (PM > 0 && (rc = dist(pairs, PM, dm, true))) return rc;
        build_matrix_kernel<<<g, 256, 0, st>>>(order, d_lo, d_sz, d_poff, A, d_fresh, d_mbase, dm, pool, mlocal);
        medoid_sums_kernel<<<g, 256, 0, st>>>(order, d_lo, d_sz, d_poff, d_soff, A, dm, M, sums);
        medoid_argmin_kernel<<<g, 256, 0, st>>>(order, d_lo, d_sz, d_soff, A, sums, d_c);
        one_to_many_kernel<<<g, 256, 0, st>>>(order, d_lo, d_moff, A, d_c, pairs);
        if (PC > 0 && (rc = dist(pairs, PC, dc, false))) return rc;
        argmax_kernel<<<g, 256, 0, st>>>(order, d_lo, d_sz, d_moff, A, dc, d_c, M, d_l);
        one_to_many_kernel<<<g, 256, 0, st>>>(order, d_lo, d_moff, A, d_l, pairs);
        if (PC > 0 && (rc = dist(pairs, PC, dl, false))) return rc;
        argmax_kernel<<<g, 256, 0, st>>>(order, d_lo, d_sz, d_moff, A, dl, d_l, M, d_r);
        one_to_many_kernel<<<g, 256, 0, st>>>(order, d_lo, d_moff, A, d_r, pairs);
        if (PC > 0 && (rc = dist(pairs, PC, dr, false))) return rc;
        split_kernel<<<g, 1024, 0, st>>>(order, order_tmp, d_lo, d_sz, d_moff, A, dl, dr, d_l, d_r, M, d_nl);
        ctx->launches += 10;
        // the partitioned ranges back, in one copy (a copy per cluster cost
        // thousands of calls at the deep levels)
        e = cudaMemcpyAsync(order, order_tmp, N * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_check(ctx, e, "partition copy");
        std::vector<int32_t> nl(A), cc(A);
        if ((e = cudaMemcpyAsync(nl.data(), d_nl, A * sizeof(int32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(cc.data(), d_c, A * sizeof(int32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_check(ctx, e, "partition level readback");
        if ((rc = msa_ctx_check(ctx, stream))) return rc;
        std::vector<int32_t> next;
        for (int k = 0; k < A; ++k) {
            const int nd = active[k];
            center[nd] = cc[k];
            if (nl[k] <= 0 || nl[k] >= hsz[k])
                return set_error(ctx, MSA_EDATA,
                                 "msa_clam_partition: cluster of %d sequences did not split (duplicate sequences?)",
                                 hsz[k]);
            const int a = nn++, b = nn++;
            left[nd] = a;
            right[nd] = b;
            lo[a] = lo[nd];
            hi[a] = lo[nd] + nl[k];
            lo[b] = hi[a];
            hi[b] = hi[nd];
            for (int c : {a, b}) {
                node_mbase[c] = node_mbase[nd];      // a sub-cluster reads its parent's matrix
                node_mstride[c] = node_mstride[nd];
                parent[c] = nd;
                left[c] = right[c] = -1;
                center[c] = -1;
                if (hi[c] - lo[c] > 1) next.push_back(c);
            }
        }
        active.swap(next);
    }
    // singleton centres
    std::vector<int32_t> h_order(N);
    cudaError_t e = cudaMemcpyAsync(h_order.data(), order, N * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "partition order readback");
    for (int k = 0; k < nn; ++k)
        if (hi[k] - lo[k] == 1) center[k] = h_order[lo[k]];
    *n_nodes = nn;
    return MSA_OK;
}

}  // namespace msa

using namespace msa;

extern "C" {

msa_status msa_clam_partition(msa_ctx *ctx, const msa_seqset *s, int32_t *order, int32_t *lo, int32_t *hi,
                              int32_t *center, int32_t *left, int32_t *right, int32_t *parent, int32_t *n_nodes,
                              void *stream) {
    return clam_partition_run(ctx, s, nullptr, order, lo, hi, center, left, right, parent, n_nodes, stream);
}

msa_status msa_clam_partition_banded(msa_ctx *ctx, const msa_seqset *s, const void *state, const uint16_t *prof,
                                     float gamma, int32_t margin, int32_t *order, int32_t *lo, int32_t *hi,
                                     int32_t *center, int32_t *left, int32_t *right, int32_t *parent,
                                     int32_t *n_nodes, void *stream) {
    if (!ctx) return MSA_EINVAL;
    if (!state || !prof) return set_error(ctx, MSA_EINVAL, "msa_clam_partition_banded: null pointer");
    if (!s || s->alphabet != MSA_DNA)
        return set_error(ctx, MSA_EUNSUPPORTED, "msa_clam_partition_banded: the band network reads DNA 4-mers");
    const PartitionBand band{state, prof, gamma, margin};
    return clam_partition_run(ctx, s, &band, order, lo, hi, center, left, right, parent, n_nodes, stream);
}


}  // extern "C"

// gap_open < 0: linear gaps (gap per position); else a run of L gaps costs gap_open + L * gap
static msa_status merge_tree_run(msa_ctx *ctx, const msa_seqset *s, const int32_t *order, const int32_t *lo,
                                 const int32_t *hi, const int32_t *center, const int32_t *left, const int32_t *right,
                                 int32_t n_nodes, int32_t match, int32_t mismatch, int32_t gap, int32_t gap_open,
                                 int32_t *pos, int32_t *width, int32_t *score, void *stream,
                                 const int32_t *sub = nullptr, int32_t nsym = 0) {
    if (!ctx || !s) return MSA_EINVAL;
    if (!order || !lo || !hi || !center || !left || !right || !pos || !width || !score)
        return set_error(ctx, MSA_EINVAL, "msa_merge_tree: null pointer");
    const int N = s->n_seqs;
    if (N == 0) return MSA_OK;
    if (n_nodes != 2 * N - 1) return set_error(ctx, MSA_EINVAL, "msa_merge_tree: a binary tree over N leaves has 2N-1 nodes");
    cudaStream_t st = (cudaStream_t)stream;
    const uint8_t gap_code = s->alphabet == MSA_DNA ? 4 : 20;
    // heights and widths (host)
    std::vector<int32_t> height(n_nodes, 0);
    std::vector<int32_t> post;  // children before parents
    {
        std::vector<int32_t> stack{0};
        std::vector<int32_t> pre;
        while (!stack.empty()) {
            const int v = stack.back();
            stack.pop_back();
            pre.push_back(v);
            if (left[v] >= 0) {
                stack.push_back(left[v]);
                stack.push_back(right[v]);
            }
        }
        post.assign(pre.rbegin(), pre.rend());
    }
    if ((int)post.size() != n_nodes) return set_error(ctx, MSA_EINVAL, "msa_merge_tree: node table is not a tree");
    int hmax = 0;
    for (int v : post) {
        if (left[v] >= 0) height[v] = 1 + std::max(height[left[v]], height[right[v]]);
        hmax = std::max(hmax, height[v]);
        score[v] = -1;
        width[v] = left[v] >= 0 ? 0 : -1;
    }
    std::vector<int64_t> h_offs(N + 1);
    cudaError_t e = cudaMemcpyAsync(h_offs.data(), s->offs, (N + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "merge offsets readback");
    for (int v = 0; v < n_nodes; ++v)
        if (left[v] < 0) width[v] = (int32_t)(h_offs[center[v] + 1] - h_offs[center[v]]);
    init_pos_kernel<<<std::min(N, 65535), 256, 0, st>>>(s->offs, N, pos);
    ++ctx->launches;
    std::vector<std::vector<int32_t>> by_h(hmax + 1);
    for (int v : post)
        if (left[v] >= 0) by_h[height[v]].push_back(v);
    Arena base{ctx->ws, ctx->ws_bytes};
    for (int h = 1; h <= hmax; ++h) {
        const std::vector<int32_t> &ms = by_h[h];
        const int M = (int)ms.size();
        if (M == 0) continue;
        std::vector<int32_t> rc_h(2 * M), pairs_h(2 * M);
        std::vector<int64_t> roff(2 * M + 1), ooff(M + 1);
        roff[0] = 0;
        ooff[0] = 0;
        int maxw = 0;
        for (int m = 0; m < M; ++m) {
            const int v = ms[m];
            const int L = left[v], R = right[v];
            rc_h[2 * m] = center[L];
            rc_h[2 * m + 1] = center[R];
            roff[2 * m + 1] = roff[2 * m] + width[L];
            roff[2 * m + 2] = roff[2 * m + 1] + width[R];
            ooff[m + 1] = ooff[m] + width[L] + width[R];
            pairs_h[2 * m] = 2 * m;
            pairs_h[2 * m + 1] = 2 * m + 1;
            maxw = std::max(maxw, std::max(width[L], width[R]));
        }
        Arena ar = base;
        int32_t *d_rc = ar.take<int32_t>(2 * M), *d_pairs = ar.take<int32_t>(2 * M);
        int64_t *d_roff = ar.take<int64_t>(2 * M + 1), *d_ooff = ar.take<int64_t>(M + 1);
        uint8_t *rows = ar.take<uint8_t>(roff[2 * M] + 16);
        int32_t *maps = ar.take<int32_t>(roff[2 * M]);
        uint8_t *ops = ar.take<uint8_t>(ooff[M] + 16);
        int32_t *d_score = ar.take<int32_t>(M), *d_len = ar.take<int32_t>(M);
        // member segments of the children
        std::vector<int32_t> seg_lo(2 * M), seg_hi(2 * M);
        std::vector<int64_t> seg_map(2 * M), seg_start(2 * M + 1);
        seg_start[0] = 0;
        for (int m = 0; m < M; ++m)
            for (int side = 0; side < 2; ++side) {
                const int c = side ? right[ms[m]] : left[ms[m]];
                const int i = 2 * m + side;
                seg_lo[i] = lo[c];
                seg_hi[i] = hi[c];
                seg_map[i] = roff[i];
                seg_start[i + 1] = seg_start[i] + (hi[c] - lo[c]);
            }
        int32_t *d_seg_lo = ar.take<int32_t>(2 * M), *d_seg_hi = ar.take<int32_t>(2 * M);
        int64_t *d_seg_map = ar.take<int64_t>(2 * M), *d_seg_start = ar.take<int64_t>(2 * M + 1);
        if (!d_seg_start) return set_error(ctx, MSA_ENOMEM, "msa_merge_tree: workspace too small at height %d", h);
        msa_status rc;
        if ((rc = h2d(ctx, d_rc, rc_h, st)) || (rc = h2d(ctx, d_pairs, pairs_h, st)) ||
            (rc = h2d(ctx, d_roff, roff, st)) || (rc = h2d(ctx, d_ooff, ooff, st)) ||
            (rc = h2d(ctx, d_seg_lo, seg_lo, st)) || (rc = h2d(ctx, d_seg_hi, seg_hi, st)) ||
            (rc = h2d(ctx, d_seg_map, seg_map, st)) || (rc = h2d(ctx, d_seg_start, seg_start, st)))
            return rc;
        center_rows_kernel<<<std::min(2 * M, 65535), 256, 0, st>>>(s->codes, s->offs, pos, d_rc, d_roff, 2 * M,
                                                                   gap_code, rows);
        ++ctx->launches;
        rc = gap_open < 0 ? nw_run(ctx, ar, rows, d_roff, 2 * M, roff[2 * M], maxw, d_pairs, M, match, mismatch, gap,
                                   d_score, ops, d_ooff, d_len, st)
                          : nw_affine_run(ctx, ar, rows, d_roff, 2 * M, roff[2 * M], maxw, d_pairs, M, match,
                                          mismatch, gap_open, gap, d_score, ops, d_ooff, d_len, st, sub, nsym);
        if (rc) return rc;
        column_maps_kernel<<<(M + 127) / 128, 128, 0, st>>>(ops, d_ooff, d_len, d_roff, M, maps);
        const int64_t members = seg_start[2 * M];
        apply_maps_kernel<<<(int)std::min<int64_t>((members + 7) / 8, 65535), 256, 0, st>>>(
            order, s->offs, d_seg_lo, d_seg_hi, d_seg_map, 2 * M, (int32_t)members, d_seg_start, maps, pos);
        ctx->launches += 2;
        std::vector<int32_t> sc(M), ln(M);
        if ((e = cudaMemcpyAsync(sc.data(), d_score, M * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(ln.data(), d_len, M * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_check(ctx, e, "merge level readback");
        if ((rc = msa_ctx_check(ctx, stream))) return rc;
        for (int m = 0; m < M; ++m) {
            score[ms[m]] = sc[m];
            width[ms[m]] = ln[m];
        }
    }
    return MSA_OK;
}

extern "C" {

msa_status msa_merge_tree(msa_ctx *ctx, const msa_seqset *s, const int32_t *order, const int32_t *lo,
                          const int32_t *hi, const int32_t *center, const int32_t *left, const int32_t *right,
                          int32_t n_nodes, int32_t match, int32_t mismatch, int32_t gap, int32_t *pos,
                          int32_t *width, int32_t *score, void *stream) {
    return merge_tree_run(ctx, s, order, lo, hi, center, left, right, n_nodes, match, mismatch, gap, -1, pos, width,
                          score, stream);
}

msa_status msa_merge_tree_affine(msa_ctx *ctx, const msa_seqset *s, const int32_t *order, const int32_t *lo,
                                 const int32_t *hi, const int32_t *center, const int32_t *left,
                                 const int32_t *right, int32_t n_nodes, int32_t match, int32_t mismatch,
                                 int32_t gap_open, int32_t gap_ext, int32_t *pos, int32_t *width, int32_t *score,
                                 void *stream) {
    if (ctx && gap_open < 0) return set_error(ctx, MSA_EINVAL, "msa_merge_tree_affine: gap_open < 0");
    return merge_tree_run(ctx, s, order, lo, hi, center, left, right, n_nodes, match, mismatch, gap_ext, gap_open,
                          pos, width, score, stream);
}

msa_status msa_merge_tree_affine_sub(msa_ctx *ctx, const msa_seqset *s, const int32_t *order, const int32_t *lo,
                                     const int32_t *hi, const int32_t *center, const int32_t *left,
                                     const int32_t *right, int32_t n_nodes, const int32_t *sub, int32_t nsym,
                                     int32_t gap_open, int32_t gap_ext, int32_t *pos, int32_t *width, int32_t *score,
                                     void *stream) {
    if (ctx && gap_open < 0) return set_error(ctx, MSA_EINVAL, "msa_merge_tree_affine_sub: gap_open < 0");
    if (ctx && !sub) return set_error(ctx, MSA_EINVAL, "msa_merge_tree_affine_sub: null table");
    if (ctx && s && nsym < (s->alphabet == MSA_DNA ? 5 : 21))
        return set_error(ctx, MSA_EINVAL, "msa_merge_tree_affine_sub: the table must cover the gap code");
    return merge_tree_run(ctx, s, order, lo, hi, center, left, right, n_nodes, 0, 0, gap_ext, gap_open, pos, width,
                          score, stream, sub, nsym);
}

msa_status msa_msa_rows(msa_ctx *ctx, const msa_seqset *s, const int32_t *order, const int32_t *pos, int32_t W,
                        uint8_t *rows, void *stream) {
    if (!ctx || !s) return MSA_EINVAL;
    if (s->n_seqs == 0) return MSA_OK;
    if (!order || !pos || !rows || !s->ascii || W < 0) return set_error(ctx, MSA_EINVAL, "msa_msa_rows: bad argument");
    rows_kernel<<<std::min(s->n_seqs, 65535), 256, 0, (cudaStream_t)stream>>>(s->ascii, s->offs, order, pos,
                                                                              s->n_seqs, W, rows);
    ++ctx->launches;
    return cuda_check(ctx, cudaGetLastError(), "msa_msa_rows");
}

}  // extern "C"
