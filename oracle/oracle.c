/*
 * Plain CPU oracle for the batched alignment DP of MuSAlS (arXiv 2601.15458).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may call this file:
 * it is loaded by the tests, by __graft_entry__.smoke() and by the CPU
 * baseline leg of bench.py, and by nothing else.  It shares no code, header,
 * table or constant with the CUDA library; it works on raw byte strings.
 *
 * What it computes (each the plain definition, full matrix, no blocking):
 *
 *  oracle_lev  -- Levenshtein distance f of Alg. 1 ("Partition", section
 *                 "Clustering"): the unit-cost edit distance, written as the
 *                 Wagner-Fischer recurrence over the full (m+1) x (n+1) matrix
 *                    D[i][0] = i, D[0][j] = j,
 *                    D[i][j] = min(D[i-1][j-1] + [a_i != b_j],
 *                                  D[i-1][j] + 1, D[i][j-1] + 1).
 *
 *  oracle_nw   -- Needleman-Wunsch global alignment used for every merge
 *                 (section "Merging", step 2), as a minimum-cost DP with a
 *                 flat cost model (match, mismatch, gap), full matrix kept,
 *                 followed by a traceback from (m, n) that prefers, among the
 *                 moves that attain D[i][j], diagonal, then up (consume a_i
 *                 against a gap), then left (consume b_j against a gap).  The
 *                 paper does not fix a tie-break; this order is the reading
 *                 this project takes.  Row 0 forces left, column 0 forces up.
 *                 The script is emitted in forward order over the bytes
 *                 'M' (diagonal, equal symbols), 'X' (diagonal, different
 *                 symbols), 'D' (up) and 'I' (left).
 *
 *  oracle_nw_affine -- the same alignment with affine gap costs (Gotoh's
 *                 three matrices): a run of L gap positions costs
 *                 open + L * ext.  H[i][j] is the best cost of a_1..i against
 *                 b_1..j, F[i][j] the best that ends with an up move, E[i][j]
 *                 the best that ends with a left move:
 *                   F[i][j] = min(F[i-1][j] + ext, H[i-1][j] + open + ext)
 *                   E[i][j] = min(E[i][j-1] + ext, H[i][j-1] + open + ext)
 *                   H[i][j] = min(H[i-1][j-1] + c(a_i, b_j), F[i][j], E[i][j])
 *                 with H[0][0] = 0, H[i][0] = F[i][0] = open + i * ext,
 *                 H[0][j] = E[0][j] = open + j * ext, E[i][0] = F[0][j] = inf.
 *                 Traceback from (m, n) in state H: H takes the diagonal,
 *                 then F, then E (the first that attains); in F every step
 *                 emits 'D' and returns to H when opening the run there
 *                 attains, else the run goes on; E likewise with 'I'.  With
 *                 open = 0 this is the linear traceback exactly.  Row 0 forces
 *                 'I', column 0 forces 'D'.
 *
 *  oracle_nw_affine_sub -- oracle_nw_affine with c(a_i, b_j) read from a
 *                 substitution table over byte values (BLOSUM62 costs for
 *                 the paper's protein merges, section "Implementation").
 *
 *  oracle_lev_pairs / oracle_nw_pairs -- the same functions mapped over a
 *                 list of pairs, threads split the pair list only; each
 *                 pair's DP is the plain single-threaded one above.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

static inline int32_t min2(int32_t x, int32_t y) { return x < y ? x : y; }

int32_t oracle_lev(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n)
{
    const int64_t cols = n + 1;
    int32_t *D = (int32_t *)malloc((size_t)(m + 1) * (size_t)cols * sizeof(int32_t));
    if (!D) return -1;
    for (int64_t j = 0; j <= n; ++j) D[j] = (int32_t)j;
    for (int64_t i = 1; i <= m; ++i) {
        D[i * cols] = (int32_t)i;
        for (int64_t j = 1; j <= n; ++j) {
            int32_t sub = D[(i - 1) * cols + (j - 1)] + (a[i - 1] != b[j - 1] ? 1 : 0);
            int32_t del = D[(i - 1) * cols + j] + 1;
            int32_t ins = D[i * cols + (j - 1)] + 1;
            D[i * cols + j] = min2(sub, min2(del, ins));
        }
    }
    int32_t d = D[m * cols + n];
    free(D);
    return d;
}

/* The substitution cost c(x, y): sub[256 x + y] when a table is given,
 * else match / mismatch by byte equality. */
static inline int32_t subst_cost(const int32_t *sub, int32_t match, int32_t mismatch, uint8_t x, uint8_t y)
{
    return sub ? sub[256 * (int)x + (int)y] : (x == y ? match : mismatch);
}

static int32_t nw_affine_core(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n, const int32_t *sub,
                              int32_t match, int32_t mismatch, int32_t open, int32_t ext,
                              int32_t *score, uint8_t *ops, int64_t *ops_len);

/* Returns 0 on success, -1 on allocation failure.  ops must hold m + n bytes. */
int32_t oracle_nw_affine(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                         int32_t match, int32_t mismatch, int32_t open, int32_t ext,
                         int32_t *score, uint8_t *ops, int64_t *ops_len)
{
    return nw_affine_core(a, m, b, n, NULL, match, mismatch, open, ext, score, ops, ops_len);
}

/* The same with a substitution table: c(a_i, b_j) = sub[256 a_i + b_j]
 * (a 256 x 256 table over byte values); 'M' / 'X' still label identity. */
int32_t oracle_nw_affine_sub(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n, const int32_t *sub,
                             int32_t open, int32_t ext, int32_t *score, uint8_t *ops, int64_t *ops_len)
{
    return nw_affine_core(a, m, b, n, sub, 0, 0, open, ext, score, ops, ops_len);
}

static int32_t nw_affine_core(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n, const int32_t *sub,
                              int32_t match, int32_t mismatch, int32_t open, int32_t ext,
                              int32_t *score, uint8_t *ops, int64_t *ops_len)
{
    const int32_t INF = 1 << 29;
    const int64_t cols = n + 1;
    const size_t cells = (size_t)(m + 1) * (size_t)cols;
    int32_t *H = (int32_t *)malloc(cells * sizeof(int32_t));
    int32_t *E = (int32_t *)malloc(cells * sizeof(int32_t));
    int32_t *F = (int32_t *)malloc(cells * sizeof(int32_t));
    if (!H || !E || !F) {
        free(H); free(E); free(F);
        return -1;
    }
    H[0] = 0;
    E[0] = F[0] = INF;
    for (int64_t j = 1; j <= n; ++j) {
        H[j] = E[j] = open + (int32_t)j * ext;
        F[j] = INF;
    }
    for (int64_t i = 1; i <= m; ++i) {
        H[i * cols] = F[i * cols] = open + (int32_t)i * ext;
        E[i * cols] = INF;
        for (int64_t j = 1; j <= n; ++j) {
            const int64_t x = i * cols + j, up = (i - 1) * cols + j, lf = i * cols + j - 1;
            F[x] = min2(F[up] + ext, H[up] + open + ext);
            E[x] = min2(E[lf] + ext, H[lf] + open + ext);
            const int32_t c = subst_cost(sub, match, mismatch, a[i - 1], b[j - 1]);
            H[x] = min2(H[(i - 1) * cols + j - 1] + c, min2(F[x], E[x]));
        }
    }
    *score = H[m * cols + n];

    int64_t i = m, j = n, k = 0;
    int state = 0;                       /* 0: H, 1: F, 2: E */
    while (i > 0 || j > 0) {
        if (i == 0) { ops[k++] = 'I'; --j; continue; }
        if (j == 0) { ops[k++] = 'D'; --i; continue; }
        const int64_t x = i * cols + j;
        if (state == 0) {
            const int32_t c = subst_cost(sub, match, mismatch, a[i - 1], b[j - 1]);
            if (H[x] == H[(i - 1) * cols + j - 1] + c) {
                ops[k++] = (a[i - 1] == b[j - 1]) ? 'M' : 'X';
                --i; --j;
            } else if (H[x] == F[x]) {
                state = 1;
            } else {
                state = 2;
            }
        } else if (state == 1) {
            ops[k++] = 'D';
            if (F[x] == H[(i - 1) * cols + j] + open + ext) state = 0;
            --i;
        } else {
            ops[k++] = 'I';
            if (E[x] == H[i * cols + j - 1] + open + ext) state = 0;
            --j;
        }
    }
    for (int64_t p = 0, q = k - 1; p < q; ++p, --q) {
        uint8_t t = ops[p]; ops[p] = ops[q]; ops[q] = t;
    }
    *ops_len = k;
    free(H); free(E); free(F);
    return 0;
}

/* Returns 0 on success, -1 on allocation failure.  ops must hold m + n bytes. */
int32_t oracle_nw(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                  int32_t match, int32_t mismatch, int32_t gap,
                  int32_t *score, uint8_t *ops, int64_t *ops_len)
{
    const int64_t cols = n + 1;
    int32_t *D = (int32_t *)malloc((size_t)(m + 1) * (size_t)cols * sizeof(int32_t));
    if (!D) return -1;
    D[0] = 0;
    for (int64_t j = 1; j <= n; ++j) D[j] = D[j - 1] + gap;
    for (int64_t i = 1; i <= m; ++i) {
        D[i * cols] = D[(i - 1) * cols] + gap;
        for (int64_t j = 1; j <= n; ++j) {
            int32_t c = (a[i - 1] == b[j - 1]) ? match : mismatch;
            int32_t diag = D[(i - 1) * cols + (j - 1)] + c;
            int32_t up = D[(i - 1) * cols + j] + gap;
            int32_t left = D[i * cols + (j - 1)] + gap;
            D[i * cols + j] = min2(diag, min2(up, left));
        }
    }
    *score = D[m * cols + n];

    /* traceback, collected in reverse */
    int64_t i = m, j = n, k = 0;
    while (i > 0 || j > 0) {
        if (i > 0 && j > 0) {
            int32_t c = (a[i - 1] == b[j - 1]) ? match : mismatch;
            if (D[i * cols + j] == D[(i - 1) * cols + (j - 1)] + c) {
                ops[k++] = (a[i - 1] == b[j - 1]) ? 'M' : 'X';
                --i; --j;
                continue;
            }
        }
        if (i > 0 && (j == 0 || D[i * cols + j] == D[(i - 1) * cols + j] + gap)) {
            ops[k++] = 'D';
            --i;
            continue;
        }
        ops[k++] = 'I';
        --j;
    }
    /* reverse into forward order */
    for (int64_t x = 0, y = k - 1; x < y; ++x, --y) {
        uint8_t t = ops[x]; ops[x] = ops[y]; ops[y] = t;
    }
    *ops_len = k;
    free(D);
    return 0;
}

/* ---- pair lists, split over threads ---------------------------------- */

typedef struct {
    const uint8_t *arena;
    const int64_t *offs;
    const int32_t *pairs;
    int64_t lo, hi;
    int32_t *out;
    /* NW only */
    int32_t match, mismatch, gap;
    uint8_t *ops;
    const int64_t *ops_off;
    int64_t *ops_len;
    int32_t err;
} job_t;

static void *lev_worker(void *arg)
{
    job_t *J = (job_t *)arg;
    for (int64_t p = J->lo; p < J->hi; ++p) {
        int32_t x = J->pairs[2 * p], y = J->pairs[2 * p + 1];
        const uint8_t *a = J->arena + J->offs[x];
        const uint8_t *b = J->arena + J->offs[y];
        int32_t d = oracle_lev(a, J->offs[x + 1] - J->offs[x], b, J->offs[y + 1] - J->offs[y]);
        if (d < 0) J->err = 1;
        J->out[p] = d;
    }
    return NULL;
}

static void *nw_worker(void *arg)
{
    job_t *J = (job_t *)arg;
    for (int64_t p = J->lo; p < J->hi; ++p) {
        int32_t x = J->pairs[2 * p], y = J->pairs[2 * p + 1];
        const uint8_t *a = J->arena + J->offs[x];
        const uint8_t *b = J->arena + J->offs[y];
        if (oracle_nw(a, J->offs[x + 1] - J->offs[x], b, J->offs[y + 1] - J->offs[y],
                      J->match, J->mismatch, J->gap, &J->out[p],
                      J->ops + J->ops_off[p], &J->ops_len[p]) != 0)
            J->err = 1;
    }
    return NULL;
}

static int32_t run_jobs(job_t *proto, int64_t P, int nthreads, void *(*fn)(void *))
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 1024) nthreads = 1024;
    if ((int64_t)nthreads > P) nthreads = (int)(P > 0 ? P : 1);
    job_t jobs[1024];
    pthread_t th[1024];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = *proto;
        jobs[t].lo = P * t / nthreads;
        jobs[t].hi = P * (t + 1) / nthreads;
        jobs[t].err = 0;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, fn, &jobs[t]);
    fn(&jobs[0]);
    int32_t err = jobs[0].err;
    for (int t = 1; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        err |= jobs[t].err;
    }
    return err ? -1 : 0;
}

int32_t oracle_lev_pairs(const uint8_t *arena, const int64_t *offs, const int32_t *pairs,
                         int64_t P, int32_t *out, int32_t nthreads)
{
    job_t J;
    memset(&J, 0, sizeof J);
    J.arena = arena; J.offs = offs; J.pairs = pairs; J.out = out;
    return run_jobs(&J, P, nthreads, lev_worker);
}

int32_t oracle_nw_pairs(const uint8_t *arena, const int64_t *offs, const int32_t *pairs,
                        int64_t P, int32_t match, int32_t mismatch, int32_t gap,
                        int32_t *score, uint8_t *ops, const int64_t *ops_off,
                        int64_t *ops_len, int32_t nthreads)
{
    job_t J;
    memset(&J, 0, sizeof J);
    J.arena = arena; J.offs = offs; J.pairs = pairs; J.out = score;
    J.match = match; J.mismatch = mismatch; J.gap = gap;
    J.ops = ops; J.ops_off = ops_off; J.ops_len = ops_len;
    return run_jobs(&J, P, nthreads, nw_worker);
}
