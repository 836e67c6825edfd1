/*
 * msa.h -- C ABI of the GB300 (sm_103a) batched alignment DP library that
 * serves the hot path of MuSAlS (arXiv 2601.15458).
 *
 * The paper builds its guide tree by Alg. 1 ("Partition", section
 * "Clustering"), which calls the Levenshtein distance f on one-to-many
 * batches, and merges clusters bottom-up (section "Merging") by aligning two
 * cluster centers with Needleman-Wunsch and noting where gaps go.  This
 * library computes those two DPs in batches on one GPU.
 *
 * Conventions shared by every call
 *  - All array arguments are DEVICE pointers owned by the caller, unless the
 *    comment says "host".  The library never frees them.  It allocates only
 *    its context workspace (msa_ctx_create) and never allocates inside a call.
 *  - Every call is asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *    default stream) and returns a status synchronously for argument errors
 *    (MSA_EINVAL: null pointer, negative count, unsupported alphabet, a size
 *    beyond the workspace -> MSA_ENOMEM).  Errors found by a kernel (index out
 *    of range, a symbol outside the alphabet, a length above max_len) are
 *    recorded in a device status word; msa_ctx_check() synchronises the
 *    stream and returns them.  Kernels never trap and never wait without a
 *    bound.
 *  - A pair (a, b) puts a on the DP rows (i = 0..m) and b on the columns
 *    (j = 0..n).  Levenshtein is symmetric; NW output is defined for the
 *    order given.
 *  - Empty sequences are allowed; P = 0 is a no-op returning MSA_OK.
 *  - Calls on one context share its workspace, its side streams (on which
 *    independent kernels of one call run side by side, joined back into
 *    `stream` before the call's work ends) and its error word: order them
 *    on the GPU (one stream, or events) and make them from one host thread
 *    at a time.  Work that must overlap takes one context per stream.
 *    msa_lev_batch_noalloc has no context and its own rule (below).
 */
#ifndef MSA_H
#define MSA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct msa_ctx msa_ctx;
typedef int32_t msa_status;

#define MSA_OK            0
#define MSA_EINVAL        1  /* bad argument (host-detected)                          */
#define MSA_ENOMEM        2  /* workspace too small for this call / allocation failed */
#define MSA_ECUDA         3  /* a CUDA runtime call failed                             */
#define MSA_ETIMEOUT      4  /* a bounded device wait ran out                          */
#define MSA_EUNSUPPORTED  5  /* configuration not built into this library              */
#define MSA_EDATA         6  /* device-detected bad data (index, symbol, length)       */

#define MSA_DNA      0       /* A C G T            -> codes 0..3,  gap code 4  */
#define MSA_PROTEIN  1       /* ACDEFGHIKLMNPQRSTVWY -> codes 0..19, gap code 20 */

/* Edit-script bytes written by msa_nw_align_batch (forward order). */
#define MSA_OP_MATCH     'M' /* diagonal, a_i == b_j                  */
#define MSA_OP_MISMATCH  'X' /* diagonal, a_i != b_j                  */
#define MSA_OP_DEL       'D' /* up: a_i against a gap (consumes a)    */
#define MSA_OP_INS       'I' /* left: b_j against a gap (consumes b)  */

/*
 * A set of sequences in one arena.  Sequence s occupies arena positions
 * [offs[s], offs[s+1]).  `ascii` holds residues (one byte each, upper case);
 * msa_pack() turns it into `codes` (one byte per position, 0..sigma-1) and
 * `planes` (bit planes: for arena word w = position / 32 and plane p < B,
 * planes[w * B + p] bit (position % 32) is bit p of the code; B = 2 for DNA,
 * 5 for protein).  Both outputs are caller-allocated with the sizes given by
 * msa_code_bytes() and msa_plane_words().
 */
typedef struct msa_seqset {
    const uint8_t *ascii;   /* device, >= total bytes, 16-byte aligned             */
    const int64_t *offs;    /* device, n_seqs + 1 entries, offs[0] = 0, ascending    */
    uint8_t *codes;         /* device, msa_code_bytes(total) bytes (written by pack) */
    uint32_t *planes;       /* device, msa_plane_words(total, alphabet) words        */
    int64_t total;          /* host copy of offs[n_seqs]                             */
    int32_t n_seqs;
    int32_t alphabet;       /* MSA_DNA or MSA_PROTEIN                                */
    int32_t max_len;        /* host: bound on every length, checked on the device    */
    int32_t reserved;
} msa_seqset;

/* ---- context ------------------------------------------------------------ */

/* Creates a context on `device` with `workspace_bytes` of device scratch
 * (<= 0 picks 1 GiB).  The workspace bounds the batch sizes of later calls. */
msa_status msa_ctx_create(msa_ctx **out, int32_t device, int64_t workspace_bytes);
void msa_ctx_destroy(msa_ctx *ctx);
/* Synchronises `stream`, returns and clears the first device-recorded error. */
msa_status msa_ctx_check(msa_ctx *ctx, void *stream);
/* Text of the last error recorded on this context (host string, owned by ctx). */
const char *msa_last_error(const msa_ctx *ctx);
/* Library version string, e.g. "msa-gb300 0.1 sm_103a". */
const char *msa_version(void);

/* Launch accounting: when enabled, each DP call brackets its DP kernels (the
 * distance / alignment kernels, not the scheduling ones) with CUDA events on
 * its stream.  msa_prof_read waits for those events and returns the summed
 * milliseconds and the number of kernels this context launched; reset != 0
 * zeroes both. */
msa_status msa_prof_enable(msa_ctx *ctx, int32_t on);
msa_status msa_prof_read(msa_ctx *ctx, double *dp_kernel_ms, int64_t *launches, int32_t reset);

/* ---- sizes (pure host arithmetic) --------------------------------------- */
int64_t msa_code_bytes(int64_t total);
int64_t msa_plane_words(int64_t total, int32_t alphabet);
/* Workspace bytes msa_lev_batch needs for P pairs over n_seqs sequences. */
int64_t msa_lev_workspace_bytes(int64_t P, int32_t n_seqs);

/* ---- A1: packed-sequence loader ----------------------------------------- */
/*
 * Reads the ASCII arena once with 16-byte loads and writes the byte codes and
 * the bit planes; checks every residue against the alphabet and every length
 * against max_len (MSA_EDATA via msa_ctx_check otherwise).
 */
msa_status msa_pack(msa_ctx *ctx, const msa_seqset *s, void *stream);

/* ---- A2/A3/A7: batched Levenshtein distance ----------------------------- */
/*
 * d_out[p] = f(seq[pairs[2p]], seq[pairs[2p+1]]), the unit-cost edit
 * distance f of Alg. 1 (section "Clustering"), exactly.
 * pairs: device int32 [P][2]; d_out: device int32 [P].  P < 2^31.
 * Pairs are grouped by their first index on the device; a warp shares the
 * bit-vector match masks of that first sequence, so listing many pairs with
 * the same first index (one-to-many, as Alg. 1 does) is the fast case.
 * Needs msa_lev_workspace_bytes(P, n_seqs) of workspace.
 */
msa_status msa_lev_batch(msa_ctx *ctx, const msa_seqset *s, const int32_t *pairs,
                         int64_t P, int32_t *d_out, void *stream);

/*
 * d_out[i] = f(seq[query], seq[idx[i]]) for i < n: one query against many
 * targets, the batch shape of Alg. 1's c, l and r distances (the query's
 * match masks are built once per warp and shared by its lanes).  idx: device
 * int32 [n]; an index outside [0, n_seqs) is reported as MSA_EDATA by
 * msa_ctx_check, query outside it as MSA_EINVAL.  Same kernels and results as
 * msa_lev_batch on the pairs (query, idx[i]).  Needs
 * msa_lev_one_to_many_workspace_bytes(n, n_seqs) of workspace.
 */
msa_status msa_lev_one_to_many(msa_ctx *ctx, const msa_seqset *s, int32_t query, const int32_t *idx, int64_t n,
                               int32_t *d_out, void *stream);
int64_t msa_lev_one_to_many_workspace_bytes(int64_t n, int32_t n_seqs);

/* Selects the kernel schedule of msa_lev_batch (the target-count thresholds
 * between the kernels, targets per task) by running this batch under each
 * candidate and timing it with CUDA events; the fastest is kept in ctx for
 * later calls.  d_out ends up holding the distances, as after
 * msa_lev_batch.  Synchronises `stream`. */
msa_status msa_lev_autotune(msa_ctx *ctx, const msa_seqset *s, const int32_t *pairs,
                            int64_t P, int32_t *d_out, void *stream);

/*
 * The schedule msa_lev_batch uses, as 4 ints:
 *   [0] lane_min_targets: a query (first index) with at least this many
 *       targets gets a warp of its own, one target per lane (default 32);
 *   [1] slot_min_targets: a query with fewer targets than [0] but at least
 *       this many shares a warp with up to 7 others, the 32 lanes taking the
 *       targets of all of them (default 2; >= [0] turns this kernel off);
 *   [2] lane_per_task: targets per warp task of the first kernel (0: from
 *       the batch size);
 *   [3] warp_per_task: targets per task of the warp-per-pair kernel, which
 *       takes every other query (default 4).
 * Any choice gives the same distances.  msa_lev_tune_set leaves an entry
 * unchanged where the value is negative (0 is accepted only for [2]);
 * MSA_EINVAL for [0], [1] or [3] equal to 0.  Host-only calls.
 */
msa_status msa_lev_tune_get(msa_ctx *ctx, int32_t *tune4);
msa_status msa_lev_tune_set(msa_ctx *ctx, const int32_t *tune4);

/*
 * Allocation-free variant of msa_lev_batch (the paper has no counterpart;
 * this is a deployment convenience).  For callers that cannot allocate
 * device memory or create a context: code running under another
 * framework's memory budget (a caching allocator that holds the free device
 * memory), plug-ins that may not allocate after start-up, loops that cannot
 * take an allocation's implicit synchronisation.  It computes the same
 * d_out[p] = f(seq[pairs[2p]], seq[pairs[2p+1]]) as msa_lev_batch, with no
 * context and no cudaMalloc / cudaFree / allocating library call: its scratch
 * is one fixed device array inside the library (about 5.8 MB, held on every
 * GPU that loads the library until the process exits).
 *  - Limits: P <= 262144 pairs and 1 <= n_seqs <= 65536 per call; larger
 *    calls, null pointers and an unknown alphabet return MSA_EINVAL, and
 *    max_len < 0 MSA_EINVAL, max_len > 16384 MSA_EUNSUPPORTED, before
 *    anything is enqueued.
 *  - The first call on a device looks the array up with that device
 *    current (cudaGetSymbolAddress), sets kernel attributes and queries
 *    occupancies; make it before any stream capture.  This set-up belongs to
 *    the device's CUDA context: after the context is destroyed and recreated
 *    (cudaDeviceReset), the next call redoes it, so that call too should
 *    come before any capture.
 *  - Every call shares the array: calls that overlap on the GPU (other
 *    streams or threads) race; issue them on one stream.
 *  - No error word: a pair with an index outside the set, or whose first
 *    sequence is longer than s->max_len, gets d_out[p] = -1.
 */
msa_status msa_lev_batch_noalloc(const msa_seqset *s, const int32_t *pairs, int64_t P, int32_t *d_out,
                                 void *stream);

/* ---- A4: banded Levenshtein with an exactness certificate --------------- */
/*
 * Same result as msa_lev_batch: d_out[p] = f(a, b) exactly.  Each pair
 * starts from the Ukkonen band k0[p] (device int32 [P]): the DP is restricted
 * to the diagonals with |j - i| + |(n - j) - (m - i)| <= k, which contain
 * every optimal path whenever f(a, b) <= k.  The banded result is accepted
 * only when it is <= the band it was computed with; otherwise the band
 * grows to min(result, 2k + 1) (at most a doubling; the result is itself an
 * upper bound of f, so that band always certifies) for up to 3 attempts, and
 * pairs still pending, or whose band reaches the whole matrix (or the
 * largest window the library's kernels hold in registers), are computed by the full
 * DP of msa_lev_batch.  k_used_out[p] (device int32 [P]) receives the band that
 * certified the pair (>= k0[p]), or max(m, n) when the full DP decided it.
 * Any k0 (even 0) gives the exact distance; a good k0 only saves work.
 * Needs msa_lev_banded_workspace_bytes(P, n_seqs) of workspace.
 */
msa_status msa_lev_banded_batch(msa_ctx *ctx, const msa_seqset *s, const int32_t *pairs, int64_t P,
                                const int32_t *k0, int32_t *d_out, int32_t *k_used_out, void *stream);
int64_t msa_lev_banded_workspace_bytes(int64_t P, int32_t n_seqs);

/* ---- A8-A10: learned band proposer -------------------------------------- */
/*
 * The paper has no learned component; this proposer only chooses the
 * starting band k0 of msa_lev_banded_batch, whose certificate keeps every
 * distance exact.  Features: 4-mer count profiles of DNA (256 bins, k-mer
 * s0 s1 s2 s3 of codes A=0 C=1 G=2 T=3 in bin 64 s0 + 16 s1 + 4 s2 + s3,
 * counted over the len - 3 windows), and for a pair (a, b) the 256 values
 * (c_a - c_b)^2 / ((len_a + len_b) / 2), squared and divided in fp32 and
 * rounded to bf16.
 * Network: y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 with W1 128x256,
 * W2 64x128, W3 1x64; bf16 weights and activations, fp32 accumulation on the
 * tensor cores; target y = f(a, b) / max(m, n).
 *
 * Model state: one device buffer of msa_mlp_state_bytes() bytes that starts
 * with the msa_mlp_num_params() fp32 parameters in the order
 * W1 (out-major, [128][256]), b1, W2 ([64][128]), b2, W3 [64], b3, and ends
 * with 64 floats of band calibration ([0] = 1 when fitted, [1..33] the
 * knots, see msa_band_calibrate; all zero = none); the rest (Adam moments,
 * gradient, bf16 copies) is private.  After writing the parameters, call
 * msa_mlp_sync() (bf16 copies, zero moments and step; the calibration is
 * left as it is).
 */
int32_t msa_mlp_num_params(void);
int64_t msa_mlp_state_bytes(void);
msa_status msa_mlp_sync(msa_ctx *ctx, void *state, void *stream);
/* prof: device uint16 [n_seqs][256]; DNA sets only, lengths <= 65535. */
msa_status msa_kmer_profile(msa_ctx *ctx, const msa_seqset *s, uint16_t *prof, void *stream);
/* X: device bf16 (as uint16 bits) [P][256], the pair features of `pairs`. */
msa_status msa_pair_features(msa_ctx *ctx, const msa_seqset *s, const uint16_t *prof, const int32_t *pairs,
                             int64_t P, uint16_t *X, void *stream);
/* yhat[p] = network output for feature row p (X bf16 [P][256]). */
msa_status msa_mlp_forward(msa_ctx *ctx, const void *state, const uint16_t *X, int64_t P, float *yhat,
                           void *stream);
/*
 * One Adam step (Kingma & Ba; beta1 0.9, beta2 0.999, eps 1e-8, fp32 master
 * weights, bf16 copies refreshed) on the minibatch rows idx[0..B) of
 * (X bf16 [N][256], y fp32 [N]; indices outside [0, N) count as zero rows),
 * minimising the mean pinball loss of quantile tau:
 * rho(r) = tau r for r = y - yhat > 0, (tau - 1) r otherwise.
 * loss_out (device float, may be null) receives the batch loss before the
 * update.  lr = 0 computes loss and gradient only (the gradient is then left
 * in the state and can be read with msa_mlp_read_grad).
 * Needs msa_mlp_train_workspace_bytes(B) of workspace.
 */
msa_status msa_mlp_train_step(msa_ctx *ctx, void *state, const uint16_t *X, const float *y, int64_t N,
                              const int32_t *idx, int32_t B, float lr, float tau, float *loss_out, void *stream);
int64_t msa_mlp_train_workspace_bytes(int32_t B);
/* Copies the current gradient (fp32, parameter order) to grad_out and zeroes it. */
msa_status msa_mlp_read_grad(msa_ctx *ctx, void *state, float *grad_out, void *stream);
/*
 * Fused features + forward + band policy for each pair:
 *   yhat[p] = network output, k_out[p] = max(|m - n|,
 *   ceil((1 + gamma) * c * max(m, n)) + margin),
 * with c = max(yhat, 0), or c = c(yhat) of msa_band_calibrate when the state
 * holds a calibration (both products rounded to fp32 in that order).
 * prof from msa_kmer_profile of the same set.
 */
msa_status msa_band_predict(msa_ctx *ctx, const void *state, const msa_seqset *s, const uint16_t *prof,
                            const int32_t *pairs, int64_t P, float gamma, int32_t margin, float *yhat,
                            int32_t *k_out, void *stream);
/*
 * Band calibration (this library's addition to the learned band: the
 * network is trained on one population of pairs and its output need not be
 * a calibrated quantile on another).  From N held-out pairs with network
 * outputs yhat[j] and true y[j] = f / max(m, n) (device fp32 arrays), fits
 * the 33 knots of a monotone map c at yhat = 0, 1/32, ..., 1 and stores them
 * in the state:
 *   bin(yhat) = min(32, max(0, floor(yhat * 32 + 0.5)))   (fp32),
 *   knot i = the tau-quantile of min(1, max(0, y)) over the pairs of bin i,
 *     the smallest v with #{y <= v} >= ceil(tau * n_i) (n_i >= 16; a bin with
 *     fewer pairs keeps i / 32),
 *   then knot i = max(knot 0 .. knot i).
 * c(yhat) interpolates the knots linearly at min(1, max(0, yhat)) * 32 (fp32,
 * each operation rounded).  Every distance stays exact whatever the band
 * (the certificate of msa_lev_banded_batch decides), so the map only moves
 * the starting band.  N = 0 removes the calibration.  tau in (0, 1].
 * One single-block kernel, 5 passes over the inputs per knot; asynchronous.
 */
msa_status msa_band_calibrate(msa_ctx *ctx, void *state, const float *yhat, const float *y, int64_t N, float tau,
                              void *stream);

/* ---- A5/A6: Needleman-Wunsch with traceback ----------------------------- */
/*
 * Global alignment of every pair (section "Merging", step 2: align the two
 * children's centers and note where gaps were added).  Minimum-cost DP with
 * a flat cost model:
 *   D[i][0] = i*gap, D[0][j] = j*gap,
 *   D[i][j] = min(D[i-1][j-1] + (a_i == b_j ? match : mismatch),
 *                 D[i-1][j] + gap, D[i][j-1] + gap).
 * Among the moves that attain D[i][j] the traceback takes diagonal, then up
 * (a_i against a gap), then left (b_j against a gap); the paper fixes no
 * tie-break and this order is the one this library defines.
 * Sequences are byte strings compared by equality (any byte values: packed
 * codes, gapped rows with a gap code, or ASCII).  Sequence s is
 * codes[offs[s] .. offs[s+1]); offs has n_seqs + 1 entries within [0, total].
 * pairs: device int32 [P][2] (a = pairs[2p], b = pairs[2p+1]).
 * Outputs (device): score_out[p] = D[m][n]; ops_out[ops_off[p] ..
 * ops_off[p] + ops_len_out[p]) = the edit script in forward order over the
 * MSA_OP_* bytes.  ops_off (device, caller-filled) must give each pair at
 * least m + n bytes.  max_len (host) bounds every length; the call uses
 * msa_nw_workspace_bytes(max_len, warps) of workspace for as many warps as
 * fit (at least 4), so it fails with MSA_ENOMEM only when 4 do not fit.
 */
msa_status msa_nw_align_batch(msa_ctx *ctx, const uint8_t *codes, const int64_t *offs, int32_t n_seqs,
                              int64_t total, int32_t max_len, const int32_t *pairs, int64_t P,
                              int32_t match, int32_t mismatch, int32_t gap, int32_t *score_out,
                              uint8_t *ops_out, const int64_t *ops_off, int32_t *ops_len_out,
                              void *stream);
/* Workspace bytes msa_nw_align_batch needs to run `warps` pairs at once. */
int64_t msa_nw_workspace_bytes(int32_t max_len, int32_t warps);
/*
 * The same alignment with affine gap costs (Gotoh; the paper's merges use
 * affine gaps with open = 10 x extend, section "Implementation"): a run of L
 * gap positions costs gap_open + L * gap_ext (gap_open >= 0, gap_ext >= 1);
 * substitutions cost match / mismatch.  Traceback from (m, n): diagonal, then
 * up, then left (the first that attains), and a gap run closes where opening
 * it attains, else it extends; with gap_open = 0 the result is exactly
 * msa_nw_align_batch's with gap = gap_ext.  Arguments and outputs as in
 * msa_nw_align_batch; per-warp scratch is about twice as large.
 */
msa_status msa_nw_align_batch_affine(msa_ctx *ctx, const uint8_t *codes, const int64_t *offs, int32_t n_seqs,
                                     int64_t total, int32_t max_len, const int32_t *pairs, int64_t P,
                                     int32_t match, int32_t mismatch, int32_t gap_open, int32_t gap_ext,
                                     int32_t *score_out, uint8_t *ops_out, const int64_t *ops_off,
                                     int32_t *ops_len_out, void *stream);

/*
 * The affine alignment with a substitution table: a diagonal move costs
 * sub[nsym * a_i + b_j] (device int32 [nsym][nsym], row-major by code,
 * nsym <= 32, entries may be negative) instead of match / mismatch; the
 * paper's protein merges use BLOSUM62 (section "Implementation"), as costs
 * -score.  'M' / 'X' still mark identical / different codes.  A pair with a
 * code >= nsym is reported as MSA_EDATA by msa_ctx_check and left unwritten.
 * Gaps, traceback, arguments and outputs as in msa_nw_align_batch_affine.
 */
msa_status msa_nw_align_batch_affine_sub(msa_ctx *ctx, const uint8_t *codes, const int64_t *offs, int32_t n_seqs,
                                         int64_t total, int32_t max_len, const int32_t *pairs, int64_t P,
                                         const int32_t *sub, int32_t nsym, int32_t gap_open, int32_t gap_ext,
                                         int32_t *score_out, uint8_t *ops_out, const int64_t *ops_off,
                                         int32_t *ops_len_out, void *stream);

/* ---- NW split at k-mer anchors (section "Discussion and Future Work") ---- */
/*
 * The paper names splitting long alignments at k-mer anchors as a way to
 * scale to longer sequences without fixing a method; this library's method:
 *   anchors: every (i, j) where the k-mer a[i .. i+k) occurs exactly once in
 *     a and exactly once in b and b[j .. j+k) is that k-mer;
 *   chain: the longest chain of anchors increasing in i and j, by patience
 *     sorting over the anchors in i order (an anchor replaces the first tail
 *     whose j is >= its own and links to the tail before it);
 *   blocks, along the chain: an anchor on the current block's diagonal that
 *     starts inside it or right after it extends the block to its own end,
 *     one that starts at or after the block's end in both sequences starts a
 *     new block, any other is dropped;
 *   each block is aligned as a run of matches ('M', cost match per column),
 *     every segment between blocks (and before the first, after the last) by
 *     msa_nw_align_batch with the same costs; scripts and costs are joined.
 * The cost is an upper bound of the NW optimum (equal to it when an optimal
 * alignment passes through every block); without anchors it is the NW
 * result.  k in 1..256; k-mers are compared as bytes (any byte values).
 * Sequences, pairs and outputs as in msa_nw_align_batch (a bad pair is
 * reported by msa_ctx_check as there and its outputs are left unwritten).
 * The workspace holds a hash table of 2^ceil(log2(2 max_len)) 20-byte slots
 * and 16 max_len bytes per resident pair block, then the segments.
 * Synchronous: the host reads the segment count, bytes and longest segment
 * once per call, then the segment alignments run as one msa_nw_align_batch.
 */
msa_status msa_nw_align_batch_anchored(msa_ctx *ctx, const uint8_t *codes, const int64_t *offs, int32_t n_seqs,
                                       int64_t total, int32_t max_len, const int32_t *pairs, int64_t P, int32_t k,
                                       int32_t match, int32_t mismatch, int32_t gap, int32_t *score_out,
                                       uint8_t *ops_out, const int64_t *ops_off, int32_t *ops_len_out, void *stream);
/* The same split under affine gaps (section "Implementation"): segments by
 * msa_nw_align_batch_affine (a gap run of L costs gap_open + L gap_ext;
 * gap_open >= 0), a block residue costs match.  The _sub variant takes the
 * substitution table of msa_nw_align_batch_affine_sub (device int32
 * [nsym][nsym], nsym <= 32; a code >= nsym is reported as MSA_EDATA by
 * msa_ctx_check): segments by that call, a block residue x costs
 * sub[x][x].  Both are defined by this library (the paper fixes no anchored
 * method); arguments and outputs as msa_nw_align_batch_anchored. */
msa_status msa_nw_align_batch_anchored_affine(msa_ctx *ctx, const uint8_t *codes, const int64_t *offs,
                                              int32_t n_seqs, int64_t total, int32_t max_len, const int32_t *pairs,
                                              int64_t P, int32_t k, int32_t match, int32_t mismatch, int32_t gap_open,
                                              int32_t gap_ext, int32_t *score_out, uint8_t *ops_out,
                                              const int64_t *ops_off, int32_t *ops_len_out, void *stream);
msa_status msa_nw_align_batch_anchored_affine_sub(msa_ctx *ctx, const uint8_t *codes, const int64_t *offs,
                                                  int32_t n_seqs, int64_t total, int32_t max_len, const int32_t *pairs,
                                                  int64_t P, int32_t k, const int32_t *sub, int32_t nsym,
                                                  int32_t gap_open, int32_t gap_ext, int32_t *score_out,
                                                  uint8_t *ops_out, const int64_t *ops_off, int32_t *ops_len_out,
                                                  void *stream);

/* ---- A11: guide tree by Alg. 1 (Partition) ------------------------------ */
/*
 * Builds the binary cluster tree of Alg. 1 (section "Clustering") over the
 * whole set, every cluster split until it is a singleton.  For a cluster C:
 * centre c = geometric median of C, taken over all of C when |C| <= 256 and
 * otherwise over the 256 members at positions floor(k |C| / 256),
 * k = 0..255, of C sorted by index (the paper allows "a smaller subset"
 * without fixing one; this is the rule of this library); l = argmax f(c, x),
 * r = argmax f(l, x) over x in C; L = {x : f(l, x) <= f(r, x)},
 * R = {x : f(r, x) < f(l, x)}.  Every argmin / argmax tie goes to the
 * smallest index.  Sequences must be distinct (the paper de-duplicates its
 * input first); a cluster that does not split returns MSA_EDATA.
 * Outputs: order (device int32 [n]) lists the sequences so that every node k
 * covers order[lo[k] .. hi[k]) and each node's range is its left child's
 * range followed by its right child's; lo, hi, center, left, right, parent
 * are HOST int32 arrays with room for 2n - 1 nodes, in breadth-first order
 * (node 0 = root; -1 = none).  *n_nodes (host) receives 2n - 1.
 * Synchronous: the host reads the left-child sizes once per tree level.
 * A cluster of at most 256 members keeps the distances of its medoid batch
 * (all its pairs) as a matrix in the workspace (up to 256 n_seqs int32 in
 * all, at most a quarter of the free workspace); it and its sub-clusters
 * read every later distance from it instead of computing it again.
 */
msa_status msa_clam_partition(msa_ctx *ctx, const msa_seqset *s, int32_t *order, int32_t *lo, int32_t *hi,
                              int32_t *center, int32_t *left, int32_t *right, int32_t *parent,
                              int32_t *n_nodes, void *stream);
/*
 * The same tree as msa_clam_partition, with the medoid batches of Alg. 1
 * started from the band the network proposes (msa_band_predict with gamma,
 * margin) and computed by the certified banded DP of msa_lev_banded_batch,
 * so every distance, and the tree, equals the full-DP result.  The c, l and
 * r batches run on the full DP: their points lie far from most of the
 * cluster, so their bands would cover most of each matrix.  state: network state (msa_mlp_state_bytes);
 * prof: msa_kmer_profile of s.  DNA sets only (MSA_EUNSUPPORTED otherwise).
 * The learned band is this library's addition, not the paper's.
 */
msa_status msa_clam_partition_banded(msa_ctx *ctx, const msa_seqset *s, const void *state, const uint16_t *prof,
                                     float gamma, int32_t margin, int32_t *order, int32_t *lo, int32_t *hi,
                                     int32_t *center, int32_t *left, int32_t *right, int32_t *parent,
                                     int32_t *n_nodes, void *stream);

/* ---- A12: bottom-up merge along the guide tree -------------------------- */
/*
 * Section "Merging": a leaf is the one-row MSA of its sequence; a parent
 * aligns its two children's centres, each as the gapped row it has in its
 * child's MSA, by NW (msa_nw_align_batch semantics; the gap is an ordinary
 * symbol, gap code 4 for DNA and 20 for protein), inserts an all-gap column
 * into the left child's rows for every MSA_OP_INS and into the right child's
 * rows for every MSA_OP_DEL, and stacks the left rows over the right rows.
 * All merges of one tree height run as one batch.
 * Inputs: the tree of msa_clam_partition (order device, the rest host).
 * Outputs: pos (device int32, one entry per arena position): pos[offs[s]+k]
 * = column of residue k of sequence s in the root MSA; width / score (HOST
 * int32 [n_nodes]): MSA width of every node and, for internal nodes, the NW
 * cost of its merge (-1 for leaves).  Synchronous (one read-back per height).
 */
msa_status msa_merge_tree(msa_ctx *ctx, const msa_seqset *s, const int32_t *order, const int32_t *lo,
                          const int32_t *hi, const int32_t *center, const int32_t *left, const int32_t *right,
                          int32_t n_nodes, int32_t match, int32_t mismatch, int32_t gap, int32_t *pos,
                          int32_t *width, int32_t *score, void *stream);
/* The same merge with affine gap costs (msa_nw_align_batch_affine's model:
 * a run of L gaps costs gap_open + L * gap_ext) for the center alignments. */
msa_status msa_merge_tree_affine(msa_ctx *ctx, const msa_seqset *s, const int32_t *order, const int32_t *lo,
                                 const int32_t *hi, const int32_t *center, const int32_t *left,
                                 const int32_t *right, int32_t n_nodes, int32_t match, int32_t mismatch,
                                 int32_t gap_open, int32_t gap_ext, int32_t *pos, int32_t *width, int32_t *score,
                                 void *stream);
/* The same merge with a substitution table for the centre alignments
 * (msa_nw_align_batch_affine_sub's model); the table must cover the gap code
 * of the centre rows (nsym >= 5 for DNA, 21 for protein). */
msa_status msa_merge_tree_affine_sub(msa_ctx *ctx, const msa_seqset *s, const int32_t *order, const int32_t *lo,
                                     const int32_t *hi, const int32_t *center, const int32_t *left,
                                     const int32_t *right, int32_t n_nodes, const int32_t *sub, int32_t nsym,
                                     int32_t gap_open, int32_t gap_ext, int32_t *pos, int32_t *width, int32_t *score,
                                     void *stream);
/* Writes the MSA rows (ASCII, '-' for gaps) in `order`: row r (W bytes at
 * rows + r*W, device) is sequence order[r]; W = width of the root. */
msa_status msa_msa_rows(msa_ctx *ctx, const msa_seqset *s, const int32_t *order, const int32_t *pos, int32_t W,
                        uint8_t *rows, void *stream);

/* ---- alignment quality (section "Evaluation") ----------------------------- */
/*
 * The three metrics of section "Evaluation" over S sampled rows of an MSA
 * (the paper uses a random sample of 10,000): rows is device u8 [R][W]
 * (msa_msa_rows), sample_rows (device int32 [S]) the rows to use and
 * sample_seqs (device int32 [S]) the index in s of each one's sequence.
 *   out3[0] percentage of gaps: per row, gap bytes / W, averaged, x 100;
 *   out3[1] p-score: over all pairs of sampled rows and all columns where
 *           neither has a gap, the share of columns whose bytes differ, x 100;
 *   out3[2] distance distortion: over all pairs of sampled rows, Hamming
 *           distance of the aligned rows (bytes differ; gap-gap is equal) /
 *           Levenshtein distance of their sequences, averaged (pairs of
 *           identical sequences have no ratio and are left out).
 * counts4 (host, optional): gap bytes, compared unit pairs, mismatched unit
 * pairs, pairs in the distortion mean.  Synchronous (host outputs).  Needs
 * workspace for S (S - 1) / 2 int32 distances plus one distance batch.
 */
msa_status msa_msa_metrics(msa_ctx *ctx, const msa_seqset *s, const uint8_t *rows, int32_t R, int32_t W,
                           const int32_t *sample_rows, const int32_t *sample_seqs, int32_t S, uint8_t gap,
                           double *out3, int64_t *counts4, void *stream);

/* ---- measurement ---------------------------------------------------------- */
/*
 * Integer-pipe throughput probe (no counterpart in the paper: it measures the
 * roofline denominator of the bit-vector kernels, whose word step is 3-input
 * logic, an add on the carry chain and a funnel shift).  Launches one kernel
 * on `stream` that runs, from registers only, op = 0 LOP3, 1 funnel shift by
 * one, 2 add with carry (8-word chains), 3 the Levenshtein word step
 * (9 operations per 32-row word, two independent columns per thread),
 * 4 integer multiply-add (the FMA pipe, for comparison), with 8 independent
 * chains per thread and every SM at its occupancy limit, `iters` loop
 * iterations.  *lane_ops (host) receives the number of lane operations the
 * launch executes; time the launch with CUDA events on `stream` and divide.
 * Uses the context workspace as the kernel's output sink.
 */
msa_status msa_probe_int_pipe(msa_ctx *ctx, int32_t op, int32_t iters, int64_t *lane_ops, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MSA_H */
