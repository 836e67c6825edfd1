/*
 * Fast seeded generator of independent DNA pairs (input data only; it holds
 * none of the alignment arithmetic).  Pair p draws from its own SplitMix64
 * stream (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014) seeded with seed + p * 0x9E3779B97F4A7C15, so
 * pairs can be generated in any order or in parallel.
 *
 * Pair p: root length L ~ U{len_lo..len_hi}, root bases uniform over ACGT;
 * divergence delta ~ U(div_lo, div_hi).  The partner walks the root site by
 * site: with probability indel_share*delta an indel event starts at the site
 * (insertion or deletion with probability 1/2, length Geometric(1/2) on
 * {1, 2, ...}; an insertion puts random bases before the site, a deletion
 * skips the site and the following ones); otherwise, with probability delta,
 * the base is replaced by one of the other three uniformly; otherwise it is
 * copied.
 */
#include <stdint.h>
#include <pthread.h>
#include <string.h>

static inline uint64_t sm64(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static inline double unif(uint64_t *s) { return (double)(sm64(s) >> 11) * (1.0 / 9007199254740992.0); }
static inline int geom_half(uint64_t *s)
{
    int k = 1;
    while (unif(s) >= 0.5) ++k;
    return k;
}

static const uint8_t ACGT[4] = {'A', 'C', 'G', 'T'};

typedef struct {
    uint64_t seed;
    int64_t p0, p1;
    int32_t len_lo, len_hi;
    double div_lo, div_hi, indel_share;
    uint8_t *buf;      /* per-pair slab of slab_cap bytes */
    int64_t slab_cap;
    int32_t *lens;     /* [2P] */
    int32_t err;
} job_t;

static void *work(void *arg)
{
    job_t *J = (job_t *)arg;
    for (int64_t p = J->p0; p < J->p1; ++p) {
        uint64_t st = J->seed + (uint64_t)p * 0x9E3779B97F4A7C15ull;
        int32_t L = J->len_lo + (int32_t)(sm64(&st) % (uint64_t)(J->len_hi - J->len_lo + 1));
        double delta = J->div_lo + (J->div_hi - J->div_lo) * unif(&st);
        double pind = J->indel_share * delta;
        uint8_t *root = J->buf + p * J->slab_cap;
        uint8_t *part = root + L;
        int64_t room = J->slab_cap - L;
        for (int32_t i = 0; i < L; ++i) root[i] = ACGT[sm64(&st) & 3];
        int64_t k = 0;
        int same = 1;
        for (int32_t i = 0; i < L; ++i) {
            if (unif(&st) < pind) {
                int g = geom_half(&st);
                same = 0;
                if (unif(&st) < 0.5) {               /* insertion, then the site itself */
                    for (int t = 0; t < g && k < room; ++t) part[k++] = ACGT[sm64(&st) & 3];
                } else {                             /* deletion of g sites */
                    i += g - 1;
                    continue;
                }
            }
            if (k >= room) { J->err = 1; break; }
            uint8_t b = root[i];
            if (unif(&st) < delta) {
                int c = (int)(strchr("ACGT", b) - "ACGT");
                b = ACGT[(c + 1 + (int)(sm64(&st) % 3)) & 3];
                same = 0;
            }
            part[k++] = b;
        }
        if (same && k > 0) {                          /* never equal to the root */
            int c = (int)(strchr("ACGT", part[0]) - "ACGT");
            part[0] = ACGT[(c + 1) & 3];
        }
        J->lens[2 * p] = L;
        J->lens[2 * p + 1] = (int32_t)k;
    }
    return NULL;
}

/* buf: n_pairs * slab_cap bytes (slab_cap >= 3 * len_hi is ample); lens: [2 n_pairs].
 * Returns 0, or -1 if some partner overflowed its slab. */
int32_t synth_divergent_pairs(uint64_t seed, int64_t n_pairs, int32_t len_lo, int32_t len_hi, double div_lo,
                              double div_hi, double indel_share, uint8_t *buf, int64_t slab_cap, int32_t *lens,
                              int32_t nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    job_t jobs[256];
    pthread_t th[256];
    for (int t = 0; t < nthreads; ++t) {
        job_t j = {seed, n_pairs * t / nthreads, n_pairs * (t + 1) / nthreads, len_lo, len_hi, div_lo, div_hi,
                   indel_share, buf, slab_cap, lens, 0};
        jobs[t] = j;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, work, &jobs[t]);
    work(&jobs[0]);
    int32_t err = jobs[0].err;
    for (int t = 1; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        err |= jobs[t].err;
    }
    return err ? -1 : 0;
}

/* Copies root p and partner p from their slabs into one arena at offs[2p],
 * offs[2p+1] (offs: [2 n_pairs + 1], prefix sums of lens). */
void synth_compact_pairs(const uint8_t *buf, int64_t slab_cap, const int32_t *lens, int64_t n_pairs,
                         const int64_t *offs, uint8_t *out)
{
    for (int64_t p = 0; p < n_pairs; ++p) {
        memcpy(out + offs[2 * p], buf + p * slab_cap, (size_t)lens[2 * p]);
        memcpy(out + offs[2 * p + 1], buf + p * slab_cap + lens[2 * p], (size_t)lens[2 * p + 1]);
    }
}
