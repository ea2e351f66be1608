/*
 * synth.c — seeded synthetic QUICCI-like descriptor generator (host C).
 *
 * This module draws inputs only: it holds none of the retrieval method's
 * arithmetic (no distance, no tree, no voting).  Both the CPU oracle and the
 * CUDA path consume what it produces, so it lives on its own.
 *
 * Descriptor model (stands in for QUICCI images of SHREC'16 meshes, §2.2 and
 * §6 of the paper: 64x64 bits, 512 bytes, bit (r, c) = layer r from the
 * bottom, radius column c from the innermost circle):
 *   - an image is the rasterisation of 2..6 smooth curves, each a quadratic
 *     col(r) = c0 + b (r - rm) + a (r - rm)^2 over a random span of rows;
 *     in row r the bits of every column boundary the curve crosses between
 *     rows r and r+1 are set (an intersection-count-change pattern);
 *   - an object owns a pool of curve sets; each database descriptor of the
 *     object is a jittered copy of one pool entry with a small bit dropout;
 *   - a query is a database descriptor with a fraction of its set bits
 *     cleared (partiality) and a fraction of all bits flipped (noise).
 *
 * Every random number comes from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014)
 * keyed by (seed, tag, index...), so any single descriptor can be regenerated
 * on its own and the output does not depend on the thread count.  Only IEEE
 * +,-,*,floor are used on doubles (no libm transcendental calls), and the file
 * is compiled with -ffp-contract=off, so x86-64 and aarch64 hosts produce the
 * same bits.
 */
#include <stdint.h>
#include <string.h>
#include <math.h>

#define SY_WORDS 64
#define SY_MAX_CURVES 6

enum { TAG_POOL = 1, TAG_DESC = 2, TAG_QSRC = 3, TAG_QNOISE = 4,
       TAG_PQ = 5, TAG_PNOISE = 6 };

static uint64_t sm_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* SplitMix64 step: advance the state by the golden gamma, mix it. */
static uint64_t sm_next(uint64_t *s)
{
    *s += 0x9e3779b97f4a7c15ULL;
    return sm_mix(*s);
}

static uint64_t stream3(uint64_t seed, uint64_t tag, uint64_t i, uint64_t j)
{
    uint64_t s = sm_mix(seed + 0x9e3779b97f4a7c15ULL * (tag + 1));
    s = sm_mix(s ^ (i + 0x632be59bd9b4e019ULL));
    s = sm_mix(s ^ (j + 0x85157af5ULL));
    return s;
}

static double unif(uint64_t *s) /* [0, 1) with 53 random bits */
{
    return (double)(sm_next(s) >> 11) * (1.0 / 9007199254740992.0);
}

static double urange(uint64_t *s, double lo, double hi)
{
    return lo + (hi - lo) * unif(s);
}

/* Irwin-Hall(4) approximation of a unit normal: arithmetic only. */
static double gauss(uint64_t *s)
{
    double u = unif(s) + unif(s) + unif(s) + unif(s);
    return (u - 2.0) * 1.7320508075688772;
}

typedef struct { double c0, b, a; int r0, r1; } curve_t;
typedef struct { int m; curve_t c[SY_MAX_CURVES]; } curveset_t;

static void draw_curveset(uint64_t seed, int64_t object, int32_t j, curveset_t *cs)
{
    uint64_t s = stream3(seed, TAG_POOL, (uint64_t)object, (uint64_t)j);
    cs->m = 2 + (int)(sm_next(&s) % (SY_MAX_CURVES - 1));   /* 2..6 */
    for (int k = 0; k < cs->m; ++k) {
        curve_t *c = &cs->c[k];
        int r0 = (int)(sm_next(&s) % 33);          /* 0..32 */
        int len = 32 + (int)(sm_next(&s) % 33);    /* 32..64 */
        c->r0 = r0;
        c->r1 = r0 + len > 64 ? 64 : r0 + len;
        c->c0 = urange(&s, 4.0, 60.0);
        c->b = urange(&s, -1.2, 1.2);
        c->a = urange(&s, -0.03, 0.03);
    }
}

static void raster(const curveset_t *cs, uint64_t *img)
{
    memset(img, 0, SY_WORDS * sizeof(uint64_t));
    for (int k = 0; k < cs->m; ++k) {
        const curve_t *c = &cs->c[k];
        double rm = 0.5 * (double)(c->r0 + c->r1);
        for (int r = c->r0; r < c->r1; ++r) {
            double d0 = (double)r - rm, d1 = (double)(r + 1) - rm;
            double x0 = c->c0 + c->b * d0 + c->a * d0 * d0;
            double x1 = c->c0 + c->b * d1 + c->a * d1 * d1;
            double lo = x0 < x1 ? x0 : x1, hi = x0 < x1 ? x1 : x0;
            if (hi < 0.0 || lo >= 64.0) continue;
            int ilo = lo < 0.0 ? 0 : (int)floor(lo);
            int ihi = hi >= 64.0 ? 63 : (int)floor(hi);
            for (int col = ilo; col <= ihi; ++col)
                img[r] |= 1ULL << col;
        }
    }
}

/* One database descriptor: object = i / per_object, a jittered pool entry. */
void synth_one(uint64_t seed, int64_t i, int64_t per_object, int32_t pool, uint64_t *out)
{
    int64_t object = i / per_object;
    uint64_t s = stream3(seed, TAG_DESC, (uint64_t)i, 0);
    int32_t j = (int32_t)(sm_next(&s) % (uint64_t)pool);
    curveset_t cs;
    draw_curveset(seed, object, j, &cs);
    for (int k = 0; k < cs.m; ++k) {
        cs.c[k].c0 += 0.6 * gauss(&s);
        cs.c[k].b += 0.05 * gauss(&s);
        cs.c[k].a += 0.002 * gauss(&s);
    }
    raster(&cs, out);
    for (int w = 0; w < SY_WORDS; ++w) {       /* 3% dropout of set bits */
        uint64_t x = out[w];
        while (x) {
            int b = __builtin_ctzll(x);
            x &= x - 1;
            if (unif(&s) < 0.03) out[w] &= ~(1ULL << b);
        }
    }
}

/* n descriptors, object_of[i] = i / per_object (nullable). */
void synth_db(uint64_t seed, int64_t n, int64_t per_object, int32_t pool,
              uint64_t *out, uint32_t *object_of, int32_t nthreads)
{
#pragma omp parallel for schedule(static, 4096) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t i = 0; i < n; ++i) {
        synth_one(seed, i, per_object, pool, out + i * SY_WORDS);
        if (object_of) object_of[i] = (uint32_t)(i / per_object);
    }
}

/* Number of flips among 4096 independent Bernoulli(p) bits, by inversion of
 * the Binomial(4096, p) distribution (pmf by the ratio recurrence). */
static int binomial_4096(double p, uint64_t *s)
{
    double u = unif(s), q = 1.0 - p, pmf = 1.0;
    for (int i = 0; i < 4096; ++i) pmf *= q;          /* P(K = 0) */
    double cdf = pmf;
    int k = 0;
    while (u >= cdf && k < 4096) {
        pmf *= (double)(4096 - k) / (double)(k + 1) * (p / q);
        cdf += pmf;
        ++k;
    }
    return k;
}

/* Clear each set bit with probability p_clear, then flip every bit with
 * probability p_flip (stream s): a Binomial(4096, p_flip) count of distinct
 * positions, drawn uniformly, which is the same distribution. */
static void add_noise(uint64_t *d, double p_clear, double p_flip, uint64_t *s)
{
    for (int w = 0; w < SY_WORDS; ++w) {
        uint64_t x = d[w];
        while (x) {
            int b = __builtin_ctzll(x);
            x &= x - 1;
            if (unif(s) < p_clear) d[w] &= ~(1ULL << b);
        }
    }
    if (p_flip <= 0.0) return;
    int k = binomial_4096(p_flip, s);
    uint64_t flip[SY_WORDS] = {0};
    for (int done = 0; done < k;) {
        int pos = (int)(sm_next(s) >> 52);             /* 12 random bits */
        uint64_t m = 1ULL << (pos & 63);
        if (flip[pos >> 6] & m) continue;               /* distinct positions */
        flip[pos >> 6] |= m;
        ++done;
    }
    for (int w = 0; w < SY_WORDS; ++w) d[w] ^= flip[w];
}

/* nq queries: a uniformly drawn database descriptor, partiality + noise.
 * src[q] = the database index each query was made from (nullable). */
void synth_queries(uint64_t seed, const uint64_t *db, int64_t n, int64_t nq,
                   double p_clear, double p_flip, uint64_t *out, int64_t *src,
                   int32_t nthreads)
{
#pragma omp parallel for schedule(static, 64) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t q = 0; q < nq; ++q) {
        uint64_t s = stream3(seed, TAG_QSRC, (uint64_t)q, 0);
        int64_t i = (int64_t)(sm_next(&s) % (uint64_t)n);
        memcpy(out + q * SY_WORDS, db + i * SY_WORDS, 512);
        uint64_t t = stream3(seed, TAG_QNOISE, (uint64_t)q, 0);
        add_noise(out + q * SY_WORDS, p_clear, p_flip, &t);
        if (src) src[q] = i;
    }
}

/* Partial-object queries, phase 1: for query q pick an object, a fraction
 * f ~ U[f_lo, f_hi] of its descriptors, clamp the count to [n_min, n_max]
 * (and to per_object), and a start so the subset is contiguous.
 * Writes object[q], start[q] (object-local) and count[q]. */
void synth_partial_plan(uint64_t seed, int64_t n_objects, int64_t per_object, int64_t nq,
                        double f_lo, double f_hi, int64_t n_min, int64_t n_max,
                        int64_t *object, int64_t *start, int64_t *count)
{
    for (int64_t q = 0; q < nq; ++q) {
        uint64_t s = stream3(seed, TAG_PQ, (uint64_t)q, 0);
        int64_t o = (int64_t)(sm_next(&s) % (uint64_t)n_objects);
        double f = urange(&s, f_lo, f_hi);
        int64_t c = (int64_t)floor(f * (double)per_object + 0.5);
        if (c < n_min) c = n_min;
        if (c > n_max) c = n_max;
        if (c > per_object) c = per_object;
        if (c < 0) c = 0;
        int64_t st = (int64_t)(sm_next(&s) % (uint64_t)(per_object - c + 1));
        object[q] = o;
        start[q] = st;
        count[q] = c;
    }
}

/* Phase 2: fill the CSR descriptor array (offsets[nq+1] from the counts of
 * phase 1) with noisy copies of each query's contiguous subset. */
void synth_partial_fill(uint64_t seed, const uint64_t *db, int64_t per_object, int64_t nq,
                        const int64_t *object, const int64_t *start, const int64_t *offsets,
                        double p_clear, double p_flip, uint64_t *qdesc, int32_t nthreads)
{
    for (int64_t q = 0; q < nq; ++q) {
        int64_t base = object[q] * per_object + start[q];
        int64_t c = offsets[q + 1] - offsets[q];
#pragma omp parallel for schedule(static, 256) num_threads(nthreads > 0 ? nthreads : 1)
        for (int64_t i = 0; i < c; ++i) {
            uint64_t *d = qdesc + (offsets[q] + i) * SY_WORDS;
            memcpy(d, db + (base + i) * SY_WORDS, 512);
            uint64_t s = stream3(seed, TAG_PNOISE, (uint64_t)q, (uint64_t)i);
            add_noise(d, p_clear, p_flip, &s);
        }
    }
}
