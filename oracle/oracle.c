/*
 * oracle.c -- CPU oracle for the stable record sort.  TEST INFRASTRUCTURE ONLY:
 * only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library.  The GPU sorter shares no code with it.
 *
 * What it computes (the plain definition the GPU path must reproduce bit for
 * bit): n records of r bytes; the key is the first k bytes read as W = k/8
 * little-endian u64 words, word 0 most significant, compared as unsigned
 * integers lexicographically; the output is the unique stable permutation
 * (equal keys keep their input order), moving whole records byte for byte.
 *
 * How: least-significant-digit radix sort with radix R = 256 whose inner sort
 * is a counting sort, as the paper's introduction describes it (Sec. 1):
 * one traversal builds a histogram of the digit values, an exclusive prefix
 * over the histogram gives, for each digit value, the number of keys with a
 * smaller digit, and a second traversal, in input order, places every record
 * at its digit's next free slot.  Because each counting pass is stable, the
 * LSD order over all 8W digits yields the stable sort by the full key (Sec. 1).
 *
 * Digit numbering: digit p (p = 0 is least significant) is byte (p mod 8) of
 * key word W-1-floor(p/8); byte b of a little-endian word is the record byte at
 * offset 8*word + b, so a digit is read straight from memory with no
 * endianness assumption.
 *
 * The threaded form splits the records into T contiguous chunks; each chunk
 * is counted on its own and the output slots are handed out in (digit, chunk)
 * order, so every chunk's records of one digit land after all earlier chunks'
 * ones: the pass stays stable.  T = 1 is the textbook single-threaded pass.
 */
#define _POSIX_C_SOURCE 200809L
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define RADIX 256

/* digit p of the record at rec (see header) */
static inline unsigned digit_at(const uint8_t *rec, uint32_t key_words, uint32_t p)
{
    uint32_t word = key_words - 1u - p / 8u;
    return rec[8u * word + (p % 8u)];
}

/* ---------------------------------------------------------------- one pass */

/* Stable counting pass on digit p of records [lo, hi) of src into dst[lo, hi)
 * (single-threaded; Sec. 1: histogram, exclusive prefix, distribution). */
static void counting_pass_range(const uint8_t *src, uint8_t *dst, uint64_t lo, uint64_t hi,
                                uint32_t r, uint32_t key_words, uint32_t p)
{
    uint64_t count[RADIX];
    uint64_t next[RADIX];
    memset(count, 0, sizeof count);
    for (uint64_t i = lo; i < hi; ++i)
        count[digit_at(src + i * r, key_words, p)]++;
    uint64_t run = lo;
    for (unsigned d = 0; d < RADIX; ++d) {
        next[d] = run;            /* keys with a smaller digit come first */
        run += count[d];
    }
    for (uint64_t i = lo; i < hi; ++i) {
        unsigned d = digit_at(src + i * r, key_words, p);
        memcpy(dst + next[d] * r, src + i * r, r);
        next[d]++;
    }
}

static int args_ok(uint32_t r, uint32_t k)
{
    return r % 8u == 0 && k % 8u == 0 && k >= 8u && k <= r;
}

/* One stable counting pass on digit p over the whole array. */
int oracle_counting_pass(const uint8_t *in, uint8_t *out, uint64_t n, uint32_t r,
                         uint32_t k, uint32_t p)
{
    if (!args_ok(r, k) || p >= 8u * (k / 8u))
        return 1;
    counting_pass_range(in, out, 0, n, r, k / 8u, p);
    return 0;
}

/* One stable counting pass on digit p inside each segment
 * [offsets[s], offsets[s+1]) -- an MSD pass over several bins at once:
 * records never leave their bin (Sec. 1, MSD variant). */
int oracle_segmented_counting_pass(const uint8_t *in, uint8_t *out, uint32_t r, uint32_t k,
                                   uint32_t p, const uint64_t *offsets, uint64_t n_segs)
{
    if (!args_ok(r, k) || p >= 8u * (k / 8u))
        return 1;
    for (uint64_t s = 0; s < n_segs; ++s) {
        if (offsets[s + 1] < offsets[s])
            return 1;
        counting_pass_range(in, out, offsets[s], offsets[s + 1], r, k / 8u, p);
    }
    return 0;
}

/* Histogram of digit p over the whole array (first traversal of a pass). */
int oracle_histogram(const uint8_t *in, uint64_t n, uint32_t r, uint32_t k, uint32_t p,
                     uint64_t *hist /* [256] */)
{
    if (!args_ok(r, k) || p >= 8u * (k / 8u))
        return 1;
    memset(hist, 0, RADIX * sizeof(uint64_t));
    for (uint64_t i = 0; i < n; ++i)
        hist[digit_at(in + i * r, k / 8u, p)]++;
    return 0;
}

/* ------------------------------------------------------------ full LSD sort */

typedef struct {
    const uint8_t *in;
    uint8_t *buf[2];          /* ping-pong buffers; buf[1] is the output */
    uint64_t n;
    uint32_t r, key_words, threads;
    uint64_t (*count)[RADIX]; /* [threads][RADIX] */
    pthread_barrier_t bar;
} lsd_job;

typedef struct {
    lsd_job *job;
    uint32_t t;
} lsd_worker;

static void *lsd_worker_main(void *arg)
{
    lsd_worker *w = (lsd_worker *)arg;
    lsd_job *j = w->job;
    const uint32_t T = j->threads, t = w->t, r = j->r, kw = j->key_words;
    const uint64_t lo = j->n * t / T, hi = j->n * (t + 1) / T;
    const uint32_t passes = 8u * kw;
    for (uint32_t p = 0; p < passes; ++p) {
        /* passes alternate so that the last one (p = passes-1, odd) writes buf[1] */
        const uint8_t *src = (p == 0) ? j->in : j->buf[p % 2u == 1u ? 0 : 1];
        uint8_t *dst = j->buf[p % 2u];
        uint64_t *cnt = j->count[t];
        memset(cnt, 0, RADIX * sizeof(uint64_t));
        for (uint64_t i = lo; i < hi; ++i)
            cnt[digit_at(src + i * r, kw, p)]++;
        pthread_barrier_wait(&j->bar);
        if (t == 0) {
            /* exclusive prefix in (digit, chunk) order: turn counts into start slots */
            uint64_t run = 0;
            for (unsigned d = 0; d < RADIX; ++d)
                for (uint32_t c = 0; c < T; ++c) {
                    uint64_t v = j->count[c][d];
                    j->count[c][d] = run;
                    run += v;
                }
        }
        pthread_barrier_wait(&j->bar);
        for (uint64_t i = lo; i < hi; ++i) {
            unsigned d = digit_at(src + i * r, kw, p);
            memcpy(dst + cnt[d] * r, src + i * r, r);
            cnt[d]++;
        }
        pthread_barrier_wait(&j->bar);
    }
    return NULL;
}

/* Stable sort of n records (see header).  out may not alias in.  threads >= 1.
 * Returns 0 on success, 1 on bad arguments, 2 when memory runs out. */
int oracle_sort(const uint8_t *in, uint8_t *out, uint64_t n, uint32_t r, uint32_t k,
                uint32_t threads)
{
    if (!args_ok(r, k) || threads == 0)
        return 1;
    if (n == 0)
        return 0;
    if (threads > 1024)
        threads = 1024;
    if ((uint64_t)threads > n)
        threads = (uint32_t)n;
    uint8_t *tmp = (uint8_t *)malloc((size_t)(n * r));
    if (!tmp)
        return 2;
    lsd_job job;
    job.in = in;
    job.buf[0] = tmp;
    job.buf[1] = out;
    job.n = n;
    job.r = r;
    job.key_words = k / 8u;
    job.threads = threads;
    job.count = (uint64_t(*)[RADIX])calloc(threads, sizeof(uint64_t[RADIX]));
    lsd_worker *ws = (lsd_worker *)calloc(threads, sizeof(lsd_worker));
    pthread_t *tids = (pthread_t *)calloc(threads, sizeof(pthread_t));
    if (!job.count || !ws || !tids) {
        free(tmp);
        free(job.count);
        free(ws);
        free(tids);
        return 2;
    }
    pthread_barrier_init(&job.bar, NULL, threads);
    for (uint32_t t = 0; t < threads; ++t) {
        ws[t].job = &job;
        ws[t].t = t;
        if (t > 0)
            pthread_create(&tids[t], NULL, lsd_worker_main, &ws[t]);
    }
    lsd_worker_main(&ws[0]);
    for (uint32_t t = 1; t < threads; ++t)
        pthread_join(tids[t], NULL);
    pthread_barrier_destroy(&job.bar);
    free(tids);
    free(ws);
    free(job.count);
    free(tmp);
    return 0;
}

/* Independent arrays: each segment [offsets[s], offsets[s+1]) is sorted on its
 * own (records never cross segments). */
int oracle_sort_segments(const uint8_t *in, uint8_t *out, const uint64_t *offsets,
                         uint64_t n_segs, uint32_t r, uint32_t k, uint32_t threads)
{
    if (!args_ok(r, k))
        return 1;
    for (uint64_t s = 0; s < n_segs; ++s) {
        if (offsets[s + 1] < offsets[s])
            return 1;
        uint64_t m = offsets[s + 1] - offsets[s];
        uint32_t t = m >= (1u << 20) ? threads : 1u;
        int rc = oracle_sort(in + offsets[s] * r, out + offsets[s] * r, m, r, k, t);
        if (rc)
            return rc;
    }
    return 0;
}
