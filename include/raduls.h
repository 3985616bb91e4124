/*
 * raduls.h -- C ABI of the GB300 (sm_103a) stable MSD radix sorter of
 * fixed-size records ("RADULS", Kokot, Deorowicz, Debudaj-Grabysz,
 * arXiv:1612.02557).
 *
 * Problem (Sec. 4 of the paper: records of 8..32 bytes whose first 8 or 16
 * bytes are the key; Sec. 1: radix sort by digits of the key): sort n records
 * of rec_bytes bytes by a key made of the first key_bytes bytes.  The key is
 * read as key_bytes/8 little-endian u64 words, word 0 most significant,
 * compared as unsigned integers lexicographically.  The sort is STABLE:
 * records with equal keys keep their input order, so the output is unique and
 * is moved bit for bit.
 *
 * Method (Sec. 3.1-3.4): MSD radix sort.  Each pass over a bin builds a digit
 * histogram, turns it into bin offsets with an exclusive prefix (Sec. 1), and
 * distributes whole records stably; big bins recurse with more passes (Sec.
 * 3.3), small bins are finished by an on-chip sort (Sec. 3.4, 3.5).  The paper
 * uses radix 256 (Sec. 3.1); here a digit is a window of 8 to 10 key bits
 * picked per bin from its size, so that two passes bring 2^31 uniform records
 * down to bins that one SM sorts in shared memory.  Key bits that are constant
 * within a bin are skipped without moving data.
 *
 * Conventions for every call below:
 *  - Pointers named d_* and the record buffers `in`/`tmp` are DEVICE pointers
 *    on the current CUDA device.  The caller owns them.  `in` and `tmp` must be
 *    16-byte aligned, must not overlap, and each must hold n_recs*rec_bytes
 *    bytes.  The sorted records end up in `in`; `tmp` is scratch whose
 *    contents afterwards are undefined.
 *  - rec_bytes % 8 == 0, key_bytes % 8 == 0, 8 <= key_bytes <= rec_bytes <= 256,
 *    and n_recs*rec_bytes must not overflow 64 bits.  n_recs <= 1 is a no-op.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL is the legacy default
 *    stream).  Argument errors are returned at once and nothing is enqueued.
 *    The library keeps a per-device workspace (allocated on first use, grown
 *    when a larger problem arrives) and may synchronise `stream` between
 *    passes to plan the next one.
 *  - Errors detected on the device (a bounded wait that ran out) are recorded
 *    in a per-device status word and returned by raduls_stream_status().  No
 *    call traps or aborts the CUDA context.
 *  - Calls from several host threads are serialised internally per device.
 */
#ifndef RADULS_H
#define RADULS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RADULS_OK = 0,
    RADULS_ERR_INVALID_ARG = 1,  /* bad size, key/record shape or NULL pointer */
    RADULS_ERR_MISALIGNED = 2,   /* in/tmp not 16-byte aligned, or overlapping */
    RADULS_ERR_UNSUPPORTED = 3,  /* rec_bytes > 256 or a mode this build lacks */
    RADULS_ERR_CUDA = 4,         /* a CUDA runtime call failed */
    RADULS_ERR_OOM = 5,          /* the workspace could not be allocated */
    RADULS_ERR_TIMEOUT = 6,      /* a bounded device-side wait ran out */
    RADULS_ERR_INTERNAL = 7      /* an internal capacity check failed on the device */
} raduls_status;

/* Sort n_recs records of rec_bytes bytes in `in` by their first key_bytes
 * bytes (stable, ascending).  See the conventions above. */
int raduls_sort(void *in, void *tmp, uint64_t n_recs, uint32_t rec_bytes, uint32_t key_bytes,
                void *stream);

/* Kernel classes of raduls_stats.kernel_ms / kernel_launches. */
enum {
    RADULS_K_SETUP = 0,     /* work-list set-up and per-level resets */
    RADULS_K_HIST = 1,      /* digit histograms of big bins (first traversal, Sec. 1) */
    RADULS_K_PLAN = 2,      /* prefix sums and sub-bin classification (Fig. 1-3 on the GPU) */
    RADULS_K_SCATTER = 3,   /* stable distribution of big bins (second traversal, Sec. 1) */
    RADULS_K_COPY = 4,      /* copy-back of finished bins left in tmp */
    RADULS_K_BLOCK = 5,     /* on-chip sorts of small bins and runs of them (Sec. 3.4-3.5) */
    RADULS_K_LEARNED = 6,   /* learned-partition fit, count and distribution */
    RADULS_K_BATCHED = 7,   /* persistent batched segmented sort */
    RADULS_K_BUCKET = 8,    /* mid-size bins: split by one CTA and sorted on chip through L2 (Sec. 3.4) */
    RADULS_K_COUNT = 9
};

/* Statistics of one sort, filled when the call returns (the call synchronises
 * its stream when a stats pointer is given). */
typedef struct {
    uint32_t grid_passes;        /* device-wide distribution passes run (Sec. 3.2-3.3) */
    uint32_t levels;             /* MSD levels planned */
    uint64_t hist_bytes_read;    /* algorithmic bytes read by histogram passes */
    uint64_t scatter_bytes;      /* algorithmic bytes read + written by distribution passes */
    uint64_t block_bytes;        /* bytes read + written by on-chip bin sorts and copies */
    uint64_t block_items;        /* on-chip sort items (packed runs of small bins) */
    uint64_t skipped_digits;     /* bin-digits skipped because they were constant */
    uint32_t learned_used;       /* 1 when the learned first partition ran */
    uint32_t learned_fell_back;  /* 1 when the learned partition was rejected */
    float    learned_ratio;      /* max bucket / ideal bucket size of the learned model */
    uint32_t gpu_launches;       /* kernels this call launched */
    uint64_t bucket_items;       /* mid-size bins split and sorted by one CTA each */
    uint64_t bucket_bytes;       /* algorithmic bytes read + written by those bins' kernel */
    /* Device time per kernel class, measured with CUDA events recorded on the
     * call's stream around each launch, and launches per class, indexed by
     * the RADULS_K_* classes above. */
    float    kernel_ms[RADULS_K_COUNT];
    uint32_t kernel_launches[RADULS_K_COUNT];
} raduls_stats;

typedef struct {
    uint32_t mode;                  /* 0 AUTO (currently the plain passes: the learned first
                                       partition is not yet faster on skewed keys), 1 PLAIN,
                                       2 LEARNED */
    uint32_t learned_log2_buckets;  /* buckets of the learned pass, log2: 8..10, 0 = 8 */
    float    fallback_ratio;        /* learned partition is rejected above this max/ideal ratio
                                       (over buckets whose key word 0 varies); 0 = 4.0 */
    uint32_t train_steps;           /* Adam steps per stage of the model fit: 0 = 16, at most
                                       4096; 0x80000000 = the warm start alone */
    raduls_stats *stats;            /* host pointer or NULL */
} raduls_opts;

/* raduls_sort with options (mode, statistics).  opts may be NULL. */
int raduls_sort_ex(void *in, void *tmp, uint64_t n_recs, uint32_t rec_bytes, uint32_t key_bytes,
                   const raduls_opts *opts, void *stream);

/* End-to-end sort of records held in HOST memory (pinned or pageable):
 * h_in's n_recs records are copied to device buffers the library owns (kept
 * between calls and grown on demand to 2 x n_recs x rec_bytes), sorted there
 * exactly as raduls_sort_ex sorts them (same options, same result), and
 * copied back into h_out.  h_out may equal h_in (in place); otherwise the
 * two ranges must not overlap.  Both copies run on the library's own copy
 * stream, in chunks (the environment variable RADULS_COPY_STREAMS spreads
 * them over up to 8 streams; on GB300 one stream already moves about 200 GB/s
 * each way, the link's rate, and more streams were slower).  The last step of the
 * sort -- the streamed on-chip bin sort, or a mid-size level when no record
 * moves after it -- runs in 8 position windows and each window's records go
 * back while the next window is sorted (RADULS_HOST_WINDOWS=0 turns this
 * off).  The
 * work is ordered on `stream` like every other call: h_in must stay unchanged
 * and h_out untouched until the stream has passed the call (synchronise it,
 * or call raduls_stream_status).  Pinned memory is much faster; pageable
 * memory takes the driver's staging path.  No alignment rule for host
 * pointers.  Errors as raduls_sort_ex, plus RADULS_ERR_OOM when the device
 * buffers cannot be grown. */
int raduls_sort_host(const void *h_in, void *h_out, uint64_t n_recs, uint32_t rec_bytes, uint32_t key_bytes,
                     const raduls_opts *opts, void *stream);

/* The same result as raduls_sort(), reached through the keys alone: the
 * records' keys are copied out with their positions as (key, index) pairs,
 * the pairs are sorted (stable, so equal keys keep their index order), and
 * the records are then moved once, by a gather into `tmp` in the pairs'
 * order, and copied back into `in`.  Every distribution pass then moves
 * key_bytes + 8 bytes per record instead of rec_bytes, which pays for wide
 * records: the paper measures how its sort time grows with the record size
 * (Sec. 4).  The pairs and their scratch (2 x n_recs x (key_bytes + 8) bytes)
 * are held in the library's per-device workspace.  Conventions and errors as
 * raduls_sort(). */
int raduls_sort_indexed(void *in, void *tmp, uint64_t n_recs, uint32_t rec_bytes, uint32_t key_bytes,
                        void *stream);

/* Distinct keys of records already SORTED by their key, with the number of
 * records holding each (the counting use of the sort, Sec. 5: k-mer
 * counting): every run of equal keys of `in` becomes one entry.  Writes the
 * runs' keys (key_bytes each, in key order) to d_keys_out, their lengths to
 * d_counts_out and the number of runs to *d_n_unique (all DEVICE memory; the
 * caller sizes d_keys_out for n_recs keys and d_counts_out for n_recs
 * counts, the most there can be).  Pointers must be 8-byte aligned.  On
 * unsorted input every maximal run of equal adjacent keys is counted as it
 * stands.  Record shapes as raduls_sort(). */
int raduls_unique_counts(const void *in, uint64_t n_recs, uint32_t rec_bytes, uint32_t key_bytes,
                         void *d_keys_out, uint64_t *d_counts_out, uint64_t *d_n_unique, void *stream);

/* Sort n_segs independent arrays in one call.  Array s occupies records
 * [d_seg_offsets[s], d_seg_offsets[s+1]) of `in` (d_seg_offsets is a DEVICE
 * array of n_segs+1 non-decreasing u64 record offsets with d_seg_offsets[0]
 * == 0); records never move between arrays.  `tmp` must hold
 * d_seg_offsets[n_segs] records.  Offsets are checked on the device; a bad
 * offset table is reported through raduls_stream_status(). */
int raduls_sort_batched(void *in, void *tmp, const uint64_t *d_seg_offsets, uint32_t n_segs,
                        uint32_t rec_bytes, uint32_t key_bytes, void *stream);

/* Synchronise `stream`, then return and clear the device-side status of the
 * current device (RADULS_OK if no device-side error was recorded). */
int raduls_stream_status(void *stream);

/* Static text for a status code. */
const char *raduls_status_string(int status);

/* ---- the learned first partition (not in the paper) ----
 *
 * A monotone two-level piecewise-linear CDF of key word 0: level 1 is the
 * exact histogram R_j of the key's top byte j over all records (the first MSD
 * pass's digit histogram, Sec. 1), with exclusive prefix C_j; level 2, per top
 * byte j, maps the key's low 56 bits through two piecewise-linear stages
 * u = f2(f1(key)).  Stage 1 has knots 2^sh_j key units apart starting at the
 * low 56 bits of the segment's first sample (base_j); a key's interval is the
 * exact integer (low - base_j) >> sh_j and its position inside the interval
 * the remainder over 2^sh_j, rounded once to fp32 (keys below base_j map to 0,
 * keys past the last knot to 1).  Stage 2 has uniform knots on [0, 1].
 * Heights are learned and non-decreasing (cumulative softplus of the
 * parameters, normalised to end at 1).  A key goes to bucket
 * floor(B * p / n), p = C_j + min(floor(u * 2^64) * R_j / 2^64, R_j - 1), all
 * in integer arithmetic, so bucket order is key order.  The heights are fitted
 * on the GPU to the empirical CDF of a sorted key sample (mean squared error):
 * each stage is warm-started at the sample's CDF at its knots, then refined by
 * Adam steps, stage 1 first, then stage 2 on stage 1's output.
 * raduls_sort_ex(mode = LEARNED) builds one internally (B = 2^learned_log2_buckets,
 * at most 1,024) after the top byte's histogram pass: one distribution pass
 * then splits the records into the B buckets (stable, so equal keys keep their
 * order), recording every bucket's smallest and largest key word 0; a bucket
 * of one key value is finished there (one-word keys) or goes on from key word
 * 1; the others are sorted by the plain passes.  When the largest bucket whose
 * key varies holds more than fallback_ratio times n / B records, the learned
 * split is not used and the plain passes sort the whole input.  These calls
 * expose the model for testing and inspection. */
typedef struct raduls_model raduls_model;

/* Fit a model with 2^log2_buckets buckets (8..16) to the n_recs records at
 * `in` (device): each stage is warm-started from the sample's CDF at its knots
 * and refined by train_steps Adam steps.  train_steps = 0 leaves both stages
 * linear (the untrained model); train_steps = 0x80000000 keeps the warm start
 * without Adam steps.  *out receives a handle owning its own device buffers. */
int raduls_model_fit(raduls_model **out, const void *in, uint64_t n_recs, uint32_t rec_bytes,
                     uint32_t key_bytes, uint32_t log2_buckets, uint32_t train_steps, void *stream);

/* More Adam steps on one stage (0 or 1) with the model's own sample. */
int raduls_model_train(raduls_model *m, uint32_t stage, uint32_t steps, void *stream);

/* Training loss of one stage (stage 0: f1 alone; stage 1: the whole leaf
 * f2(f1(t))), as the mean squared CDF error on the sample (host double), and
 * its gradient w.r.t. that stage's parameters, written into the device float
 * array d_grad (n_params entries, see raduls_model_sizes; other entries are
 * left untouched). */
int raduls_model_loss_grad(raduls_model *m, uint32_t stage, double *h_loss, float *d_grad, void *stream);

/* Bucket of each key word (device u64 in, device u32 out). */
int raduls_model_buckets(const raduls_model *m, const uint64_t *d_keys, uint64_t n_keys, uint32_t *d_out,
                         void *stream);

/* Parameter-array length, sample size and log2 of the bucket count. */
int raduls_model_sizes(const raduls_model *m, uint32_t *n_params, uint32_t *n_sample, uint32_t *log2_buckets);

/* Copy the model to host arrays (any pointer may be NULL): root counts
 * [256] u64; segment tables [2][256] x {float x0, float inv_w, uint32
 * first_knot, uint32 knots, uint32 first_param, uint32 pad} (stage 1 then
 * stage 2); parameters and knot heights [n_params] float; sorted sample
 * [n_sample] u64. */
int raduls_model_copy_out(const raduls_model *m, uint64_t *h_root_counts, void *h_segments, float *h_theta,
                          float *h_heights, uint64_t *h_sample, void *stream);

void raduls_model_free(raduls_model *m);

/* ---- single-step entry points (one kernel each; used to test each step) ---- */

/* Histogram of digit `digit` (0 = least significant key byte; byte digit%8 of
 * key word key_bytes/8-1-digit/8) over all n_recs records: d_hist_out[256] u64
 * (device).  First traversal of a counting pass (Sec. 1). */
int raduls_histogram(const void *in, uint64_t n_recs, uint32_t rec_bytes, uint32_t key_bytes,
                     uint32_t digit, uint64_t *d_hist_out, void *stream);

/* One stable distribution pass on digit `digit` over the whole array, `in` ->
 * `out` (device, n_recs*rec_bytes each, not overlapping): the histogram, the
 * exclusive prefix and the stable scatter of Sec. 1 done by the GPU pass
 * kernels (chunk histograms chained by a single-pass look-back, then a
 * scatter whose tiles are ranked and regrouped in shared memory). */
int raduls_distribution_pass(const void *in, void *out, uint64_t n_recs, uint32_t rec_bytes,
                             uint32_t key_bytes, uint32_t digit, void *stream);

/* Same result as raduls_histogram(), without any allocation.  The paper has
 * no counterpart: this is for callers that cannot let a library allocate
 * device memory -- an application whose device memory is all reserved up
 * front by its own allocator, a latency-critical loop that cannot afford the
 * device-wide synchronisation of cudaMalloc/cudaFree, or code running while a
 * stream is being captured, where allocation calls are not allowed.
 *
 * The call's scratch (work counters, the work item, the histogram row and one
 * u32 per 16384-record tile) lives in a fixed 1 MiB array inside the library,
 * which every GPU that loads the library holds until the process exits.
 * Inputs larger than that tile map allows -- more than 260,928 tiles of
 * 16,384 records, i.e. more than 4,275,044,352 records -- are rejected with
 * RADULS_ERR_UNSUPPORTED before anything is launched.  The call returns
 * argument and launch errors only: its kernel has no bounded wait and records
 * no device-side status (raduls_stream_status() does not report on it).  The first call on a device looks the array's address up
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls on a device share the one array, and
 * each call rewrites everything it reads from it, but calls that overlap on
 * the GPU (for instance on two streams) race on it: serialise them. */
int raduls_histogram_static(const void *in, uint64_t n_recs, uint32_t rec_bytes, uint32_t key_bytes,
                            uint32_t digit, uint64_t *d_hist_out, void *stream);

/* Settings picked by raduls_autotune. */
typedef struct {
    int32_t  scatter_variant;  /* distribution kernel shape (threads x records per thread, widest digit) */
    uint32_t scatter_tile;     /* records per distribution tile of that shape */
    uint32_t block_cap;        /* largest bin (or run of small bins / arrays) sorted by one CTA on chip */
    uint32_t bucket_max;       /* largest mid-size bin sorted by one CTA through L2 (0: class off) */
    float    best_ms;          /* sort time of the chosen setting on the tuning input */
    uint32_t candidates;       /* settings timed */
    uint32_t digit_bits;       /* widest digit of a distribution pass, in bits (8..10) */
    uint32_t leaf;             /* sub-bin size (records) the digit widths aim at */
    uint32_t bin_sort;         /* 1: small bins go to the streamed on-chip sort first */
} raduls_tuning;

/* Autotuner of the launch shapes, digit widths and size-class thresholds
 * (the paper has no counterpart; its scheduling constants, Sec. 3.2-3.5, are
 * CPU-specific).  Fills `in` with seeded uniform records (SplitMix64 words),
 * sorts them once per candidate setting -- every distribution tile shape
 * that fits the record width (shapes 0-15; 16-21 differ from 11 and 9 only
 * in how warps rank or store, kept for comparison), the widest digit at 8, 9
 * and 10 bits, two sub-bin size targets, the on-chip class at its full and
 * half capacity, the streamed on-chip bin sort on and off, the mid-size
 * class off, at half and at full size -- with `tmp` as scratch, times each
 * with CUDA events (best of two), and keeps the fastest for later calls on
 * this device with this record width (candidates go from the default shape
 * outward, and the winner must beat the default by more than 1% in a final
 * alternating re-timing, so timing noise never trades the default for a
 * setting that only uniform keys tolerate): plain sorts when d_seg_offsets
 * is NULL, batched sorts (with those offsets) otherwise.  `in` and `tmp`
 * hold n_recs records; their contents are undefined afterwards.
 * Synchronises `stream`; not for use inside a stream capture.  `out` may be
 * NULL.  Environment overrides still take precedence: RADULS_SCATTER_VARIANT
 * (one distribution shape for every level), RADULS_SCATTER8 / 9 / 10 (the
 * shape of levels whose widest digit has that many bits), RADULS_WMAX
 * (widest digit, 8..10), RADULS_LEAF (sub-bin size target),
 * RADULS_BLOCK_CAP, RADULS_BUCKET_MAX (mid-size class, 0 = off),
 * RADULS_BIN_SORT (0/1: the streamed on-chip sort), RADULS_BIN_VARIANT. */
int raduls_autotune(void *in, void *tmp, uint64_t n_recs, uint32_t rec_bytes, uint32_t key_bytes,
                    const uint64_t *d_seg_offsets, uint32_t n_segs, raduls_tuning *out, void *stream);

/* Forget every tuned setting (back to the built-in shapes). */
int raduls_autotune_reset(void);

/* Test hook: make the next distribution pass withhold the published counts
 * of histogram chunk `tile` (65,536 records per chunk, numbered over the
 * pass's bins) so that its successors' bounded look-back waits run out
 * (kind 1); make the next batched call withhold the ready flag of pushed
 * queue item number `tile` so that the persistent kernel's bounded wait for it
 * runs out (kind 2); or clear the hooks (kind 0).  The call then reports
 * RADULS_ERR_TIMEOUT through raduls_stream_status() and skips the rest of its
 * work; the context stays usable. */
int raduls_debug_inject(uint32_t kind, uint64_t tile);

/* Device-side wait limit in nanoseconds for look-back spins (default 2e9). */
int raduls_set_wait_limit_ns(uint64_t ns);

#ifdef __cplusplus
}
#endif

#endif /* RADULS_H */
