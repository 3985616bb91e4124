// kernels.h -- host-side launch wrappers of the sorter's kernels (internal).
#pragma once

#include "common.cuh"

namespace raduls {

// Launch shapes of one record width, chosen by the driver.
struct Shape {
    u32 rw;          // record words (rec_bytes / 8)
    u32 key_words;   // key words (key_bytes / 8)
    u32 tile_h;      // records per histogram tile
    u32 tile_s;      // records per distribution tile
    u32 tile_c;      // records per copy tile
    u32 cap_b;       // largest bin sorted on chip
    u32 bucket_max;  // largest bin split and sorted by one CTA through L2 (0: none)
    int scat_var;    // distribution kernel variant
    int block_var;   // on-chip sort kernel variant
    int bucket_var;  // mid-size bin kernel variant (-1: none for this record width)
    u32 leaf;        // sub-bin size the distribution passes' digit widths aim at
    u32 wmax;        // widest digit of a distribution pass (bits, 8..WIDE_MAX)
    int bins_var;    // streamed on-chip finisher variant (-1: the general on-chip kernel alone)
    bool scat_by_width;  // each level's distribution shape follows its widest digit
    int scat_var8, scat_var9, scat_var10;  // the shapes of 8-, 9- and 10-bit levels when it does
};

// The distribution shape of a level whose widest digit has w bits.
int level_scatter_variant(const Shape &s, u32 w);

Shape choose_shape(u32 rw, u32 key_words, bool batched = false);

// Persistent-grid sizes (CTAs) of each kernel for a shape on the current device.
u32 hist_grid(const Shape &s);
u32 block_grid(const Shape &s);
u32 copy_grid();

// Histogram of a key byte over every bin of the grid list (the histogram-only
// entry points): per-bin rows of 256 counts and the OR / AND of the key word.
cudaError_t launch_hist(const Shape &s, const u64 *in, const u64 *tmp, const WorkItem *items,
                        const u32 *tile_item, u64 *hist, u64 *orand, Counters *ctrs, cudaStream_t st);
// fb: the list of items the streamed bin sort left (count block_fb) instead
// of the on-chip list itself (count block).
cudaError_t launch_block_sort(const Shape &s, u64 *in, const u64 *tmp, const WorkItem *blocks,
                              Counters *ctrs, const u64 *seg_off, cudaStream_t st, bool fb = false);

// The streamed on-chip finisher (binsort.cu): every on-chip item it can take
// (a single bin or a run of one parent's sub-bins, up to its capacity) sorted
// in shared memory while the next one loads; the rest go to `fb` (capacity
// fb_cap) for launch_block_sort(..., fb = true).  -1 / 0: no variant for rw.
int binsort_variant_for(u32 rw);
u32 binsort_cap_of(int var);
u32 binsort_rw_of(int var);
// With `order` non-null, only window `window` of the on-chip list is taken:
// items order[wstart[window]] .. order[wstart[window + 1] - 1].
cudaError_t launch_bin_sort(int var, u64 *in, const u64 *tmp, const WorkItem *blocks, WorkItem *fb, Counters *ctrs,
                            u32 key_words, u64 fb_cap, u64 wait_ns, cudaStream_t st, const u32 *order = nullptr,
                            const u32 *wstart = nullptr, u32 window = 0);

// The distribution pass over chunks (wide.cu): a histogram of every chunk's
// digit window whose counts are chained along each bin's chunks by a
// decoupled look-back (status words: per chunk and digit value, the records
// of that value in the bin's chunks up to and including it), then a scatter in
// which every CTA distributes whole chunks on its own.
cudaError_t launch_whist(const Shape &s, const u64 *in, const u64 *tmp, const WorkItem *items, const u32 *tile_item,
                         const u64 *cell_off, u64 *status, u64 *orand, Counters *ctrs, const Model *model,
                         const u32 *epoch, u64 wait_ns, u32 inject_chunk, cudaStream_t st);
cudaError_t launch_wscatter(const Shape &s, u64 *in, u64 *tmp, const WorkItem *items, const u32 *tile_item,
                            const u64 *cell_off, const u64 *status, Counters *ctrs, const Model *model, u64 wait_ns,
                            cudaStream_t st);
u32 wscatter_tile_of(int var);
u32 wscatter_kmax_of(int var);  // most digit values a variant handles
// out[i] = the count held by status word row[i] (i < k).
cudaError_t launch_status_counts(const u64 *row, u64 *out, u32 k, cudaStream_t st);
u32 wscatter_grid(const Shape &s);

// Planning kernels (plan.cu).
struct PlanArgs {
    WorkItem *grid_cur;
    WorkItem *grid_next;
    WorkItem *scat;
    WorkItem *blocks;
    WorkItem *copies;
    u64 *hist;
    const u64 *orand;
    u32 *tile_hist;   // tile -> item map of histogram tiles (next level)
    u32 *tile_scat;   // tile -> item map of distribution tiles (this level)
    u32 *tile_copy;   // tile -> item map of copy tiles
    Counters *ctrs;
    Caps caps;
    u32 key_words;
    u32 rw;
    u32 cap_b;
    u32 warp_bin;     // sub-bins up to this size are sorted by one warp inside a run
    u32 tile_h, tile_s, tile_c;
    u32 single_pass;  // 1: distribute every item once, no children (single-step API)
    u32 top_digit;    // most significant key digit (8 * key_words - 1)
    WorkItem *buckets_cur;   // mid-size bins sorted by one CTA each in this level
    WorkItem *buckets_next;  // mid-size bins found in this level (sorted in the next one)
    WorkItem *buckets_split; // mid-size bins of this level with heavy code groups (stable split)
    u32 bucket_max;          // bins of plain digits with count <= bucket_max go there (0: never)
    u64 *bucket_scratch;     // bucket_max record slots per CTA of the mid-size bin kernel (bucket_slot_bytes each)
    const u32 *bucket_order;  // non-null: the mid-size kernel takes only window bucket_window of this list
    const u32 *bucket_wstart; // (bin indices grouped by position window; see launch_bucket_windows)
    u32 bucket_window;
    u64 *status;              // look-back status words of this level's chunks (then the digit starts)
    const u64 *cell_cur;      // first status word of every current grid item (by slot)
    u64 *cell_next;           // same for the next grid list
    u32 leaf;                 // sub-bin size the digit widths aim at
    u32 wmax;                 // widest digit of a pass (bits)
    const Model *model;       // the learned model of a learned pass (its buckets' key ranges)
};

// Position windows of the last mid-size level (an end-to-end sort copies each
// window back to the host while the next one is sorted).
constexpr u32 BUCKET_WINDOWS_MAX = 8;

// CTAs of the mid-size bin kernel (one per SM): its scratch holds that many regions.
u32 bucket_grid();
// Bytes of one record's slot in a mid-size CTA's scratch region (16-byte
// records take a whole 32-byte sector; see slot_words in midsize.cuh).
inline size_t bucket_slot_bytes(u32 rw) { return rw == 2 ? 32u : (size_t)rw * 8u; }

__device__ __forceinline__ u32 ceil_div_u64(u64 a, u32 b) { return (u32)((a + b - 1) / b); }

// Append a learned-digit or key-window bin to the next grid list, claim its
// look-back status words (chunks x 2^w) and map its histogram chunks.
__device__ __forceinline__ void append_grid_item(const PlanArgs &a, u64 begin, u64 count, u32 digit, u32 flags,
                                                 u32 w)
{
    const u32 slot = atomicAdd(&a.ctrs->grid_next, 1u);
    atomicMax(&a.ctrs->wmax_next, w);
    const u32 nt = ceil_div_u64(count, a.tile_h);
    const u32 tb = atomicAdd(&a.ctrs->grid_next_tiles, nt);
    const u64 cells = (u64)nt << w;
    const u64 co = atomicAdd(&a.ctrs->cells_next, cells);
    if (slot >= a.caps.grid || (u64)tb + nt > a.caps.hist_tiles || co + cells > a.caps.cells) {
        set_error(a.ctrs, ST_INTERNAL);
        return;
    }
    WorkItem it;
    it.begin = begin;
    it.count = count;
    it.digit = digit;
    it.flags = flags;
    it.tile_base = tb;
    it.row = slot;
    a.grid_next[slot] = it;
    a.cell_next[slot] = co;
    for (u32 j = 0; j < nt; ++j)
        a.tile_hist[tb + j] = slot;
}

// Append a bin whose records agree on every key bit at or above `hi`: a
// mid-size bin goes to the next level's mid-size list (no histogram pass: its
// kernel counts for itself, from the byte holding bit hi - 1 down), any other
// to the next grid list with a digit width picked for its size.
__device__ __forceinline__ void append_bin_hi(const PlanArgs &a, u64 begin, u64 count, u32 hi, u32 flags,
                                              u32 wmax = 0)
{
    flags &= ~(ITEM_W_MASK | ITEM_C_MASK);
    if (a.bucket_max && count <= a.bucket_max) {
        const u32 slot = atomicAdd(&a.ctrs->bucket_next, 1u);
        if (slot >= a.caps.grid) {
            set_error(a.ctrs, ST_INTERNAL);
            return;
        }
        WorkItem it;
        it.begin = begin;
        it.count = count;
        it.digit = (hi - 1u) / 8u;
        it.flags = flags;
        it.tile_base = 0;
        it.row = 0;
        a.buckets_next[slot] = it;
        return;
    }
    const u32 w = pick_width(count, hi, a.leaf, wmax ? wmax : a.wmax);
    u32 digit, fl;
    grid_pos(hi, w, flags, digit, fl);
    append_grid_item(a, begin, count, digit, fl, w);
}

// Same, for a bin whose key bytes above `digit` agree (byte-based callers).
__device__ __forceinline__ void append_bin(const PlanArgs &a, u64 begin, u64 count, u32 digit, u32 flags)
{
    append_bin_hi(a, begin, count, 8u * digit + 8u, flags);
}

// Mid-size bins (bucketsort.cu): every bin of a.buckets_cur is sorted by one
// CTA that reads it from HBM once and keeps its scratch copy in L2.
cudaError_t launch_bucket(const Shape &s, u64 *in, u64 *tmp, const PlanArgs &a, cudaStream_t st);

// Device queue of the batched persistent kernel: the mid-size arrays first
// (largest work), then the on-chip items (blocks list), then items the kernel
// pushes itself (slots published through ready[]).
struct BatchQueue {
    const WorkItem *mid;
    const WorkItem *blocks;
    WorkItem *dyn;
    u32 *ready;
    u32 cap_dyn;
    const u32 *withhold;  // device word: the pushed slot whose ready flag is withheld (test hook; ~0u: none)
};

cudaError_t launch_batched_persistent(const Shape &s, u64 *in, u64 *tmp, const PlanArgs &a, const BatchQueue &q,
                                      const u64 *seg_off, u64 wait_ns, cudaStream_t st);

cudaError_t launch_init(Counters *ctrs, WorkItem *grid0, WorkItem *blocks, u32 *tile_hist, u64 n, u32 top_digit,
                        u32 cap_b, u32 tile_h, u32 force_grid, WorkItem *bucket0, u32 bucket_max, u64 *cell0,
                        u32 leaf, u32 wmax, cudaStream_t st);
// Clear the level's OR / AND words (and, zero_rows, its per-bin histogram rows
// for the histogram-only traversal).
cudaError_t launch_prep(u64 *hist, u64 *orand, const Counters *ctrs, u32 n_grid_hint, u32 zero_rows,
                        cudaStream_t st);
cudaError_t launch_plan(const PlanArgs &a, u32 n_grid, cudaStream_t st);
cudaError_t launch_advance(Counters *ctrs, cudaStream_t st);
cudaError_t launch_keep_learned(Counters *ctrs, float ratio, cudaStream_t st);
cudaError_t launch_bucket_windows(const WorkItem *items, const Counters *ctrs, u64 n, u32 nw, u32 *order,
                                  u32 *wstart, cudaStream_t st);
cudaError_t launch_bucket_window_reset(Counters *ctrs, cudaStream_t st);
// On-chip items grouped by position window (as launch_bucket_windows), and
// the left-over list's counter moved past the items a window has finished.
cudaError_t launch_block_windows(const WorkItem *items, const Counters *ctrs, u64 n, u32 nw, u32 *order,
                                 u32 *wstart, cudaStream_t st);
cudaError_t launch_fb_window_reset(Counters *ctrs, cudaStream_t st);
cudaError_t launch_batched_init(const u64 *off, u32 n_segs, WorkItem *grid0, WorkItem *blocks, u32 *tile_hist,
                                Counters *ctrs, Caps caps, u32 top, u32 cap_b, u32 tile_h, WorkItem *bucket0,
                                u32 bucket_max, u64 *cell0, u32 leaf, u32 wmax, cudaStream_t st);
cudaError_t launch_check_drained(Counters *ctrs, cudaStream_t st);
cudaError_t launch_epoch_next(u32 *ep, u64 *status, u64 words, cudaStream_t st);
cudaError_t launch_copy(const Shape &s, u64 *in, const u64 *tmp, const WorkItem *copies, const u32 *tile_copy,
                        Counters *ctrs, cudaStream_t st);

// Key-index sort and runs of equal keys (extras.cu).
cudaError_t launch_build_pairs(const u64 *in, u64 n, u32 rw, u32 kw, u64 *pairs, cudaStream_t st);
cudaError_t launch_gather(const u64 *in, u64 n, u32 rw, const u64 *pairs, u32 pw, u64 *out, cudaStream_t st);
u64 rle_tiles(u64 n);
cudaError_t launch_rle(const u64 *in, u64 n, u32 rw, u32 kw, u64 *tile_buf, u64 *keys, u64 *counts, u64 *n_runs,
                       cudaStream_t st);

// Learned model (learned.cu).
cudaError_t lm_launch_sample(const u64 *in, u64 n, u32 rw, u32 S, u64 *out, cudaStream_t st);
cudaError_t lm_launch_build(const u64 *sample, u32 S, u32 k_extra, const u64 *root_hist, u64 n, u32 log2b,
                            const float *h, Model *M, u32 *seg_start, u32 max_knots, u64 *bmin, u64 *bmax,
                            cudaStream_t st);
cudaError_t lm_launch_init(float *theta, float *am, float *av, u32 n_params, cudaStream_t st);
cudaError_t lm_launch_step(const Model *M, u32 stage, float *theta, float *am, float *av, float *h, float *tot,
                           double *E, double *G, double *Z, double *loss, const u64 *sample, const u32 *seg_start,
                           u32 S, float lr, int step, float *grad_out, cudaStream_t st);
cudaError_t lm_launch_warm(const Model *M, u32 stage, const u64 *sample, const u32 *seg_start, float *theta,
                           cudaStream_t st);
cudaError_t lm_launch_heights(const Model *M, const float *theta, float *h, float *tot, double *E, double *G,
                              double *Z, double *loss, cudaStream_t st);
// Heavy keys of the sorted sample (runs of at least thr equal keys).
cudaError_t lm_launch_heavy(const u64 *sample, u32 S, u32 thr, u64 *heavy, Model *M, cudaStream_t st);
// The balance check of a model on its sample: the largest bucket load of the
// keys that are not heavy over the ideal S / B (load: KMAX u32 scratch).
cudaError_t lm_launch_ratio(const Model *M, const u64 *sample, u32 S, u32 *load, Counters *ctrs, float limit,
                            cudaStream_t st);
// Every bucket's key range back to empty (before a learned pass).
cudaError_t lm_launch_minmax_reset(const Model *M, cudaStream_t st);
cudaError_t lm_launch_bucket(const Model *M, const u64 *keys, u64 n, u32 *out, cudaStream_t st);

}  // namespace raduls
