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
    int scat_var;    // distribution kernel variant
    int block_var;   // on-chip sort kernel variant
};

Shape choose_shape(u32 rw, u32 key_words);

// Persistent-grid sizes (CTAs) of each kernel for a shape on the current device.
u32 hist_grid(const Shape &s);
u32 scatter_grid(const Shape &s);
u32 block_grid(const Shape &s);
u32 copy_grid();

cudaError_t launch_hist(const Shape &s, const u64 *in, const u64 *tmp, const WorkItem *items,
                        const u32 *tile_item, u64 *hist, u64 *orand, u64 *dlight, Counters *ctrs,
                        const Model *model, cudaStream_t st);
cudaError_t launch_scatter(const Shape &s, u64 *in, u64 *tmp, const WorkItem *items, const u32 *tile_item,
                           const u64 *bases, u64 *status, Counters *ctrs, const u32 *epoch, u64 wait_ns,
                           u32 inject_tile, const Model *model, cudaStream_t st);
cudaError_t launch_block_sort(const Shape &s, u64 *in, const u64 *tmp, const WorkItem *blocks,
                              Counters *ctrs, const u64 *seg_off, cudaStream_t st);

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
};

cudaError_t launch_init(Counters *ctrs, WorkItem *grid0, WorkItem *blocks, u32 *tile_hist, u64 n, u32 top_digit,
                        u32 cap_b, u32 tile_h, u32 force_grid, cudaStream_t st);
cudaError_t launch_prep(u64 *hist, u64 *orand, u64 *dlight, const Counters *ctrs, u32 n_grid_hint,
                        cudaStream_t st);
cudaError_t launch_plan(const PlanArgs &a, u32 n_grid, cudaStream_t st);
cudaError_t launch_advance(Counters *ctrs, cudaStream_t st);
cudaError_t launch_batched_init(const u64 *off, u32 n_segs, WorkItem *grid0, WorkItem *blocks, u32 *tile_hist,
                                Counters *ctrs, Caps caps, u32 top, u32 cap_b, u32 tile_h, cudaStream_t st);
cudaError_t launch_epoch_next(u32 *ep, u64 *status, u64 words, cudaStream_t st);
cudaError_t launch_copy(const Shape &s, u64 *in, const u64 *tmp, const WorkItem *copies, const u32 *tile_copy,
                        Counters *ctrs, cudaStream_t st);

// Learned model (learned.cu).
cudaError_t lm_launch_sample(const u64 *in, u64 n, u32 rw, u32 S, u64 *out, cudaStream_t st);
cudaError_t lm_launch_build(const u64 *sample, u32 S, u32 k_extra, const u64 *root_hist, u64 n, u32 log2b,
                            const float *h, Model *M, u32 *seg_start, u32 max_knots, cudaStream_t st);
cudaError_t lm_launch_init(float *theta, float *am, float *av, u32 n_params, cudaStream_t st);
cudaError_t lm_launch_step(const Model *M, u32 stage, float *theta, float *am, float *av, float *h, float *tot,
                           double *E, double *G, double *Z, double *loss, const u64 *sample, const u32 *seg_start,
                           u32 S, float lr, int step, float *grad_out, cudaStream_t st);
cudaError_t lm_launch_warm(const Model *M, u32 stage, const u64 *sample, const u32 *seg_start, float *theta,
                           cudaStream_t st);
cudaError_t lm_launch_heights(const Model *M, const float *theta, float *h, float *tot, double *E, double *G,
                              double *Z, double *loss, cudaStream_t st);
cudaError_t lm_launch_ratio(const u64 *dlight, Counters *ctrs, const Model *M, float limit, cudaStream_t st);
cudaError_t lm_launch_heavy(const u64 *sample, u32 S, u32 thr, u64 *heavy, Model *M, cudaStream_t st);
cudaError_t lm_launch_bucket(const Model *M, const u64 *keys, u64 n, u32 *out, cudaStream_t st);

}  // namespace raduls
