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
                        const u32 *tile_item, u64 *hist, u64 *orand, Counters *ctrs, cudaStream_t st);
cudaError_t launch_scatter(const Shape &s, u64 *in, u64 *tmp, const WorkItem *items, const u32 *tile_item,
                           const u64 *bases, u64 *status, Counters *ctrs, u32 epoch, u64 wait_ns,
                           u32 inject_tile, cudaStream_t st);
cudaError_t launch_block_sort(const Shape &s, u64 *in, const u64 *tmp, const WorkItem *blocks,
                              Counters *ctrs, cudaStream_t st);

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
    u32 tile_h, tile_s, tile_c;
    u32 single_pass;  // 1: distribute every item once, no children (single-step API)
};

cudaError_t launch_init(Counters *ctrs, WorkItem *grid0, WorkItem *blocks, u32 *tile_hist, u64 n, u32 top_digit,
                        u32 cap_b, u32 tile_h, u32 force_grid, cudaStream_t st);
cudaError_t launch_prep(u64 *hist, u64 *orand, const Counters *ctrs, u32 n_grid_hint, cudaStream_t st);
cudaError_t launch_plan(const PlanArgs &a, u32 n_grid, cudaStream_t st);
cudaError_t launch_advance(Counters *ctrs, cudaStream_t st);
cudaError_t launch_copy(const Shape &s, u64 *in, const u64 *tmp, const WorkItem *copies, const u32 *tile_copy,
                        Counters *ctrs, cudaStream_t st);

}  // namespace raduls
