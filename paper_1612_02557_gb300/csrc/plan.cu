// plan.cu -- device-side planning of the MSD recursion.
//
// After the histogram of every big bin is known, plan_kernel does on the GPU
// what the paper's scheduler does on the CPU (Fig. 1-3, Sec. 3.2-3.4): it
// turns each histogram into sub-bin offsets (exclusive prefix, Sec. 1), and
// sends every sub-bin where it belongs:
//   * still bigger than one CTA can sort on chip -> next device-wide pass on
//     the next digit (the "big bins" of Sec. 3.3, Fig. 2);
//   * small -> packed with its small neighbours into runs of at most cap_b
//     records that one CTA sorts on chip (the "small"/"tiny" bins of Sec. 3.4
//     and 3.5, Fig. 3);
//   * no digits left but still in the scratch buffer -> copied back.
// A bin small enough for one CTA to sort through L2 (bucket_max) goes to the
// mid-size list instead of the next grid list (bucketsort.cu).
// A bin whose digit is the same for all its records is not distributed: it
// moves on to its next varying digit without any data movement.
#include "kernels.h"

namespace raduls {

__device__ void append_copy(const PlanArgs &a, u64 begin, u64 count)
{
    const u32 slot = atomicAdd(&a.ctrs->copy, 1u);
    const u32 nt = ceil_div_u64(count, a.tile_c);
    const u32 tb = atomicAdd(&a.ctrs->copy_tiles, nt);
    if (slot >= a.caps.copy || (u64)tb + nt > a.caps.copy_tiles) {
        set_error(a.ctrs, ST_INTERNAL);
        return;
    }
    WorkItem it;
    it.begin = begin;
    it.count = count;
    it.digit = 0;
    it.flags = ITEM_IN_TMP;
    it.tile_base = tb;
    it.row = slot;
    a.copies[slot] = it;
    for (u32 j = 0; j < nt; ++j)
        a.tile_copy[tb + j] = slot;
}

__device__ void append_block(const PlanArgs &a, u64 begin, u64 count, u32 digit, u32 flags)
{
    const u64 slot = atomicAdd(&a.ctrs->block, 1ull);
    if (slot >= a.caps.block || count > a.cap_b) {
        set_error(a.ctrs, ST_INTERNAL);
        return;
    }
    WorkItem it;
    it.begin = begin;
    it.count = count;
    it.digit = digit;
    it.flags = flags;
    it.tile_base = 0;
    it.row = 0;
    a.blocks[slot] = it;
}

// A learned bucket whose key word 0 is the same for all its records: with a
// one-word key its records are equal keys, already in their stable order.
__device__ __forceinline__ bool bucket_single_key(const PlanArgs &a, u32 c)
{
    return a.model && a.model->bmin[c] == a.model->bmax[c];
}

// A learned bucket of more than cap_b records: sorted from the highest bit of
// key word 0 that varies inside it (from its smallest and largest key), or
// from key word 1 when its word 0 is one value; a one-word bucket of one
// value is finished.
__device__ __forceinline__ void learned_child(const PlanArgs &a, u32 c, u64 begin, u64 count, u32 flags)
{
    if (bucket_single_key(a, c)) {
        if (a.key_words > 1u)
            append_bin_hi(a, begin, count, 64u * (a.key_words - 1u), flags);
        else if (flags & ITEM_IN_TMP)
            append_copy(a, begin, count);
        return;
    }
    // the bucket's keys agree on every bit of word 0 above the highest one in
    // which its smallest and largest key differ: the next pass starts there
    const u64 diff = a.model->bmin[c] ^ a.model->bmax[c];
    append_bin_hi(a, begin, count, 64u * (a.key_words - 1u) + 64u - (u32)__clzll((long long)diff), flags);
}

// The highest key bit below `lo` that may still vary inside a bin whose key
// word `word` has OR `vor` and AND `vand` over its records, plus one (0: none
// left).  Bits below lo inside that word are checked; when all of them are
// constant, the next word's top is returned (its own histogram will tell).
__device__ __forceinline__ u32 next_varying_hi(u32 lo, u64 vor, u64 vand)
{
    if (lo == 0)
        return 0;
    const u32 sl = lo % 64u;
    if (sl == 0)
        return lo;
    const u64 diff = (vor ^ vand) & ((1ull << sl) - 1ull);
    return diff ? (lo - sl) + (64u - (u32)__clzll((long long)diff)) : lo - sl;
}

constexpr u32 PLAN_THREADS = 256;
constexpr u64 PLAN_SKEW = 8;  // a sub-bin this many times the mean marks a skewed bin

// Block-wide exclusive scan of one u64 per thread (PLAN_THREADS threads);
// `total` gets the sum.  Contains barriers.
__device__ __forceinline__ u64 plan_scan(u64 v, u64 &total, u64 *wsum)
{
    const u32 lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    u64 incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u64 x = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= (u32)o)
            incl += x;
    }
    if (lane == 31)
        wsum[w] = incl;
    __syncthreads();
    u64 add = 0, tot = 0;
#pragma unroll
    for (u32 i = 0; i < PLAN_THREADS / 32; ++i) {
        add += i < w ? wsum[i] : 0ull;
        tot += wsum[i];
    }
    total = tot;
    __syncthreads();
    return add + incl - v;
}

// One CTA per big bin of the level: its histogram is the inclusive counts its
// last chunk published; the exclusive prefix of it (Sec. 1) gives every
// sub-bin's start, written over those counts for the distribution kernel.
// Then every sub-bin is sent where it belongs (see the file comment).
__global__ void __launch_bounds__(PLAN_THREADS) plan_kernel(PlanArgs a)
{
    __shared__ u64 s_wsum[PLAN_THREADS / 32];
    __shared__ u64 s_key[KMAX];            // run key of every small sub-bin (~0: not small)
    __shared__ u32 s_slot, s_tb, s_nt;
    __shared__ u64 s_blk;
    __shared__ u32 s_err;
    const u32 tid = threadIdx.x;
    if (tid == 0)
        s_err = ld_relaxed_u32(&a.ctrs->err);
    __syncthreads();
    if (s_err)
        return;  // a histogram that failed (timeout) leaves nothing to plan
    const u32 n_grid = a.ctrs->grid_cur;
    const u32 smallmax = a.cap_b / 2u < a.warp_bin ? a.cap_b / 2u : a.warp_bin;
    const u64 run_target = a.cap_b - smallmax;
    for (u32 g = blockIdx.x; g < n_grid; g += gridDim.x) {
        const WorkItem it = a.grid_cur[g];
        const u32 p = it.digit;
        const bool learned = p == DIGIT_LEARNED;
        const u32 wb = item_w(it.flags);
        const u32 K = 1u << wb;
        const u32 hi = learned ? 0u : item_hi(p, it.flags);
        const u32 lo = learned ? 0u : hi - wb;
        const u32 nch = ceil_div_u64(it.count, a.tile_h);
        u64 *row = a.status + a.cell_cur[g] + (u64)(nch - 1u) * K;
        if (learned && !a.ctrs->learned_ok) {
            // the learned partition failed its balance check: the bin is not
            // distributed on it and goes on with the plain key digits
            if (tid == 0)
                append_bin(a, it.begin, it.count, a.top_digit, it.flags);
            __syncthreads();
            continue;
        }
        // this thread's values: [v0, v0 + nv)
        const u32 per = K >= PLAN_THREADS ? K / PLAN_THREADS : 1u;
        const u32 v0 = K >= PLAN_THREADS ? tid * per : tid;
        const u32 nv = (K >= PLAN_THREADS || tid < K) ? per : 0u;
        u64 part = 0;
        bool cst = false, heavy = false;
        for (u32 i = 0; i < nv; ++i) {
            const u64 h = row[v0 + i] & LB_VAL_MASK;
            part += h;
            cst |= (h == it.count);
            heavy |= h * K > PLAN_SKEW * it.count;
        }
        const int is_const = __syncthreads_or(cst);
        // a sub-bin far above the bin's mean: the keys are skewed, and the
        // children split 8 bits at a time (wider digits would leave many small
        // sub-bins behind)
        const u32 child_wmax = __syncthreads_or(heavy) ? 8u : 0u;
        const u64 vor = a.orand[2ull * g], vand = a.orand[2ull * g + 1];
        // children skip the bits below the window that are constant in the whole bin
        const u32 chi = learned ? 0u : next_varying_hi(lo, vor, vand);
        if (is_const && !a.single_pass) {
            // a constant digit: no data movement, the bin moves on
            if (tid == 0) {
                if (learned) {
                    append_bin(a, it.begin, it.count, a.top_digit, it.flags);
                } else {
                    atomicAdd(&a.ctrs->skipped, (u64)(hi - chi));
                    if (chi > 0)
                        append_bin_hi(a, it.begin, it.count, chi, it.flags);
                    else if (it.flags & ITEM_IN_TMP)
                        append_copy(a, it.begin, it.count);
                }
            }
            __syncthreads();
            continue;
        }
        // this bin is distributed in this level's pass, chunk by chunk
        if (tid == 0) {
            const u32 slot = atomicAdd(&a.ctrs->scatter, 1u);
            const u32 tb = atomicAdd(&a.ctrs->scatter_tiles, nch);
            if (slot >= a.caps.grid || (u64)tb + nch > a.caps.scat_tiles) {
                set_error(a.ctrs, ST_INTERNAL);
                s_nt = 0;
            } else {
                WorkItem sc = it;
                sc.tile_base = tb;
                sc.row = g;
                a.scat[slot] = sc;
                s_nt = nch;
            }
            s_slot = slot;
            s_tb = tb;
        }
        // exclusive prefix of the histogram: the start of every sub-bin (Sec. 1)
        u64 total = 0;
        u64 run = it.begin + plan_scan(part, total, s_wsum);
        for (u32 i = 0; i < nv; ++i) {
            const u64 h = row[v0 + i] & LB_VAL_MASK;
            row[v0 + i] = run;  // the row becomes the sub-bin starts
            run += h;
        }
        for (u32 jj = tid; jj < s_nt; jj += PLAN_THREADS)
            a.tile_scat[s_tb + jj] = s_slot;
        if (a.single_pass) {
            __syncthreads();
            continue;
        }
        const u32 cflags = it.flags ^ ITEM_IN_TMP;
        const bool to_in = (cflags & ITEM_IN_TMP) != 0;  // children sit in tmp and must come back
        const u64 end = it.begin + it.count;
        if (!learned && chi == 0) {
            // no key bit left that varies: every sub-bin is final, only to move back
            if (tid == 0 && to_in)
                append_copy(a, it.begin, it.count);
            __syncthreads();
            continue;
        }
        __syncthreads();  // every start is written
        auto start_of = [&](u32 c) { return c < K ? row[c] : end; };
        // big sub-bins go on by themselves; small ones are counted into run keys
        u64 kpart = 0;  // (non-small sub-bins << 48) | small records
        for (u32 i = 0; i < nv; ++i) {
            const u32 c = v0 + i;
            const u64 b = start_of(c), h = start_of(c + 1) - b;
            if (h > a.cap_b) {
                if (learned)
                    learned_child(a, c, b, h, cflags);
                else
                    append_bin_hi(a, b, h, chi, cflags, child_wmax);
            }
            const bool small = !learned && h <= smallmax;
            kpart += small ? h : (1ull << 48);
        }
        u64 ktot = 0;
        u64 kex = plan_scan(kpart, ktot, s_wsum);
        for (u32 i = 0; i < nv; ++i) {
            const u32 c = v0 + i;
            const u64 h = start_of(c + 1) - start_of(c);
            const bool small = !learned && h <= smallmax;
            s_key[c] = small ? (((kex >> 48) << 40) | (((kex & ((1ull << 48) - 1ull)) / run_target) << 8) |
                                (u64)(c >> 8))
                             : ~0ull;
            kex += small ? h : (1ull << 48);
        }
        __syncthreads();
        // on-chip items: runs of small sub-bins (one per run head) and single
        // sub-bins up to cap_b records; one reservation per bin
        auto is_head = [&](u32 c) {
            return s_key[c] != ~0ull && (c == 0 || s_key[c - 1] != s_key[c]);
        };
        auto run_end = [&](u32 c) {
            u32 e = c + 1;
            while (e < K && s_key[e] == s_key[c])
                ++e;
            return e;
        };
        // a small learned bucket of one key value (one-word keys) needs no sort
        auto done_bucket = [&](u32 c) { return learned && a.key_words == 1u && bucket_single_key(a, c); };
        auto single = [&](u64 h) { return h > 1 && h <= a.cap_b && (learned || h > smallmax); };
        u64 nitems = 0;
        for (u32 i = 0; i < nv; ++i) {
            const u32 c = v0 + i;
            const u64 b = start_of(c), h = start_of(c + 1) - b;
            if (is_head(c)) {
                const u64 rc = start_of(run_end(c)) - b;
                nitems += (rc > 1 || (rc == 1 && to_in)) ? 1u : 0u;
            } else if (single(h) && !(h > 0 && done_bucket(c))) {
                nitems += 1;
            }
        }
        u64 ntot = 0;
        u64 nex = plan_scan(nitems, ntot, s_wsum);
        if (tid == 0)
            s_blk = ntot ? atomicAdd(&a.ctrs->block, ntot) : 0ull;
        __syncthreads();
        if (s_blk + ntot > a.caps.block) {
            if (tid == 0)
                set_error(a.ctrs, ST_INTERNAL);
            __syncthreads();
            continue;
        }
        u64 slot = s_blk + nex;
        for (u32 i = 0; i < nv; ++i) {
            const u32 c = v0 + i;
            const u64 b = start_of(c), h = start_of(c + 1) - b;
            WorkItem bi;
            bi.tile_base = 0;
            bi.row = 0;
            if (is_head(c)) {
                const u64 rc = start_of(run_end(c)) - b;
                if (rc > 1 || (rc == 1 && to_in)) {
                    bi.begin = b;
                    bi.count = rc;
                    bi.digit = lo;  // a run holds the parent's window
                    bi.flags = (cflags & ~(ITEM_W_MASK | ITEM_C_MASK)) | ITEM_RUN | (wb << ITEM_W_SHIFT);
                    a.blocks[slot++] = bi;
                }
            } else if (h > 0 && h <= a.cap_b && done_bucket(c)) {
                if (to_in)
                    append_copy(a, b, h);
            } else if (single(h)) {
                bi.begin = b;
                bi.count = h;
                bi.flags = cflags & ~(ITEM_W_MASK | ITEM_C_MASK);
                if (learned && bucket_single_key(a, c))
                    grid_pos(64u * (a.key_words - 1u), 8u, bi.flags, bi.digit, bi.flags);  // from key word 1
                else if (learned)
                    bi.digit = a.top_digit;
                else
                    grid_pos(chi, 8u, bi.flags, bi.digit, bi.flags);  // exact top bit for the on-chip sort
                a.blocks[slot++] = bi;
            } else if (learned && h == 1 && to_in) {
                append_copy(a, b, h);
            }
        }
        __syncthreads();
    }
}

// The first level's work item: the whole input as one grid bin (with a digit
// width picked for its size; wmax == 0: the byte `top` itself, for the single
// step entry points and the learned first pass), one mid-size bin or one
// on-chip item.
__global__ void init_kernel(Counters *ctrs, WorkItem *grid0, WorkItem *blocks, u32 *tile_hist, u64 n, u32 top,
                            u32 cap_b, u32 tile_h, u32 force_grid, WorkItem *bucket0, u32 bucket_max, u64 *cell0,
                            u32 leaf, u32 wmax)
{
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    const bool mid = !force_grid && n > cap_b && n <= bucket_max;
    const bool grid = !mid && (force_grid || n > cap_b);
    const u32 nt = grid ? (u32)((n + tile_h - 1) / tile_h) : 0u;
    if (i == 0) {
        Counters c = {};
        if (mid) {
            WorkItem it = {0ull, n, top, 0u, 0u, 0u};
            bucket0[0] = it;
            c.bucket_cur = 1;
        } else if (grid) {
            // the learned digit takes wmax bits (log2 of the model's bucket count)
            u32 w = (top == DIGIT_LEARNED && wmax > 0) ? wmax : 8u;
            WorkItem it = {0ull, n, top, w << ITEM_W_SHIFT, 0u, 0u};
            if (top != DIGIT_LEARNED && wmax > 0) {
                w = pick_width(n, 8u * top + 8u, leaf, wmax);
                grid_pos(8u * top + 8u, w, 0u, it.digit, it.flags);
            }
            grid0[0] = it;
            if (cell0)
                cell0[0] = 0;
            c.grid_cur = 1;
            c.grid_cur_tiles = nt;
            c.cells_cur = (u64)nt << w;
        } else if (n > 1) {
            WorkItem it = {0ull, n, top, 0u, 0u, 0u};
            blocks[0] = it;
            c.block = 1;
        }
        *ctrs = c;
    }
    for (u64 j = i; j < nt; j += (u64)gridDim.x * blockDim.x)
        tile_hist[j] = 0;
}

__global__ void prep_kernel(u64 *hist, u64 *orand, const Counters *ctrs, u32 zero_rows)
{
    const u64 rows = ctrs->grid_cur;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; zero_rows && i < rows * RADIX; i += stride)
        hist[i] = 0;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += stride) {
        orand[2 * i] = 0;
        orand[2 * i + 1] = ~0ull;
    }
}

// After the learned pass's restart (init clears the counters): its balance
// check passed with this ratio.
__global__ void keep_learned_kernel(Counters *c, float ratio)
{
    c->learned_ok = 1;
    c->learned_fell_back = 0;
    c->learned_ratio = ratio;
}

cudaError_t launch_keep_learned(Counters *ctrs, float ratio, cudaStream_t st)
{
    keep_learned_kernel<<<1, 1, 0, st>>>(ctrs, ratio);
    return cudaGetLastError();
}

__global__ void advance_kernel(Counters *c)
{
    c->levels += 1;
    if (c->scatter)
        c->grid_passes += 1;
    c->grid_cur = c->grid_next;
    c->grid_cur_tiles = c->grid_next_tiles;
    c->cells_cur = c->cells_next;
    c->cells_next = 0;
    c->wmax_cur = c->wmax_next;
    c->wmax_next = 0;
    c->grid_next = 0;
    c->grid_next_tiles = 0;
    c->scatter = 0;
    c->scatter_tiles = 0;
    c->tile_ctr[0] = 0;
    c->tile_ctr[1] = 0;
    c->bucket_cur = c->bucket_next;
    c->bucket_next = 0;
    c->bucket_split = 0;
    c->split_ctr = 0;
    c->tile_ctr[4] = 0;
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS)
copy_kernel(u64 *__restrict__ in, const u64 *__restrict__ tmp, const WorkItem *__restrict__ copies,
            const u32 *__restrict__ tile_copy, Counters *__restrict__ ctrs, u32 tile_c, u32 rw)
{
    __shared__ u32 s_tile;
    if (cta_failed(ctrs))
        return;
    const u32 n_tiles = ctrs->copy_tiles;
    for (;;) {
        if (threadIdx.x == 0)
            s_tile = atomicAdd(&ctrs->tile_ctr[2], 1u);
        __syncthreads();
        const u32 t = s_tile;
        __syncthreads();
        if (t >= n_tiles)
            break;
        const WorkItem it = copies[tile_copy[t]];
        const u64 lo = it.begin + (u64)(t - it.tile_base) * tile_c;
        const u64 hi = min(it.begin + it.count, lo + tile_c);
        const u64 w0 = lo * rw, w1 = hi * rw;
        for (u64 i = w0 + threadIdx.x; i < w1; i += THREADS)
            in[i] = __ldcs(tmp + i);
        if (threadIdx.x == 0)
            atomicAdd(&ctrs->block_bytes, 2ull * (w1 - w0) * 8u);
    }
}

// ------------------------------------------------------------ batched sort

__global__ void batched_reset_kernel(Counters *ctrs)
{
    Counters c = {};
    *ctrs = c;
}

// Offsets must start at 0 and never decrease; otherwise nothing is sorted.
__global__ void batched_validate_kernel(const u64 *__restrict__ off, u32 n_segs, Counters *ctrs)
{
    for (u32 s = blockIdx.x * blockDim.x + threadIdx.x; s < n_segs; s += gridDim.x * blockDim.x)
        if (off[s + 1] < off[s] || (s == 0 && off[0] != 0))
            set_error(ctrs, ST_BAD_ARG);
}

// Classify every array by size: bigger than a mid-size bin -> first grid list
// (its top key digit); bigger than cap_b -> the persistent kernel's mid-size
// queue; bigger than warp_bin -> one on-chip item; otherwise -> a run of
// consecutive small arrays whose starts share a window of `win` records and
// whose indices share a block of 256 (so a run holds < cap_b records and at
// most 256 arrays), sorted one warp per array.
__global__ void batched_classify_kernel(const u64 *__restrict__ off, u32 n_segs, WorkItem *grid0, WorkItem *blocks,
                                        u32 *tile_hist, Counters *ctrs, Caps caps, u32 top, u32 cap_b, u32 warp_bin,
                                        u32 tile_h, u32 win, WorkItem *bucket0, u32 bucket_max, u64 *cell0, u32 leaf,
                                        u32 wmax)
{
    if (ctrs->err)
        return;
    auto small = [&](u32 s) { return off[s + 1] - off[s] <= warp_bin; };
    auto key = [&](u32 s) { return (off[s] / win) * 1048576ull + (s >> 8); };
    for (u32 s = blockIdx.x * blockDim.x + threadIdx.x; s < n_segs; s += gridDim.x * blockDim.x) {
        const u64 a = off[s], c = off[s + 1] - a;
        if (c > cap_b && c <= bucket_max) {
            // mid-size arrays: the persistent kernel's queue (largest work first)
            const u32 slot = atomicAdd(&ctrs->bmid, 1u);
            if (slot >= n_segs) {
                set_error(ctrs, ST_INTERNAL);
                continue;
            }
            WorkItem it = {a, c, top, 0u, 0u, 0u};
            bucket0[slot] = it;
        } else if (c > cap_b) {
            const u32 slot = atomicAdd(&ctrs->grid_cur, 1u);
            const u32 nt = (u32)((c + tile_h - 1) / tile_h);
            const u32 tb = atomicAdd(&ctrs->grid_cur_tiles, nt);
            const u32 w = pick_width(c, 8u * top + 8u, leaf, wmax);
            const u64 cells = (u64)nt << w;
            const u64 co = atomicAdd(&ctrs->cells_cur, cells);
            if (slot >= caps.grid || (u64)tb + nt > caps.hist_tiles || co + cells > caps.cells) {
                set_error(ctrs, ST_INTERNAL);
                continue;
            }
            WorkItem it = {a, c, top, 0u, tb, slot};
            grid_pos(8u * top + 8u, w, 0u, it.digit, it.flags);
            grid0[slot] = it;
            cell0[slot] = co;
            for (u32 t = 0; t < nt; ++t)
                tile_hist[tb + t] = slot;
        } else if (c > warp_bin) {
            const u64 slot = atomicAdd(&ctrs->block, 1ull);
            if (slot >= caps.block) {
                set_error(ctrs, ST_INTERNAL);
                continue;
            }
            WorkItem it = {a, c, top, 0u, 0u, 0u};
            blocks[slot] = it;
        } else if (s == 0 || !small(s - 1) || key(s - 1) != key(s)) {
            u32 e = s + 1;
            while (e < n_segs && small(e) && key(e) == key(s))
                ++e;
            const u64 total = off[e] - a;
            if (total > 1) {
                const u64 slot = atomicAdd(&ctrs->block, 1ull);
                if (slot >= caps.block) {
                    set_error(ctrs, ST_INTERNAL);
                    continue;
                }
                WorkItem it = {a, total, top, ITEM_RUN | ITEM_SEG, s, e - s};
                blocks[slot] = it;
            }
        }
    }
}

// After the last level nothing may be left unsorted.
__global__ void check_drained_kernel(Counters *ctrs)
{
    if (ctrs->grid_cur != 0 || ctrs->bucket_cur != 0)
        set_error(ctrs, ST_INTERNAL);
}

cudaError_t launch_check_drained(Counters *ctrs, cudaStream_t st)
{
    check_drained_kernel<<<1, 1, 0, st>>>(ctrs);
    return cudaGetLastError();
}

cudaError_t launch_batched_init(const u64 *off, u32 n_segs, WorkItem *grid0, WorkItem *blocks, u32 *tile_hist,
                                Counters *ctrs, Caps caps, u32 top, u32 cap_b, u32 tile_h, WorkItem *bucket0,
                                u32 bucket_max, u64 *cell0, u32 leaf, u32 wmax, cudaStream_t st)
{
    batched_reset_kernel<<<1, 1, 0, st>>>(ctrs);
    const u32 blocks_n = n_segs / 256 + 1 < 4096 ? n_segs / 256 + 1 : 4096;
    batched_validate_kernel<<<blocks_n, 256, 0, st>>>(off, n_segs, ctrs);
    batched_classify_kernel<<<blocks_n, 256, 0, st>>>(off, n_segs, grid0, blocks, tile_hist, ctrs, caps, top, cap_b,
                                                      WARP_BIN, tile_h, cap_b - WARP_BIN, bucket0, bucket_max, cell0,
                                                      leaf, wmax);
    return cudaGetLastError();
}

// Look-back epoch held on the device: the next distribution launch's epoch.
// When it would wrap, the status words are cleared first (wrap flag ep[1]).
__global__ void epoch_next_kernel(u32 *ep)
{
    u32 e = ep[0] + 1u;
    ep[1] = 0;
    if (e >= LB_EPOCH_MASK) {
        e = 1;
        ep[1] = 1;
    }
    ep[0] = e;
}

__global__ void status_clear_kernel(const u32 *ep, u64 *status, u64 words)
{
    if (!ep[1])
        return;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (u64)gridDim.x * blockDim.x)
        status[i] = 0;
}

cudaError_t launch_epoch_next(u32 *ep, u64 *status, u64 words, cudaStream_t st)
{
    epoch_next_kernel<<<1, 1, 0, st>>>(ep);
    status_clear_kernel<<<1024, 256, 0, st>>>(ep, status, words);
    return cudaGetLastError();
}

cudaError_t launch_init(Counters *ctrs, WorkItem *grid0, WorkItem *blocks, u32 *tile_hist, u64 n, u32 top_digit,
                        u32 cap_b, u32 tile_h, u32 force_grid, WorkItem *bucket0, u32 bucket_max, u64 *cell0,
                        u32 leaf, u32 wmax, cudaStream_t st)
{
    init_kernel<<<256, 256, 0, st>>>(ctrs, grid0, blocks, tile_hist, n, top_digit, cap_b, tile_h, force_grid, bucket0,
                                     bucket_max, cell0, leaf, wmax);
    return cudaGetLastError();
}

cudaError_t launch_prep(u64 *hist, u64 *orand, const Counters *ctrs, u32 n_grid_hint, u32 zero_rows, cudaStream_t st)
{
    u64 work = (u64)n_grid_hint * (zero_rows ? RADIX : 1u);
    u64 want = (work + 255) / 256 + 1;
    u32 blocks = (u32)(want < 4096ull ? want : 4096ull);
    prep_kernel<<<blocks, 256, 0, st>>>(hist, orand, ctrs, zero_rows);
    return cudaGetLastError();
}

cudaError_t launch_plan(const PlanArgs &a, u32 n_grid, cudaStream_t st)
{
    // n_grid == 0: count unknown on the host (device-driven levels): a fixed grid loops
    u32 blocks = n_grid == 0 ? 1216u : (n_grid < 65535u ? n_grid : 65535u);
    plan_kernel<<<blocks, PLAN_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_advance(Counters *ctrs, cudaStream_t st)
{
    advance_kernel<<<1, 1, 0, st>>>(ctrs);
    return cudaGetLastError();
}

// Mid-size bins of this level grouped by position window: window w holds the
// bins whose first record lies in [w n / nw, (w + 1) n / nw).  order[] lists
// bin indices window by window (any order inside a window), wstart[w] is
// where window w starts in order[] (wstart[nw] = number of bins).
__global__ void __launch_bounds__(1024)
bucket_window_kernel(const WorkItem *__restrict__ items, const Counters *__restrict__ ctrs, u64 n, u32 nw,
                     u32 *__restrict__ order, u32 *__restrict__ wstart)
{
    __shared__ u32 cnt[BUCKET_WINDOWS_MAX], pos[BUCKET_WINDOWS_MAX];
    const u32 m = ctrs->bucket_cur;
    const u32 tid = threadIdx.x;
    auto win_of = [&](u64 b) {
        const u64 w = n ? b * nw / n : 0;
        return (u32)(w < nw ? w : nw - 1u);
    };
    if (tid < BUCKET_WINDOWS_MAX)
        cnt[tid] = 0;
    __syncthreads();
    for (u32 i = tid; i < m; i += blockDim.x)
        atomicAdd(&cnt[win_of(items[i].begin)], 1u);
    __syncthreads();
    if (tid == 0) {
        u32 acc = 0;
        for (u32 w = 0; w < nw; ++w) {
            wstart[w] = acc;
            pos[w] = acc;
            acc += cnt[w];
        }
        wstart[nw] = acc;
    }
    __syncthreads();
    for (u32 i = tid; i < m; i += blockDim.x)
        order[atomicAdd(&pos[win_of(items[i].begin)], 1u)] = i;
}

// The same grouping for the on-chip items (end-to-end sorts whose last step
// is the streamed bin sort): order[] lists indices into the on-chip list
// window by window, wstart[w] is where window w starts.
__global__ void __launch_bounds__(1024)
block_window_kernel(const WorkItem *__restrict__ items, const Counters *__restrict__ ctrs, u64 n, u32 nw,
                    u32 *__restrict__ order, u32 *__restrict__ wstart)
{
    __shared__ u32 cnt[BUCKET_WINDOWS_MAX], pos[BUCKET_WINDOWS_MAX];
    const u64 m = ctrs->block;
    const u32 tid = threadIdx.x;
    auto win_of = [&](u64 b) {
        const u64 w = n ? b * nw / n : 0;
        return (u32)(w < nw ? w : nw - 1u);
    };
    if (tid < BUCKET_WINDOWS_MAX)
        cnt[tid] = 0;
    __syncthreads();
    for (u64 i = tid; i < m; i += blockDim.x)
        atomicAdd(&cnt[win_of(items[i].begin)], 1u);
    __syncthreads();
    if (tid == 0) {
        u32 acc = 0;
        for (u32 w = 0; w < nw; ++w) {
            wstart[w] = acc;
            pos[w] = acc;
            acc += cnt[w];
        }
        wstart[nw] = acc;
    }
    __syncthreads();
    for (u64 i = tid; i < m; i += blockDim.x)
        order[atomicAdd(&pos[win_of(items[i].begin)], 1u)] = (u32)i;
}

// After a window's left-overs are sorted: every item on the left-over list so
// far is done, the next window's general kernel starts after them.
__global__ void fb_window_reset_kernel(Counters *c)
{
    c->fb_ctr = (u32)c->block_fb;
}

// Before the next window: the mid-size kernel's item counter and this level's
// stable-split list start over (the previous window's split items are done).
__global__ void bucket_window_reset_kernel(Counters *c)
{
    c->tile_ctr[4] = 0;
    c->bucket_split = 0;
    c->split_ctr = 0;
}

cudaError_t launch_bucket_windows(const WorkItem *items, const Counters *ctrs, u64 n, u32 nw, u32 *order,
                                  u32 *wstart, cudaStream_t st)
{
    if (nw < 1 || nw > BUCKET_WINDOWS_MAX)
        return cudaErrorInvalidValue;
    bucket_window_kernel<<<1, 1024, 0, st>>>(items, ctrs, n, nw, order, wstart);
    return cudaGetLastError();
}

cudaError_t launch_block_windows(const WorkItem *items, const Counters *ctrs, u64 n, u32 nw, u32 *order,
                                 u32 *wstart, cudaStream_t st)
{
    if (nw < 1 || nw > BUCKET_WINDOWS_MAX)
        return cudaErrorInvalidValue;
    block_window_kernel<<<1, 1024, 0, st>>>(items, ctrs, n, nw, order, wstart);
    return cudaGetLastError();
}

cudaError_t launch_fb_window_reset(Counters *ctrs, cudaStream_t st)
{
    fb_window_reset_kernel<<<1, 1, 0, st>>>(ctrs);
    return cudaGetLastError();
}

cudaError_t launch_bucket_window_reset(Counters *ctrs, cudaStream_t st)
{
    bucket_window_reset_kernel<<<1, 1, 0, st>>>(ctrs);
    return cudaGetLastError();
}

u32 copy_grid()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (u32)sms * 4u;
}

cudaError_t launch_copy(const Shape &s, u64 *in, const u64 *tmp, const WorkItem *copies, const u32 *tile_copy,
                        Counters *ctrs, cudaStream_t st)
{
    copy_kernel<256><<<copy_grid(), 256, 0, st>>>(in, tmp, copies, tile_copy, ctrs, s.tile_c, s.rw);
    return cudaGetLastError();
}

}  // namespace raduls
