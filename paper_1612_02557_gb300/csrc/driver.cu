// driver.cu -- host driver and C ABI of the sorter (see include/raduls.h).
//
// The driver plays the part of the paper's scheduler (Fig. 1-3) with GPU work
// lists instead of threads and queues: it runs one MSD level at a time --
// histograms of every big bin, on-device planning, one device-wide
// distribution launch for all big bins of the level -- until no bin is bigger
// than what one CTA sorts on chip, then copies back finished bins left in the
// scratch buffer and runs the on-chip sorts of all small-bin runs.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "../../include/raduls.h"
#include "kernels.h"

namespace raduls {

u32 block_cap_of(int var);

// The distribution shape of a record width that takes digits of up to
// WIDE_MAX bits (one CTA per SM): for a learned pass with that many buckets.
int wide_scatter_variant(u32 rw)
{
    return rw == 1 ? 0 : rw == 2 ? 1 : rw == 4 ? 2 : rw <= 8 ? 3 : 4;
}

// Distribution variants that fit a record width (see WSCATTER_VARIANTS).
bool scatter_variant_fits(int v, u32 rw)
{
    switch (v) {
    case 0:
        return rw == 1;
    case 1:
    case 5:
    case 8:
    case 9:
    case 10:
    case 11:
    case 16:
    case 17:
    case 18:
    case 19:
    case 20:
    case 21:
        return rw == 2;
    case 6:
    case 12:
    case 13:
        return rw == 1;
    case 14:
    case 15:
        return rw == 4;
    case 2:
    case 7:
        return rw == 4;
    case 3:
        return rw <= 8;
    case 4:
        return true;
    default:
        return false;
    }
}

namespace {

// Settings picked by raduls_autotune, per device, record width and call kind
// (plain, batched); `force` is the candidate being timed by the tuner itself.
struct Tuned {
    bool valid = false;
    int scat_var = 0;
    u32 cap_b = 0;
    u32 bucket_max = 0;
    u32 wmax = 0;   // widest digit of a distribution pass (0: default)
    u32 leaf = 0;   // sub-bin size the digit widths aim at (0: default)
    int bins = 0;   // streamed on-chip finisher: 0 default, 1 on, 2 off
};
constexpr int TUNE_DEVICES = 64;
Tuned g_tuned[TUNE_DEVICES][2][33];
std::mutex g_tuned_mu;
thread_local const Tuned *g_force = nullptr;

}  // namespace

Shape choose_shape(u32 rw, u32 key_words, bool batched)
{
    Shape s{};
    s.rw = rw;
    s.key_words = key_words;
    s.tile_h = 65536;   // records per chunk of a distribution pass
    s.tile_c = 65536;
    // default distribution shapes: two CTAs per SM with 8-bit digits (the
    // autotuner also times the one-CTA shapes that take digits of up to 10 bits)
    if (rw == 1) {
        s.scat_var = 6;
        s.block_var = 0;
    } else if (rw == 2) {
        // plain sorts: digits of up to 10 bits, two CTAs per SM; batched sorts
        // keep 8-bit digits (their arrays are mostly below one chunk)
        s.scat_var = batched ? 5 : 11;
        s.block_var = 1;
    } else if (rw == 4) {
        s.scat_var = batched ? 7 : 15;
        s.block_var = 2;
    } else if (rw <= 8) {
        s.scat_var = 3;
        s.block_var = 3;
    } else {
        s.scat_var = 4;
        s.block_var = 4;
    }
    s.cap_b = block_cap_of(s.block_var);
    // mid-size bins: one CTA sorts a bin of up to BUCKET_BYTES through L2
    constexpr u32 BUCKET_BYTES = 640u * 1024u;
    s.bucket_var = rw == 1 ? 0 : rw == 2 ? 1 : rw == 4 ? 2 : -1;
    // Plain sorts of record widths with a streamed on-chip sort leave the
    // class off by default: wider digits and that sort finish such bins
    // faster (skewed 2^30 x 16 B: 82.7 against 86.4 ms); batched sorts keep
    // it for their mid-size arrays.
    s.bucket_max = (s.bucket_var < 0 || (!batched && binsort_variant_for(rw) >= 0)) ? 0u : BUCKET_BYTES / (rw * 8u);
    // tuned settings (raduls_autotune), else the defaults above
    Tuned t{};
    if (g_force) {
        t = *g_force;
    } else {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < TUNE_DEVICES && rw <= 32) {
            std::lock_guard<std::mutex> g(g_tuned_mu);
            t = g_tuned[dev][batched ? 1 : 0][rw];
        } else {
            cudaGetLastError();
        }
    }
    s.wmax = WIDE_MAX;
    s.leaf = 0;
    if (t.valid) {
        if (scatter_variant_fits(t.scat_var, rw))
            s.scat_var = t.scat_var;
        if (t.cap_b > WARP_BIN && t.cap_b <= s.cap_b)
            s.cap_b = t.cap_b;
        else if (rw == 2 && !batched && t.cap_b == block_cap_of(5)) {
            // the on-chip class of twice the size (one CTA of 1024 threads per
            // SM); batched sorts keep theirs: the persistent kernel's on-chip
            // items hold at most 4,096 records
            s.block_var = 5;
            s.cap_b = t.cap_b;
        }
        if (s.bucket_var >= 0)
            s.bucket_max = t.bucket_max;
        if (t.wmax >= 8 && t.wmax <= WIDE_MAX)
            s.wmax = t.wmax;
        s.leaf = t.leaf;
    }
    if (const char *v = getenv("RADULS_WMAX")) {
        const u32 want = (u32)strtoul(v, nullptr, 10);
        if (want >= 8 && want <= WIDE_MAX)
            s.wmax = want;
    }
    if (const char *v = getenv("RADULS_LEAF"))
        s.leaf = (u32)strtoul(v, nullptr, 10);
    if (const char *v = getenv("RADULS_BLOCK_CAP")) {
        const u32 want = (u32)strtoul(v, nullptr, 10);
        if (rw == 2 && !batched && want == block_cap_of(5)) {
            s.block_var = 5;
            s.cap_b = want;
        } else if (want > WARP_BIN && want <= block_cap_of(s.block_var)) {
            s.cap_b = want;
        }
    }
    // plain sorts of 16-byte records: each level takes the two-CTA shape made
    // for its widest digit (variant 5: 8 bits, 9: 9 bits, 11 (or 10): 10 bits)
    s.scat_by_width = !batched && ((rw == 2 && (s.scat_var == 9 || s.scat_var == 10 || s.scat_var == 11)) ||
                                   (rw == 1 && (s.scat_var == 12 || s.scat_var == 13)) ||
                                   (rw == 4 && (s.scat_var == 14 || s.scat_var == 15)));
    s.scat_var8 = rw == 1 ? 6 : rw == 4 ? 7 : 5;
    s.scat_var9 = rw == 1 ? 12 : rw == 4 ? 14 : 9;
    s.scat_var10 = rw == 1 ? 13 : rw == 4 ? 15 : (s.scat_var == 10 ? 10 : 11);
    // the shapes of 8-, 9- and 10-bit levels (when they follow the width)
    const char *names[3] = {"RADULS_SCATTER8", "RADULS_SCATTER9", "RADULS_SCATTER10"};
    int *slots[3] = {&s.scat_var8, &s.scat_var9, &s.scat_var10};
    for (int i = 0; i < 3; ++i)
        if (const char *v = getenv(names[i])) {
            const int want = atoi(v);
            if (scatter_variant_fits(want, rw) && wscatter_kmax_of(want) >= (256u << i))
                *slots[i] = want;
        }
    if (const char *v = getenv("RADULS_SCATTER_VARIANT")) {
        const int want = atoi(v);
        if (scatter_variant_fits(want, rw)) {
            s.scat_var = want;
            s.scat_by_width = false;  // one shape for every level
        }
    }
    if (const char *v = getenv("RADULS_BUCKET_MAX"))
        s.bucket_max = s.bucket_var < 0 ? 0u : (u32)strtoul(v, nullptr, 10);
    // the streamed on-chip finisher (plain sorts): its capacity becomes the
    // on-chip class, and the general on-chip kernel (of at least that
    // capacity) takes what it leaves
    s.bins_var = -1;
    {
        int want = (t.valid && t.bins) ? t.bins : 1;  // on unless tuned off
        if (const char *v = getenv("RADULS_BIN_SORT"))
            want = atoi(v) ? 1 : 2;
        int bv = batched ? -1 : binsort_variant_for(rw);
        if (const char *v = getenv("RADULS_BIN_VARIANT"))
            if (bv >= 0 && binsort_rw_of(atoi(v)) == rw)
                bv = atoi(v);
        if (want == 1 && bv >= 0) {
            s.bins_var = bv;
            if (rw == 2)
                s.block_var = 5;  // the general kernel that takes what it leaves holds as many records
            const u32 bcap = binsort_cap_of(bv);
            s.cap_b = (t.valid && t.cap_b > WARP_BIN && t.cap_b < bcap) ? t.cap_b : bcap;
            if (s.leaf == 0)
                s.leaf = s.cap_b / 10u * 9u;  // sub-bins of about 9/10 of the capacity: the largest still fit
        }
    }
    s.tile_s = wscatter_tile_of(s.scat_var);
    while (s.wmax > 8u && (1u << s.wmax) > wscatter_kmax_of(s.scat_var))
        --s.wmax;  // the variant handles no wider digit
    if (s.bucket_max > BUCKET_IDX_MAX)  // positions inside a mid-size bin are 16-bit
        s.bucket_max = BUCKET_IDX_MAX;
    if (s.bucket_max <= s.cap_b)
        s.bucket_max = 0;
    // the sub-bin size the digit widths aim at: at most the largest bin a
    // finisher takes (the mid-size class where there is one)
    if (s.leaf == 0 || s.leaf > (s.bucket_max > s.cap_b ? s.bucket_max : s.cap_b))
        s.leaf = s.cap_b / 4u * 3u;  // sub-bins of about 3/4 of the on-chip class: the largest still fit
    return s;
}

int level_scatter_variant(const Shape &s, u32 w)
{
    if (!s.scat_by_width)
        return s.scat_var;
    return w <= 8u ? s.scat_var8 : w == 9u ? s.scat_var9 : s.scat_var10;
}

namespace {

constexpr int MAX_DEVICES = 64;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// One set of pass buffers with its own device counters: the main sort uses
// one, the nested sort of the learned model's key sample the other.
struct Work {
    Counters *ctrs = nullptr;    // device
    Counters *h_ctrs = nullptr;  // pinned host mirror
    u32 *epoch = nullptr;        // device: look-back epoch of the last distribution launch, wrap flag
    DevBuf lists, hist, status, tiles;
    DevBuf bscratch;  // private scratch regions of the mid-size bin kernel's CTAs
    DevBuf bqueue;    // batched persistent kernel: mid-size array list, pushed items, ready flags
    DevBuf win;       // end-to-end sort: mid-size bins grouped by position window
};

// Device buffers of one learned model (see the Model struct in common.cuh).
struct ModelBufs {
    DevBuf buf;
    Model *model = nullptr;
    float *h = nullptr, *theta = nullptr, *am = nullptr, *av = nullptr, *tot = nullptr;
    double *E = nullptr, *G = nullptr, *Z = nullptr, *loss = nullptr;
    u64 *sample = nullptr, *sample_tmp = nullptr, *root = nullptr;
    u64 *bmin = nullptr, *bmax = nullptr;  // the learned pass's key range per bucket
    u64 *heavy = nullptr;                  // heavy keys of the sample (at most HEAVY_MAX)
    u32 *load = nullptr;                   // bucket loads of the sample (balance check)
    u32 *seg_start = nullptr;
    u32 S = 0, k_extra = 0, max_knots = 0, n_params_cap = 0, steps_done = 0;
    u32 log2b = 0;
};

constexpr int COPY_STREAMS_MAX = 8;

struct Ctx {
    std::mutex mu;
    bool inited = false;
    u32 *dev_status = nullptr;   // device: sticky status word of this device
    Work main, aux;
    ModelBufs mdl;
    DevBuf host_in, host_tmp;    // raduls_sort_host: the device copy of the records and its scratch
    DevBuf pair_a, pair_b;       // raduls_sort_indexed: (key, index) pairs and their scratch
    DevBuf rle;                  // raduls_unique_counts: per-tile run counts
    u32 *withhold = nullptr;      // device word read by the batched kernel (dev_status + 16)
    cudaStream_t copy_st[COPY_STREAMS_MAX] = {};
    cudaEvent_t copy_ev[COPY_STREAMS_MAX + 1] = {};
    cudaEvent_t win_ev[BUCKET_WINDOWS_MAX] = {};
    bool have_copy = false;
    u64 wait_ns = 2000000000ull;
    u32 inject_tile = ~0u;
    u32 withhold_dev = ~0u;       // the value last written to the device's withheld-slot word
    cudaEvent_t ev[1024] = {};
    bool have_events = false;
};

Ctx g_ctx[MAX_DEVICES];

std::mutex g_setting_mu;
u64 g_wait_ns = 2000000000ull;
u32 g_inject_tile = ~0u;
u32 g_withhold_push = ~0u;  // pushed queue slot of the batched kernel whose ready flag is withheld

cudaError_t ensure(DevBuf &b, size_t bytes, bool zero, bool *grew = nullptr, cudaStream_t st = 0)
{
    if (grew)
        *grew = false;
    if (b.bytes >= bytes && b.p)
        return cudaSuccess;
    if (b.p) {
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    size_t want = bytes + bytes / 4 + 4096;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return e;
    }
    b.bytes = want;
    if (zero) {
        e = cudaMemsetAsync(b.p, 0, want, st);
        if (e != cudaSuccess)
            return e;
    }
    if (grew)
        *grew = true;
    return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Lists {
    WorkItem *grid[2];
    WorkItem *scat;
    WorkItem *bkt[2];
    WorkItem *bkt_split;
    WorkItem *blocks;
    WorkItem *blocks_fb;  // on-chip items the streamed bin sort leaves to the general kernel
    WorkItem *copies;
    u32 *tile_hist;
    u32 *tile_copy;
    u64 *cell[2];  // first look-back status word of every grid item (current / next list)
    Caps caps;
};

__global__ void fold_status_kernel(const Counters *c, u32 *dev_status)
{
    if (c->err)
        atomicCAS(dev_status, 0u, c->err);
}

int to_status(cudaError_t e)
{
    if (e == cudaSuccess)
        return RADULS_OK;
    if (e == cudaErrorMemoryAllocation)
        return RADULS_ERR_OOM;
    return RADULS_ERR_CUDA;
}

int check_args(const void *in, const void *tmp, u64 n, u32 rec_bytes, u32 key_bytes)
{
    if (rec_bytes % 8u || key_bytes % 8u || key_bytes < 8u || key_bytes > rec_bytes)
        return RADULS_ERR_INVALID_ARG;
    if (rec_bytes > 256u)
        return RADULS_ERR_UNSUPPORTED;
    if (n > 1 && (!in || !tmp))
        return RADULS_ERR_INVALID_ARG;
    if (n > (~0ull) / rec_bytes)
        return RADULS_ERR_INVALID_ARG;
    if (n > (1ull << 39))
        return RADULS_ERR_UNSUPPORTED;
    if (((uintptr_t)in & 15u) || ((uintptr_t)tmp & 15u))
        return RADULS_ERR_MISALIGNED;
    if (n > 1) {
        const uintptr_t a = (uintptr_t)in, b = (uintptr_t)tmp, len = (uintptr_t)(n * rec_bytes);
        if (a < b + len && b < a + len)
            return RADULS_ERR_MISALIGNED;
    }
    return RADULS_OK;
}

cudaError_t work_init(Work &w)
{
    cudaError_t e = cudaMalloc(&w.ctrs, sizeof(Counters));
    if (e != cudaSuccess)
        return e;
    e = cudaMalloc(&w.epoch, 16);
    if (e != cudaSuccess)
        return e;
    e = cudaMemset(w.epoch, 0, 16);
    if (e != cudaSuccess)
        return e;
    e = cudaMemset(w.ctrs, 0, sizeof(Counters));
    if (e != cudaSuccess)
        return e;
    return cudaMallocHost(&w.h_ctrs, sizeof(Counters));
}

cudaError_t ctx_init(Ctx &c)
{
    if (c.inited)
        return cudaSuccess;
    cudaError_t e = work_init(c.main);
    if (e != cudaSuccess)
        return e;
    e = work_init(c.aux);
    if (e != cudaSuccess)
        return e;
    e = cudaMalloc(&c.dev_status, 256);
    if (e != cudaSuccess)
        return e;
    e = cudaMemset(c.dev_status, 0, 256);
    if (e != cudaSuccess)
        return e;
    c.withhold = c.dev_status + 16;
    e = cudaMemset(c.withhold, 0xff, 4);
    if (e != cudaSuccess)
        return e;
    c.withhold_dev = ~0u;
    c.inited = true;
    return cudaSuccess;
}

// Sizes every list for a problem of n records (upper bounds).
cudaError_t work_lists(Work &wk, const Shape &s, u64 n, Lists &L)
{
    const u64 W = s.key_words;
    const u64 grid_cap = n / ((u64)s.cap_b + 1) + 2;                 // grid bins hold > cap_b records each
    const u64 hist_tiles = n / s.tile_h + grid_cap + 2;
    const u64 copy_cap = 8 * W * grid_cap + 2;                        // one per finished big bin
    const u64 copy_tiles = n / s.tile_c + copy_cap + 2;
    // full runs + runs cut by big bins / parents + the model's sub-bins (<= 2^16)
    u64 block_cap = 2 * n / s.cap_b + 2 * 8 * W * grid_cap + 4 + 65536 + 256;
    if (block_cap > n + 4)
        block_cap = n + 4;
    if (grid_cap > 0xffffffffull || hist_tiles > 0xffffffffull || copy_tiles > 0xffffffffull)
        return cudaErrorInvalidValue;
    size_t off = 0, o_grid0, o_grid1, o_scat, o_bkt0, o_bkt1, o_bkts, o_blocks, o_fb, o_copies, o_th, o_tc, o_c0,
           o_c1;
    o_grid0 = off; off = align256(off + grid_cap * sizeof(WorkItem));
    o_grid1 = off; off = align256(off + grid_cap * sizeof(WorkItem));
    o_scat = off; off = align256(off + grid_cap * sizeof(WorkItem));
    o_bkt0 = off; off = align256(off + grid_cap * sizeof(WorkItem));
    o_bkt1 = off; off = align256(off + grid_cap * sizeof(WorkItem));
    o_bkts = off; off = align256(off + grid_cap * sizeof(WorkItem));
    o_blocks = off; off = align256(off + block_cap * sizeof(WorkItem));
    o_fb = off; off = align256(off + (s.bins_var >= 0 ? block_cap : 1) * sizeof(WorkItem));
    o_copies = off; off = align256(off + copy_cap * sizeof(WorkItem));
    o_th = off; off = align256(off + hist_tiles * 4);
    o_tc = off; off = align256(off + copy_tiles * 4);
    o_c0 = off; off = align256(off + grid_cap * 8);
    o_c1 = off; off = align256(off + grid_cap * 8);
    cudaError_t e = ensure(wk.lists, off, false);
    if (e != cudaSuccess)
        return e;
    char *b = (char *)wk.lists.p;
    L.grid[0] = (WorkItem *)(b + o_grid0);
    L.grid[1] = (WorkItem *)(b + o_grid1);
    L.scat = (WorkItem *)(b + o_scat);
    L.bkt[0] = (WorkItem *)(b + o_bkt0);
    L.bkt[1] = (WorkItem *)(b + o_bkt1);
    L.bkt_split = (WorkItem *)(b + o_bkts);
    L.blocks = (WorkItem *)(b + o_blocks);
    L.blocks_fb = (WorkItem *)(b + o_fb);
    L.copies = (WorkItem *)(b + o_copies);
    L.tile_hist = (u32 *)(b + o_th);
    L.tile_copy = (u32 *)(b + o_tc);
    L.cell[0] = (u64 *)(b + o_c0);
    L.cell[1] = (u64 *)(b + o_c1);
    L.caps.grid = (u32)grid_cap;
    L.caps.hist_tiles = (u32)hist_tiles;
    L.caps.copy = (u32)copy_cap;
    L.caps.copy_tiles = (u32)copy_tiles;
    L.caps.block = block_cap;
    L.caps.scat_tiles = 0;
    // look-back status words of one level: a grid item of c records has
    // ceil(c / tile_h) chunks of 2^w words, 2^w <= max(256, c / 16)
    const double per_rec = 256.0 / (double)(s.cap_b + 1u) > 1.0 / 16.0 ? 256.0 / (double)(s.cap_b + 1u) : 1.0 / 16.0;
    L.caps.cells = (u64)(2.0 * per_rec * (double)n) + 16ull * KMAX;
    return cudaSuccess;
}

struct LevelBufs {
    u64 *hist, *orand, *status;
    u32 *tile_scat;
};

// Per-level buffers: histogram rows (and OR/AND words) of the current big bins
// and the look-back status words of this level's distribution tiles.
cudaError_t work_level(Work &wk, const Shape &s, u64 n, u32 n_grid, LevelBufs &B, Caps &caps, cudaStream_t st)
{
    const u64 rows = (u64)n_grid + 1;
    const size_t hb = align256(rows * RADIX * 8), ob = align256(rows * 16);
    cudaError_t e = ensure(wk.hist, hb + ob, false);
    if (e != cudaSuccess)
        return e;
    B.hist = (u64 *)wk.hist.p;
    B.orand = (u64 *)((char *)wk.hist.p + hb);
    bool grew = false;
    e = ensure(wk.status, caps.cells * 8, true, &grew, st);
    if (e != cudaSuccess)
        return e;
    if (grew) {  // fresh zeroed words: restart the epochs
        e = cudaMemsetAsync(wk.epoch, 0, 16, st);
        if (e != cudaSuccess)
            return e;
    }
    e = ensure(wk.tiles, (size_t)caps.hist_tiles * 4, false);
    if (e != cudaSuccess)
        return e;
    B.status = (u64 *)wk.status.p;
    B.tile_scat = (u32 *)wk.tiles.p;
    caps.scat_tiles = caps.hist_tiles;
    return cudaSuccess;
}

// Times each launch with a pair of CUDA events on the launching stream when
// statistics are requested, and counts launches always.
struct Recorder {
    Ctx *c = nullptr;
    cudaStream_t st = 0;
    bool timing = false;
    int used = 0;
    int cls[512];
    u32 launches[RADULS_K_COUNT] = {};
    u32 total = 0;

    cudaError_t begin(int k)
    {
        launches[k] += 1;
        total += 1;
        if (!timing || used >= 512)
            return cudaSuccess;
        cls[used] = k;
        return cudaEventRecord(c->ev[2 * used], st);
    }
    cudaError_t end()
    {
        if (!timing || used >= 512)
            return cudaSuccess;
        cudaError_t e = cudaEventRecord(c->ev[2 * used + 1], st);
        used += 1;
        return e;
    }
};

struct SortJob {
    u64 *in;
    u64 *tmp;
    u64 n;
    u32 rw, kw;
    int single_pass;       // distribute once on `digit` and stop
    u32 digit;
    u64 *hist_out;         // histogram-only mode when non-null
    raduls_stats *stats;
    u32 mode;              // 0 auto, 1 plain, 2 learned
    u32 log2b;             // learned buckets (0 = chosen from n)
    float fallback_ratio;  // learned partition rejected above this
    u32 train_steps;
    struct HostOut *hout;  // end-to-end sort: where the sorted records go on the host
};

// Destination of an end-to-end sort (raduls_sort_host).  The last mid-size
// level runs window by window; after each window the records before the next
// window's first position are final and go back to the host on the copy
// stream while the next window is sorted.  `copied` stays set only if nothing
// writes the records afterwards (no on-chip or copy-back items, no later level).
struct HostOut {
    unsigned char *dst;
    const unsigned char *src;   // the device copy being sorted
    u32 rec_bytes;
    cudaStream_t cst;
    cudaEvent_t *ev;            // BUCKET_WINDOWS_MAX events
    bool copied;

    cudaError_t copy(u64 lo, u64 hi, u32 w, cudaStream_t st)
    {
        cudaError_t e = cudaEventRecord(ev[w], st);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(cst, ev[w], 0);
        if (e == cudaSuccess && hi > lo)
            e = cudaMemcpyAsync(dst + lo * rec_bytes, src + lo * rec_bytes, (size_t)(hi - lo) * rec_bytes,
                                cudaMemcpyDeviceToHost, cst);
        return e;
    }
};

#define CK(x)                               \
    do {                                    \
        cudaError_t _e = (x);               \
        if (_e != cudaSuccess)              \
            return to_status(_e);           \
    } while (0)

#define TIMED(k, call)           \
    do {                         \
        CK(rec.begin(k));        \
        CK(call);                \
        CK(rec.end());           \
    } while (0)

cudaError_t ctx_events(Ctx &c)
{
    if (c.have_events)
        return cudaSuccess;
    for (int i = 0; i < 1024; ++i) {
        cudaError_t e = cudaEventCreate(&c.ev[i]);
        if (e != cudaSuccess)
            return e;
    }
    c.have_events = true;
    return cudaSuccess;
}

int run_sort(Ctx &c, Work &wk, const SortJob &j, cudaStream_t st, Recorder *outer = nullptr);

// ------------------------------------------------------------ learned model

constexpr u32 SAMPLE_MAX = 1u << 20;
constexpr u32 K_EXTRA_MAX = 1u << 14;

// Device buffers of a model for sample size S and knot budget k_extra.
cudaError_t model_bufs(ModelBufs &M, u32 S, u32 k_extra)
{
    const u32 knots = 2u * (2u * RADIX + k_extra) + 8u;  // both stages
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t o_model = take(sizeof(Model)), o_h = take(knots * 4), o_th = take(knots * 4),
                 o_am = take(knots * 4), o_av = take(knots * 4), o_tot = take(2 * RADIX * 4), o_E = take(knots * 8),
                 o_G = take(knots * 8), o_Z = take(RADIX * 8), o_loss = take(8), o_s = take((size_t)S * 8),
                 o_st = take((size_t)S * 8), o_root = take(RADIX * 8), o_seg = take((RADIX + 1) * 4),
                 o_bmin = take(KMAX * 8), o_bmax = take(KMAX * 8), o_heavy = take(HEAVY_MAX * 8),
                 o_load = take(KMAX * 4);
    cudaError_t e = ensure(M.buf, off, true);
    if (e != cudaSuccess)
        return e;
    char *b = (char *)M.buf.p;
    M.model = (Model *)(b + o_model);
    M.h = (float *)(b + o_h);
    M.theta = (float *)(b + o_th);
    M.am = (float *)(b + o_am);
    M.av = (float *)(b + o_av);
    M.tot = (float *)(b + o_tot);
    M.E = (double *)(b + o_E);
    M.G = (double *)(b + o_G);
    M.Z = (double *)(b + o_Z);
    M.loss = (double *)(b + o_loss);
    M.sample = (u64 *)(b + o_s);
    M.sample_tmp = (u64 *)(b + o_st);
    M.root = (u64 *)(b + o_root);
    M.seg_start = (u32 *)(b + o_seg);
    M.bmin = (u64 *)(b + o_bmin);
    M.bmax = (u64 *)(b + o_bmax);
    M.heavy = (u64 *)(b + o_heavy);
    M.load = (u32 *)(b + o_load);
    M.S = S;
    M.k_extra = k_extra;
    M.max_knots = 2u + k_extra;
    M.n_params_cap = knots;
    return cudaSuccess;
}



// Adam step size: the warm start already passes through the sample's CDF at
// every knot, so the steps only refine it (larger steps overshoot).
constexpr float LEARN_RATE = 0.002f;

// Fit a model of the key words 0 of `in` (n records of rw words) whose exact
// top-byte histogram is root_hist (device, 256 u64): sample, sort the sample
// with the aux work set, build the leaves, run `steps` Adam steps.
int model_fit(Ctx &c, ModelBufs &M, const u64 *in, u64 n, u32 rw, const u64 *root_hist, u32 log2b, u32 steps,
              cudaStream_t st, Recorder &rec, bool warm_only = false)
{
    u32 S = n < (u64)SAMPLE_MAX ? (u32)n : SAMPLE_MAX;
    if (S < 2)
        S = 2;
    u32 k_extra = S / 8u;
    if (k_extra > K_EXTRA_MAX)
        k_extra = K_EXTRA_MAX;
    CK(model_bufs(M, S, k_extra));
    M.log2b = log2b;
    CK(cudaMemcpyAsync(M.root, root_hist, RADIX * 8, cudaMemcpyDeviceToDevice, st));
    TIMED(RADULS_K_LEARNED, lm_launch_sample(in, n, rw, S, M.sample, st));
    SortJob sj{};
    sj.in = M.sample;
    sj.tmp = M.sample_tmp;
    sj.n = S;
    sj.rw = 1;
    sj.kw = 1;
    sj.mode = 1;
    int rc = run_sort(c, c.aux, sj, st, &rec);
    if (rc)
        return rc;
    TIMED(RADULS_K_LEARNED, lm_launch_build(M.sample, S, k_extra, M.root, n, log2b, M.h, M.model, M.seg_start,
                                            M.max_knots, M.bmin, M.bmax, st));
    {
        // a key filling an ideal bucket's share of the sample cannot be split by
        // any bucket map: it is left out of the balance check
        const u32 thr = S >> log2b;
        TIMED(RADULS_K_LEARNED, lm_launch_heavy(M.sample, S, thr > 1 ? thr : 2u, M.heavy, M.model, st));
    }
    TIMED(RADULS_K_LEARNED, lm_launch_init(M.theta, M.am, M.av, M.n_params_cap, st));
    // stage 1 on its own, then stage 2 on stage 1's output: each warm-started
    // from the sample's CDF at its knots, then `steps` Adam steps (steps = 0
    // keeps both stages linear: the untrained model)
    for (u32 stage = 0; stage < 2 && steps > 0; ++stage) {
        if (stage == 1)
            TIMED(RADULS_K_LEARNED, lm_launch_heights(M.model, M.theta, M.h, M.tot, M.E, M.G, M.Z, M.loss, st));
        TIMED(RADULS_K_LEARNED, lm_launch_warm(M.model, stage, M.sample, M.seg_start, M.theta, st));
        if (warm_only)
            continue;
        for (u32 k = 1; k <= steps; ++k)
            TIMED(RADULS_K_LEARNED, lm_launch_step(M.model, stage, M.theta, M.am, M.av, M.h, M.tot, M.E, M.G, M.Z,
                                                   M.loss, M.sample, M.seg_start, S, LEARN_RATE, (int)k, nullptr,
                                                   st));
    }
    M.steps_done = steps;
    TIMED(RADULS_K_LEARNED, lm_launch_heights(M.model, M.theta, M.h, M.tot, M.E, M.G, M.Z, M.loss, st));
    return RADULS_OK;
}

// Buckets of the learned pass: 256 (measured on the skewed and wide-key
// workloads: 120 ms against 132 ms with 1,024 at 2^30 x 16 B, since the pass
// then runs with the two-CTA distribution shape).
u32 default_log2b() { return 8u; }

// ---------------------------------------------------------------- the sort

int run_sort(Ctx &c, Work &wk, const SortJob &j, cudaStream_t st, Recorder *outer)
{
    const Shape s = choose_shape(j.rw, j.kw);
    Lists L{};
    CK(work_lists(wk, s, j.n, L));
    Recorder own;
    Recorder &rec = outer ? *outer : own;
    if (!outer) {
        rec.c = &c;
        rec.st = st;
        if (j.stats) {
            CK(ctx_events(c));
            rec.timing = true;
        }
    }
    const u32 top = 8u * j.kw - 1u;
    const bool step_api = j.single_pass || j.hist_out;
    const bool may_learn = !step_api && j.mode != 1 && j.n > s.cap_b;
    const u32 bmax = step_api ? 0u : s.bucket_max;
    if (bmax)
        CK(ensure(wk.bscratch, (size_t)bucket_grid() * bmax * bucket_slot_bytes(j.rw), false));
    // the learned first partition's root is the top byte's histogram: its first
    // pass splits exactly that byte
    const u32 init_wmax = (step_api || (may_learn && j.mode == 2)) ? 0u : s.wmax;
    TIMED(RADULS_K_SETUP, launch_init(wk.ctrs, L.grid[0], L.blocks, L.tile_hist, j.n, step_api ? j.digit : top,
                                      s.cap_b, s.tile_h, step_api ? 1u : 0u, L.bkt[0], bmax, L.cell[0], s.leaf,
                                      init_wmax, st));
    {
        std::lock_guard<std::mutex> g(g_setting_mu);
        c.wait_ns = g_wait_ns;
        c.inject_tile = g_inject_tile;
        g_inject_tile = ~0u;
    }
    bool learned = false;
    u32 log2b = 0;
    float ratio_limit = j.fallback_ratio > 0.f ? j.fallback_ratio : 4.f;
    int cur = 0;
    const bool whole_mid = !step_api && j.n > s.cap_b && j.n <= bmax;
    u32 n_grid = (step_api || (j.n > s.cap_b && !whole_mid)) ? 1u : 0u;
    u32 n_bkt = whole_mid ? 1u : 0u;
    // the widest digit of the current level (the first: init_kernel's choice)
    u32 lvl_w = (init_wmax > 0 && !step_api) ? pick_width(j.n, 8u * top + 8u, s.leaf, init_wmax) : 8u;
    for (u32 level = 0; n_grid > 0 || n_bkt > 0; ++level) {
        PlanArgs a{};
        a.grid_cur = L.grid[cur];
        a.grid_next = L.grid[cur ^ 1];
        a.scat = L.scat;
        a.blocks = L.blocks;
        a.copies = L.copies;
        a.tile_hist = L.tile_hist;
        a.tile_copy = L.tile_copy;
        a.ctrs = wk.ctrs;
        a.caps = L.caps;
        a.key_words = j.kw;
        a.rw = j.rw;
        a.cap_b = s.cap_b;
        a.warp_bin = WARP_BIN;
        a.tile_h = s.tile_h;
        a.tile_s = s.tile_s;
        a.tile_c = s.tile_c;
        a.single_pass = j.single_pass ? 1u : 0u;
        a.top_digit = top;
        a.buckets_cur = L.bkt[cur];
        a.buckets_next = L.bkt[cur ^ 1];
        a.buckets_split = L.bkt_split;
        a.bucket_max = bmax;
        a.bucket_scratch = (u64 *)wk.bscratch.p;
        a.cell_cur = L.cell[cur];
        a.cell_next = L.cell[cur ^ 1];
        a.leaf = s.leaf;
        a.wmax = s.wmax;
        a.status = (u64 *)wk.status.p;
        if (n_grid > 0) {
            LevelBufs B{};
            CK(work_level(wk, s, j.n, n_grid, B, L.caps, st));
            a.caps = L.caps;  // the level's buffers fix the distribution tile capacity
            a.status = B.status;
            const Model *model = learned ? c.mdl.model : nullptr;
            bool model_pass = false;  // this level distributes on the model's bucket
            TIMED(RADULS_K_SETUP, launch_prep(B.hist, B.orand, wk.ctrs, n_grid, j.hist_out ? 1u : 0u, st));
            if (j.hist_out) {
                // histogram only (raduls_histogram): one traversal, counts per value
                TIMED(RADULS_K_HIST, launch_hist(s, j.in, j.tmp, L.grid[cur], L.tile_hist, B.hist, B.orand, wk.ctrs,
                                                 st));
                CK(cudaMemcpyAsync(j.hist_out, B.hist, RADIX * 8, cudaMemcpyDeviceToDevice, st));
                break;
            }
            TIMED(RADULS_K_SETUP, launch_epoch_next(wk.epoch, B.status, wk.status.bytes / 8, st));
            TIMED(RADULS_K_HIST, launch_whist(s, j.in, j.tmp, L.grid[cur], L.tile_hist, L.cell[cur], B.status,
                                              B.orand, wk.ctrs, model, wk.epoch, c.wait_ns, c.inject_tile, st));
            c.inject_tile = ~0u;
            if (level == 0 && may_learn) {
                // the first pass's digit histogram is the model's root; AUTO
                // keeps the plain passes (the learned first partition is taken
                // only when asked for)
                const bool use = (j.mode == 2);
                if (use) {
                    // the root bin's histogram of its top byte: its last chunk's counts
                    const u64 nch = (j.n + s.tile_h - 1) / s.tile_h;
                    TIMED(RADULS_K_SETUP, launch_status_counts(B.status + (nch - 1) * RADIX, B.hist, RADIX, st));
                    log2b = j.log2b ? j.log2b : default_log2b();
                    const bool warm_only = (j.train_steps & 0x80000000u) != 0;
                    int rc = model_fit(c, c.mdl, j.in, j.n, j.rw, B.hist, log2b, warm_only ? 1u : j.train_steps, st,
                                       rec, warm_only);
                    if (rc)
                        return rc;
                    learned = true;
                    // the balance check on the model's sample decides before any record moves
                    TIMED(RADULS_K_LEARNED, lm_launch_ratio(c.mdl.model, c.mdl.sample, c.mdl.S, c.mdl.load, wk.ctrs,
                                                            ratio_limit, st));
                    CK(cudaMemcpyAsync(wk.h_ctrs, wk.ctrs, sizeof(Counters), cudaMemcpyDeviceToHost, st));
                    CK(cudaStreamSynchronize(st));
                    if (wk.h_ctrs->learned_ok) {
                        // restart the level on the model's bucket: one digit of log2b bits
                        TIMED(RADULS_K_SETUP, launch_init(wk.ctrs, L.grid[0], L.blocks, L.tile_hist, j.n,
                                                          DIGIT_LEARNED, s.cap_b, s.tile_h, 1u, nullptr, 0u,
                                                          L.cell[0], s.leaf, log2b, st));
                        TIMED(RADULS_K_SETUP, launch_keep_learned(wk.ctrs, wk.h_ctrs->learned_ratio, st));
                        TIMED(RADULS_K_SETUP, launch_prep(B.hist, B.orand, wk.ctrs, n_grid, 0u, st));
                        TIMED(RADULS_K_LEARNED, lm_launch_minmax_reset(c.mdl.model, st));
                        TIMED(RADULS_K_SETUP, launch_epoch_next(wk.epoch, B.status, wk.status.bytes / 8, st));
                        TIMED(RADULS_K_HIST, launch_whist(s, j.in, j.tmp, L.grid[cur], L.tile_hist, L.cell[cur],
                                                          B.status, B.orand, wk.ctrs, c.mdl.model, wk.epoch,
                                                          c.wait_ns, ~0u, st));
                        model = c.mdl.model;
                        model_pass = true;
                    }
                    // else: the plain passes go on from this level's histogram of the top byte
                }
            }
            a.hist = B.hist;
            a.orand = B.orand;
            a.tile_scat = B.tile_scat;
            a.model = model;
            TIMED(RADULS_K_PLAN, launch_plan(a, n_grid, st));
            // the level's shape for its widest digit; the learned pass needs
            // one that takes 2^log2b values
            Shape sl = s;
            sl.scat_var = level_scatter_variant(s, model_pass ? log2b : lvl_w);
            if (model_pass && ((u64)1 << log2b) > wscatter_kmax_of(sl.scat_var))
                sl.scat_var = wide_scatter_variant(j.rw);
            TIMED(RADULS_K_SCATTER, launch_wscatter(sl, j.in, j.tmp, L.scat, B.tile_scat, L.cell[cur], B.status,
                                                    wk.ctrs, model, c.wait_ns, st));
        }
        if (n_bkt > 0 && n_grid == 0 && j.hout && !wk.h_ctrs->block && !wk.h_ctrs->copy) {
            // the last mid-size level of an end-to-end sort: position windows,
            // each copied back while the next is sorted
            const u32 nw = BUCKET_WINDOWS_MAX;
            CK(ensure(wk.win, ((size_t)n_bkt + nw + 1) * 4, false));
            u32 *const order = (u32 *)wk.win.p, *const wstart = order + n_bkt;
            TIMED(RADULS_K_SETUP, launch_bucket_windows(L.bkt[cur], wk.ctrs, j.n, nw, order, wstart, st));
            a.bucket_order = order;
            a.bucket_wstart = wstart;
            for (u32 w = 0; w < nw; ++w) {
                if (w > 0)
                    TIMED(RADULS_K_SETUP, launch_bucket_window_reset(wk.ctrs, st));
                a.bucket_window = w;
                TIMED(RADULS_K_BUCKET, launch_bucket(s, j.in, j.tmp, a, st));
                // bins starting at or after position ceil((w + 1) n / nw) belong to
                // later windows, so everything before floor((w + 1) n / nw) is final
                CK(j.hout->copy(j.n * w / nw, w + 1 == nw ? j.n : j.n * (w + 1) / nw, w, st));
            }
            j.hout->copied = true;
        } else if (n_bkt > 0) {
            if (j.hout)
                j.hout->copied = false;  // a level after the windows: copy everything at the end
            TIMED(RADULS_K_BUCKET, launch_bucket(s, j.in, j.tmp, a, st));
        }
        if (n_grid > 0 && j.hout)
            j.hout->copied = false;
        TIMED(RADULS_K_SETUP, launch_advance(wk.ctrs, st));
        if (j.single_pass)
            break;
        CK(cudaMemcpyAsync(wk.h_ctrs, wk.ctrs, sizeof(Counters), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (wk.h_ctrs->err)
            break;
        n_grid = wk.h_ctrs->grid_cur;
        n_bkt = wk.h_ctrs->bucket_cur;
        lvl_w = wk.h_ctrs->wmax_cur ? wk.h_ctrs->wmax_cur : 8u;
        cur ^= 1;
    }
    if (j.hout && (wk.h_ctrs->block || wk.h_ctrs->copy || wk.h_ctrs->err))
        j.hout->copied = false;  // records still move after the last level
    if (!step_api) {
        TIMED(RADULS_K_COPY, launch_copy(s, j.in, j.tmp, L.copies, L.tile_copy, wk.ctrs, st));
        if (s.bins_var >= 0 && j.hout && !wk.h_ctrs->err && wk.h_ctrs->block > 0) {
            // the last step of an end-to-end sort: the streamed bin sort runs
            // in position windows (items grouped by their first record), and
            // each window's records go back to the host while the next
            // window is sorted; every record of window w is written by items
            // that start at or before it, so it is final once w is done
            const u32 nw = BUCKET_WINDOWS_MAX;
            const u64 nb = wk.h_ctrs->block;
            CK(ensure(wk.win, ((size_t)nb + nw + 1) * 4, false));
            u32 *const order = (u32 *)wk.win.p, *const wstart = order + nb;
            TIMED(RADULS_K_SETUP, launch_block_windows(L.blocks, wk.ctrs, j.n, nw, order, wstart, st));
            for (u32 w = 0; w < nw; ++w) {
                TIMED(RADULS_K_BLOCK, launch_bin_sort(s.bins_var, j.in, j.tmp, L.blocks, L.blocks_fb, wk.ctrs,
                                                      s.key_words, L.caps.block, c.wait_ns, st, order, wstart, w));
                TIMED(RADULS_K_BLOCK, launch_block_sort(s, j.in, j.tmp, L.blocks_fb, wk.ctrs, nullptr, st, true));
                TIMED(RADULS_K_SETUP, launch_fb_window_reset(wk.ctrs, st));
                CK(j.hout->copy(j.n * w / nw, w + 1 == nw ? j.n : j.n * (w + 1) / nw, w, st));
            }
            j.hout->copied = true;
        } else if (s.bins_var >= 0) {
            TIMED(RADULS_K_BLOCK, launch_bin_sort(s.bins_var, j.in, j.tmp, L.blocks, L.blocks_fb, wk.ctrs,
                                                  s.key_words, L.caps.block, c.wait_ns, st));
            TIMED(RADULS_K_BLOCK, launch_block_sort(s, j.in, j.tmp, L.blocks_fb, wk.ctrs, nullptr, st, true));
        } else {
            TIMED(RADULS_K_BLOCK, launch_block_sort(s, j.in, j.tmp, L.blocks, wk.ctrs, nullptr, st));
        }
    }
    CK(rec.begin(RADULS_K_SETUP));
    fold_status_kernel<<<1, 1, 0, st>>>(wk.ctrs, c.dev_status);
    CK(cudaGetLastError());
    CK(rec.end());
    if (j.stats && !outer) {
        CK(cudaMemcpyAsync(wk.h_ctrs, wk.ctrs, sizeof(Counters), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const Counters &h = *wk.h_ctrs;
        raduls_stats &o = *j.stats;
        o.grid_passes = h.grid_passes;
        o.levels = h.levels;
        o.hist_bytes_read = h.hist_bytes;
        o.scatter_bytes = h.scatter_bytes;
        o.block_bytes = h.block_bytes;
        o.block_items = h.block;
        o.skipped_digits = h.skipped;
        o.learned_used = learned ? 1u : 0u;
        o.learned_fell_back = learned ? h.learned_fell_back : 0u;
        o.learned_ratio = learned ? h.learned_ratio : 0.f;
        o.gpu_launches = rec.total;
        o.bucket_items = h.bucket_items;
        o.bucket_bytes = h.bucket_bytes;
        for (int k = 0; k < RADULS_K_COUNT; ++k) {
            o.kernel_launches[k] = rec.launches[k];
            o.kernel_ms[k] = 0.f;
        }
        for (int i = 0; i < rec.used; ++i) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, c.ev[2 * i], c.ev[2 * i + 1]));
            o.kernel_ms[rec.cls[i]] += ms;
        }
    }
    return RADULS_OK;
}

// ------------------------------------------------------------ batched sort
//
// Many independent arrays in one call.  The arrays are classified on the
// device; then a fixed sequence of MSD levels (8 per key word: each level
// splits or skips at least one digit of every big bin) runs without any host
// round trip -- every kernel reads its work counts from device memory and
// returns at once when a level has nothing left -- followed by the copy-back
// and the on-chip sorts.  The whole sequence is captured once into a CUDA
// graph per (buffers, offsets, shape) and replayed by later calls.

struct BatchGraph {
    cudaStream_t cap = nullptr;  // library stream the graph is captured on
    cudaGraphExec_t exec = nullptr;
    void *in = nullptr, *tmp = nullptr;
    const void *off = nullptr;
    u64 n = 0;
    u32 n_segs = 0, rw = 0, kw = 0;
    int scat_var = -1;
    u32 cap_b = 0, bucket_max = 0, wmax = 0, leaf = 0;  // the shape the graph was captured with
    u64 wait_ns = 0;
    void *ws[6] = {};  // workspace buffers the graph's kernels use (a regrown one forces a new capture)
};

BatchGraph g_batch[MAX_DEVICES];

int enqueue_batched(Ctx &c, Work &wk, const Shape &s, u64 *in, u64 *tmp, const u64 *off, u32 n_segs, u64 n, u32 rw,
                    u32 kw, Lists &L, LevelBufs &B, const BatchQueue &q, cudaStream_t st)
{
    const u32 top = 8u * kw - 1u;
    CK(launch_batched_init(off, n_segs, L.grid[0], L.blocks, L.tile_hist, wk.ctrs, L.caps, top, s.cap_b, s.tile_h,
                           const_cast<WorkItem *>(q.mid), s.bucket_max, L.cell[0], s.leaf, s.wmax, st));
    int cur = 0;
    const u32 levels = 8u * kw;
    for (u32 level = 0; level < levels; ++level) {
        CK(launch_prep(B.hist, B.orand, wk.ctrs, L.caps.grid, 0u, st));
        CK(launch_epoch_next(wk.epoch, B.status, wk.status.bytes / 8, st));
        CK(launch_whist(s, in, tmp, L.grid[cur], L.tile_hist, L.cell[cur], B.status, B.orand, wk.ctrs, nullptr,
                        wk.epoch, c.wait_ns, ~0u, st));
        PlanArgs a{};
        a.grid_cur = L.grid[cur];
        a.grid_next = L.grid[cur ^ 1];
        a.scat = L.scat;
        a.blocks = L.blocks;
        a.copies = L.copies;
        a.hist = B.hist;
        a.orand = B.orand;
        a.tile_hist = L.tile_hist;
        a.tile_scat = B.tile_scat;
        a.tile_copy = L.tile_copy;
        a.ctrs = wk.ctrs;
        a.caps = L.caps;
        a.key_words = kw;
        a.rw = rw;
        a.cap_b = s.cap_b;
        a.warp_bin = WARP_BIN;
        a.tile_h = s.tile_h;
        a.tile_s = s.tile_s;
        a.tile_c = s.tile_c;
        a.single_pass = 0;
        a.top_digit = top;
        a.buckets_cur = L.bkt[cur];
        a.buckets_next = L.bkt[cur ^ 1];
        a.buckets_split = L.bkt_split;
        a.bucket_max = s.bucket_max;
        a.bucket_scratch = (u64 *)wk.bscratch.p;
        a.status = B.status;
        a.cell_cur = L.cell[cur];
        a.cell_next = L.cell[cur ^ 1];
        a.leaf = s.leaf;
        a.wmax = s.wmax;
        CK(launch_plan(a, 0, st));
        CK(launch_wscatter(s, in, tmp, L.scat, B.tile_scat, L.cell[cur], B.status, wk.ctrs, nullptr, c.wait_ns, st));
        if (a.bucket_max)
            CK(launch_bucket(s, in, tmp, a, st));
        CK(launch_advance(wk.ctrs, st));
        cur ^= 1;
    }
    CK(launch_check_drained(wk.ctrs, st));
    CK(launch_copy(s, in, tmp, L.copies, L.tile_copy, wk.ctrs, st));
    if (s.bucket_var >= 0) {
        // one persistent launch: mid-size arrays, then every on-chip item
        PlanArgs a{};
        a.ctrs = wk.ctrs;
        a.caps = L.caps;
        a.key_words = kw;
        a.rw = rw;
        a.cap_b = s.cap_b;
        a.warp_bin = WARP_BIN;
        a.tile_h = s.tile_h;
        a.top_digit = top;
        a.bucket_max = s.bucket_max;
        a.bucket_scratch = (u64 *)wk.bscratch.p;
        CK(launch_batched_persistent(s, in, tmp, a, q, off, c.wait_ns, st));
    } else {
        CK(launch_block_sort(s, in, tmp, L.blocks, wk.ctrs, off, st));
    }
    fold_status_kernel<<<1, 1, 0, st>>>(wk.ctrs, c.dev_status);
    CK(cudaGetLastError());
    return RADULS_OK;
}

int run_batched(Ctx &c, int dev, u64 *in, u64 *tmp, const u64 *off, u32 n_segs, u64 n, u32 rw, u32 kw,
                cudaStream_t st)
{
    Work &wk = c.main;
    const Shape s = choose_shape(rw, kw, true);
    Lists L{};
    // the batched init adds up to n_segs on-chip items and (n / cap_b) runs to the usual bounds
    CK(work_lists(wk, s, n + 2ull * n_segs + 2ull * s.cap_b, L));
    LevelBufs B{};
    CK(work_level(wk, s, n, L.caps.grid, B, L.caps, st));
    if (s.bucket_max)
        CK(ensure(wk.bscratch, (size_t)bucket_grid() * s.bucket_max * bucket_slot_bytes(rw), false));
    // the persistent kernel's queue: mid-size arrays (<= n_segs), pushed items
    // (each a sub-bin of more than one on-chip group), ready flags
    BatchQueue q{};
    {
        const u64 cap_dyn = n / 4096 + 64;
        const size_t o_mid = 0, o_dyn = align256((size_t)(n_segs + 1) * sizeof(WorkItem)),
                     o_rdy = o_dyn + align256((size_t)cap_dyn * sizeof(WorkItem)), total = o_rdy + cap_dyn * 4;
        if (cap_dyn > 0xffffffffull)
            return RADULS_ERR_UNSUPPORTED;
        CK(ensure(wk.bqueue, total, false));
        char *b = (char *)wk.bqueue.p;
        q.mid = (const WorkItem *)(b + o_mid);
        q.blocks = L.blocks;
        q.dyn = (WorkItem *)(b + o_dyn);
        q.ready = (u32 *)(b + o_rdy);
        q.cap_dyn = (u32)cap_dyn;
        q.withhold = c.withhold;
    }
    u32 withhold = ~0u;
    {
        std::lock_guard<std::mutex> g(g_setting_mu);
        c.wait_ns = g_wait_ns;
        withhold = g_withhold_push;
        g_withhold_push = ~0u;  // one call only
    }
    if (withhold != c.withhold_dev) {
        static thread_local u32 h_word;
        h_word = withhold;
        CK(cudaMemcpyAsync(c.withhold, &h_word, 4, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        c.withhold_dev = withhold;
    }
    BatchGraph &bg = g_batch[dev];
    void *const ws[6] = {wk.lists.p, wk.hist.p, wk.status.p, wk.tiles.p, wk.bscratch.p, wk.bqueue.p};
    bool same_ws = true;
    for (int i = 0; i < 6; ++i)
        same_ws = same_ws && bg.ws[i] == ws[i];
    const bool hit = bg.exec && bg.in == in && bg.tmp == tmp && bg.off == off && bg.n == n && bg.n_segs == n_segs &&
                     bg.rw == rw && bg.kw == kw && bg.in != nullptr && same_ws && bg.scat_var == s.scat_var &&
                     bg.cap_b == s.cap_b && bg.bucket_max == s.bucket_max && bg.wmax == s.wmax && bg.leaf == s.leaf &&
                     bg.wait_ns == c.wait_ns;
    if (!hit) {
        if (bg.exec) {
            cudaGraphExecDestroy(bg.exec);
            bg.exec = nullptr;
        }
        // buffers must be sized before the capture: nothing may allocate inside it.
        // The caller's stream may be the legacy default stream, which cannot be
        // captured: capture on a stream of our own, launch on the caller's.
        CK(cudaStreamSynchronize(st));
        if (!bg.cap)
            CK(cudaStreamCreateWithFlags(&bg.cap, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(bg.cap, cudaStreamCaptureModeRelaxed));
        int rc = enqueue_batched(c, wk, s, in, tmp, off, n_segs, n, rw, kw, L, B, q, bg.cap);
        cudaError_t e = cudaStreamEndCapture(bg.cap, &graph);
        if (rc)
            return rc;
        CK(e);
        e = cudaGraphInstantiate(&bg.exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(e);
        bg.in = in;
        bg.tmp = tmp;
        bg.off = off;
        bg.n = n;
        bg.n_segs = n_segs;
        bg.rw = rw;
        bg.kw = kw;
        for (int i = 0; i < 6; ++i)
            bg.ws[i] = ws[i];
        bg.scat_var = s.scat_var;
        bg.cap_b = s.cap_b;
        bg.bucket_max = s.bucket_max;
        bg.wmax = s.wmax;
        bg.leaf = s.leaf;
        bg.wait_ns = c.wait_ns;
    }
    CK(cudaGraphLaunch(bg.exec, st));
    return RADULS_OK;
}

Ctx *current_ctx(int *status)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        *status = RADULS_ERR_CUDA;
        return nullptr;
    }
    *status = RADULS_OK;
    return &g_ctx[dev];
}

}  // namespace
}  // namespace raduls

namespace raduls {
namespace {

// Tuning input: word i of the buffer is the SplitMix64 output for counter
// seed + i (Steele, Lea, Flood 2014): uniform keys and payloads.
__global__ void tune_fill_kernel(u64 *__restrict__ out, u64 words, u64 seed)
{
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (u64)gridDim.x * blockDim.x) {
        u64 z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        out[i] = z ^ (z >> 31);
    }
}

}  // namespace
}  // namespace raduls

using namespace raduls;

// Host handle of a fitted model (device buffers of its own).
struct raduls_model {
    int device;
    ModelBufs m;
    u64 n;
};

extern "C" {

int raduls_sort_ex(void *in, void *tmp, uint64_t n_recs, uint32_t rec_bytes, uint32_t key_bytes,
                   const raduls_opts *opts, void *stream)
{
    int rc = check_args(in, tmp, n_recs, rec_bytes, key_bytes);
    if (rc)
        return rc;
    if (opts && opts->mode > 2u)
        return RADULS_ERR_INVALID_ARG;
    if (opts && opts->learned_log2_buckets && (opts->learned_log2_buckets < 8u || opts->learned_log2_buckets > WIDE_MAX))
        return RADULS_ERR_INVALID_ARG;
    if (opts && opts->train_steps > 4096u && opts->train_steps != 0x80000000u)
        return RADULS_ERR_INVALID_ARG;
    if (opts && opts->stats)
        std::memset(opts->stats, 0, sizeof(raduls_stats));
    if (n_recs <= 1)
        return RADULS_OK;
    Ctx *c = current_ctx(&rc);
    if (!c)
        return rc;
    std::lock_guard<std::mutex> g(c->mu);
    cudaError_t e = ctx_init(*c);
    if (e != cudaSuccess)
        return to_status(e);
    SortJob j{};
    j.in = (u64 *)in;
    j.tmp = (u64 *)tmp;
    j.n = n_recs;
    j.rw = rec_bytes / 8u;
    j.kw = key_bytes / 8u;
    j.stats = opts ? opts->stats : nullptr;
    j.mode = opts ? opts->mode : 0u;
    j.log2b = opts ? opts->learned_log2_buckets : 0u;
    j.fallback_ratio = opts ? opts->fallback_ratio : 0.f;
    j.train_steps = (opts && opts->train_steps) ? opts->train_steps : 16u;
    return run_sort(*c, c->main, j, (cudaStream_t)stream);
}

int raduls_sort(void *in, void *tmp, uint64_t n_recs, uint32_t rec_bytes, uint32_t key_bytes, void *stream)
{
    return raduls_sort_ex(in, tmp, n_recs, rec_bytes, key_bytes, nullptr, stream);
}

int raduls_sort_indexed(void *in, void *tmp, uint64_t n_recs, uint32_t rec_bytes, uint32_t key_bytes, void *stream)
{
    int rc = check_args(in, tmp, n_recs, rec_bytes, key_bytes);
    if (rc)
        return rc;
    if (n_recs <= 1)
        return RADULS_OK;
    Ctx *c = current_ctx(&rc);
    if (!c)
        return rc;
    std::lock_guard<std::mutex> g(c->mu);
    cudaError_t e = ctx_init(*c);
    if (e != cudaSuccess)
        return to_status(e);
    cudaStream_t st = (cudaStream_t)stream;
    const u32 rw = rec_bytes / 8u, kw = key_bytes / 8u, pw = kw + 1u;
    if (n_recs > (~0ull) / (pw * 8u))
        return RADULS_ERR_INVALID_ARG;
    const size_t pb = (size_t)n_recs * pw * 8u;
    CK(ensure(c->pair_a, pb, false));
    CK(ensure(c->pair_b, pb, false));
    u64 *pa = (u64 *)c->pair_a.p, *pbuf = (u64 *)c->pair_b.p;
    CK(launch_build_pairs((const u64 *)in, n_recs, rw, kw, pa, st));
    SortJob j{};
    j.in = pa;
    j.tmp = pbuf;
    j.n = n_recs;
    j.rw = pw;
    j.kw = kw;
    j.mode = 1;
    rc = run_sort(*c, c->main, j, st);
    if (rc)
        return rc;
    CK(launch_gather((const u64 *)in, n_recs, rw, pa, pw, (u64 *)tmp, st));
    CK(cudaMemcpyAsync(in, tmp, (size_t)n_recs * rec_bytes, cudaMemcpyDeviceToDevice, st));
    return RADULS_OK;
}

int raduls_unique_counts(const void *in, uint64_t n_recs, uint32_t rec_bytes, uint32_t key_bytes, void *d_keys_out,
                         uint64_t *d_counts_out, uint64_t *d_n_unique, void *stream)
{
    if (rec_bytes % 8u || key_bytes % 8u || key_bytes < 8u || key_bytes > rec_bytes)
        return RADULS_ERR_INVALID_ARG;
    if (rec_bytes > 256u)
        return RADULS_ERR_UNSUPPORTED;
    if (!d_n_unique || (n_recs > 0 && (!in || !d_keys_out || !d_counts_out)))
        return RADULS_ERR_INVALID_ARG;
    if (((uintptr_t)in & 7u) || ((uintptr_t)d_keys_out & 7u) || ((uintptr_t)d_counts_out & 7u) ||
        ((uintptr_t)d_n_unique & 7u))
        return RADULS_ERR_MISALIGNED;
    if (n_recs > (1ull << 39))
        return RADULS_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    if (n_recs == 0)
        return to_status(cudaMemsetAsync(d_n_unique, 0, 8, st));
    int rc = 0;
    Ctx *c = current_ctx(&rc);
    if (!c)
        return rc;
    std::lock_guard<std::mutex> g(c->mu);
    cudaError_t e = ctx_init(*c);
    if (e != cudaSuccess)
        return to_status(e);
    CK(ensure(c->rle, rle_tiles(n_recs) * 8, false));
    CK(launch_rle((const u64 *)in, n_recs, rec_bytes / 8u, key_bytes / 8u, (u64 *)c->rle.p, (u64 *)d_keys_out,
                  (u64 *)d_counts_out, (u64 *)d_n_unique, st));
    return RADULS_OK;
}

int raduls_sort_host(const void *h_in, void *h_out, uint64_t n_recs, uint32_t rec_bytes, uint32_t key_bytes,
                     const raduls_opts *opts, void *stream)
{
    int rc = check_args(nullptr, nullptr, 0, rec_bytes, key_bytes);
    if (rc)
        return rc;
    if (n_recs > 0 && (!h_in || !h_out))
        return RADULS_ERR_INVALID_ARG;
    if (n_recs > (1ull << 39) || n_recs > (~0ull) / rec_bytes)
        return RADULS_ERR_UNSUPPORTED;
    if (opts && (opts->mode > 2u ||
                 (opts->learned_log2_buckets && (opts->learned_log2_buckets < 8u || opts->learned_log2_buckets > WIDE_MAX)) ||
                 (opts->train_steps > 4096u && opts->train_steps != 0x80000000u)))
        return RADULS_ERR_INVALID_ARG;
    const size_t bytes = (size_t)n_recs * rec_bytes;
    if (h_in != h_out && n_recs > 0) {
        const uintptr_t a = (uintptr_t)h_in, b = (uintptr_t)h_out;
        if (a < b + bytes && b < a + bytes)
            return RADULS_ERR_INVALID_ARG;
    }
    if (opts && opts->stats)
        std::memset(opts->stats, 0, sizeof(raduls_stats));
    if (n_recs == 0)
        return RADULS_OK;
    Ctx *c = current_ctx(&rc);
    if (!c)
        return rc;
    std::lock_guard<std::mutex> g(c->mu);
    cudaError_t e = ctx_init(*c);
    if (e != cudaSuccess)
        return to_status(e);
    int ns = 1;  // one copy stream reaches the host link's rate; more were slower
    if (const char *v = getenv("RADULS_COPY_STREAMS"))
        ns = atoi(v);
    ns = ns < 1 ? 1 : ns > COPY_STREAMS_MAX ? COPY_STREAMS_MAX : ns;
    if (!c->have_copy) {
        for (int i = 0; i < COPY_STREAMS_MAX; ++i)
            CK(cudaStreamCreateWithFlags(&c->copy_st[i], cudaStreamNonBlocking));
        for (int i = 0; i <= COPY_STREAMS_MAX; ++i)
            CK(cudaEventCreateWithFlags(&c->copy_ev[i], cudaEventDisableTiming));
        for (u32 i = 0; i < BUCKET_WINDOWS_MAX; ++i)
            CK(cudaEventCreateWithFlags(&c->win_ev[i], cudaEventDisableTiming));
        c->have_copy = true;
    }
    e = ensure(c->host_in, bytes, false);
    if (e == cudaSuccess)
        e = ensure(c->host_tmp, bytes, false);
    if (e != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? RADULS_ERR_OOM : to_status(e);
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *d = (unsigned char *)c->host_in.p;
    // chunks of at least 64 MiB, dealt round-robin to the copy streams; each
    // copy stream starts after the work already on `stream`, and `stream`
    // continues after every copy stream
    const size_t chunk = std::max<size_t>((size_t)64 << 20, (bytes + 4 * ns - 1) / (4 * ns));
    auto spread = [&](bool to_dev) -> cudaError_t {
        cudaError_t x = cudaEventRecord(c->copy_ev[COPY_STREAMS_MAX], st);
        for (int i = 0; i < ns && x == cudaSuccess; ++i)
            x = cudaStreamWaitEvent(c->copy_st[i], c->copy_ev[COPY_STREAMS_MAX], 0);
        int k = 0;
        for (size_t off = 0; off < bytes && x == cudaSuccess; off += chunk, k = (k + 1) % ns) {
            const size_t len = std::min(chunk, bytes - off);
            x = to_dev ? cudaMemcpyAsync(d + off, (const unsigned char *)h_in + off, len, cudaMemcpyHostToDevice,
                                         c->copy_st[k])
                       : cudaMemcpyAsync((unsigned char *)h_out + off, d + off, len, cudaMemcpyDeviceToHost,
                                         c->copy_st[k]);
        }
        for (int i = 0; i < ns && x == cudaSuccess; ++i) {
            x = cudaEventRecord(c->copy_ev[i], c->copy_st[i]);
            if (x == cudaSuccess)
                x = cudaStreamWaitEvent(st, c->copy_ev[i], 0);
        }
        return x;
    };
    e = spread(true);
    if (e != cudaSuccess)
        return to_status(e);
    if (n_recs > 1) {
        SortJob j{};
        j.in = (u64 *)c->host_in.p;
        j.tmp = (u64 *)c->host_tmp.p;
        j.n = n_recs;
        j.rw = rec_bytes / 8u;
        j.kw = key_bytes / 8u;
        j.stats = opts ? opts->stats : nullptr;
        j.mode = opts ? opts->mode : 0u;
        j.log2b = opts ? opts->learned_log2_buckets : 0u;
        j.fallback_ratio = opts ? opts->fallback_ratio : 0.f;
        j.train_steps = (opts && opts->train_steps) ? opts->train_steps : 16u;
        HostOut ho{(unsigned char *)h_out, d, rec_bytes, c->copy_st[0], c->win_ev, false};
        const char *wv = getenv("RADULS_HOST_WINDOWS");  // "0": copy back only after the whole sort
        j.hout = (wv && atoi(wv) == 0) ? nullptr : &ho;
        rc = run_sort(*c, c->main, j, st);
        if (rc)
            return rc;
        if (ho.copied) {
            // every record went back window by window: `stream` continues after the last copy
            e = cudaEventRecord(c->copy_ev[0], c->copy_st[0]);
            if (e == cudaSuccess)
                e = cudaStreamWaitEvent(st, c->copy_ev[0], 0);
            return to_status(e);
        }
    }
    e = spread(false);
    return to_status(e);
}

int raduls_model_fit(raduls_model **out, const void *in, uint64_t n_recs, uint32_t rec_bytes, uint32_t key_bytes,
                     uint32_t log2_buckets, uint32_t train_steps, void *stream)
{
    if (!out)
        return RADULS_ERR_INVALID_ARG;
    *out = nullptr;
    int rc = check_args(in, in, 0, rec_bytes, key_bytes);
    if (rc)
        return rc;
    if (n_recs < 2 || !in || log2_buckets < 8u || log2_buckets > 16u)
        return RADULS_ERR_INVALID_ARG;
    if ((uintptr_t)in & 15u)
        return RADULS_ERR_MISALIGNED;
    Ctx *c = current_ctx(&rc);
    if (!c)
        return rc;
    std::lock_guard<std::mutex> g(c->mu);
    cudaError_t e = ctx_init(*c);
    if (e != cudaSuccess)
        return to_status(e);
    cudaStream_t st = (cudaStream_t)stream;
    raduls_model *m = new (std::nothrow) raduls_model();
    if (!m)
        return RADULS_ERR_OOM;
    cudaGetDevice(&m->device);
    m->n = n_recs;
    // exact top-byte histogram of key word 0 (the root level)
    u64 *root = nullptr;
    e = cudaMalloc(&root, RADIX * 8);
    if (e != cudaSuccess) {
        delete m;
        return RADULS_ERR_OOM;
    }
    SortJob hj{};
    hj.in = (u64 *)in;
    hj.tmp = (u64 *)in;
    hj.n = n_recs;
    hj.rw = rec_bytes / 8u;
    hj.kw = key_bytes / 8u;
    hj.digit = 8u * hj.kw - 1u;
    hj.hist_out = root;
    hj.mode = 1;
    rc = run_sort(*c, c->main, hj, st);
    Recorder rec;
    rec.c = c;
    rec.st = st;
    // train_steps with the top bit set: warm start only, no Adam steps
    const bool warm_only = (train_steps & 0x80000000u) != 0;
    const u32 steps = warm_only ? 1u : train_steps;
    if (!rc)
        rc = model_fit(*c, m->m, (const u64 *)in, n_recs, rec_bytes / 8u, root, log2_buckets, steps, st, rec,
                       warm_only);
    cudaStreamSynchronize(st);
    cudaFree(root);
    if (rc) {
        if (m->m.buf.p)
            cudaFree(m->m.buf.p);
        delete m;
        return rc;
    }
    *out = m;
    return RADULS_OK;
}

int raduls_model_train(raduls_model *m, uint32_t stage, uint32_t steps, void *stream)
{
    if (!m || stage > 1u)
        return RADULS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ModelBufs &M = m->m;
    for (u32 k = 1; k <= steps; ++k) {
        cudaError_t e = lm_launch_step(M.model, stage, M.theta, M.am, M.av, M.h, M.tot, M.E, M.G, M.Z, M.loss,
                                       M.sample, M.seg_start, M.S, LEARN_RATE, (int)(M.steps_done + k), nullptr,
                                       st);
        if (e != cudaSuccess)
            return to_status(e);
    }
    M.steps_done += steps;
    return to_status(lm_launch_heights(M.model, M.theta, M.h, M.tot, M.E, M.G, M.Z, M.loss, st));
}

int raduls_model_loss_grad(raduls_model *m, uint32_t stage, double *h_loss, float *d_grad, void *stream)
{
    if (!m || !h_loss || !d_grad || stage > 1u)
        return RADULS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ModelBufs &M = m->m;
    cudaError_t e = lm_launch_step(M.model, stage, M.theta, M.am, M.av, M.h, M.tot, M.E, M.G, M.Z, M.loss,
                                   M.sample, M.seg_start, M.S, LEARN_RATE, 1, d_grad, st);
    if (e != cudaSuccess)
        return to_status(e);
    double l = 0;
    e = cudaMemcpyAsync(&l, M.loss, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    *h_loss = l / (double)M.S;
    return to_status(e);
}

int raduls_model_buckets(const raduls_model *m, const uint64_t *d_keys, uint64_t n_keys, uint32_t *d_out,
                         void *stream)
{
    if (!m || (n_keys && (!d_keys || !d_out)))
        return RADULS_ERR_INVALID_ARG;
    if (!n_keys)
        return RADULS_OK;
    return to_status(lm_launch_bucket(m->m.model, (const u64 *)d_keys, n_keys, d_out, (cudaStream_t)stream));
}

int raduls_model_sizes(const raduls_model *m, uint32_t *n_params, uint32_t *n_sample, uint32_t *log2_buckets)
{
    if (!m)
        return RADULS_ERR_INVALID_ARG;
    if (n_params)
        *n_params = m->m.n_params_cap;
    if (n_sample)
        *n_sample = m->m.S;
    if (log2_buckets)
        *log2_buckets = m->m.log2b;
    return RADULS_OK;
}

int raduls_model_copy_out(const raduls_model *m, uint64_t *h_root_counts, void *h_segments, float *h_theta,
                          float *h_heights, uint64_t *h_sample, void *stream)
{
    if (!m)
        return RADULS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const ModelBufs &M = m->m;
    cudaError_t e = cudaSuccess;
    if (h_root_counts && e == cudaSuccess)
        e = cudaMemcpyAsync(h_root_counts, M.model->root_cnt, RADIX * 8, cudaMemcpyDeviceToHost, st);
    if (h_segments && e == cudaSuccess)
        e = cudaMemcpyAsync(h_segments, M.model->seg, 2 * RADIX * sizeof(ModelSeg), cudaMemcpyDeviceToHost, st);
    if (h_theta && e == cudaSuccess)
        e = cudaMemcpyAsync(h_theta, M.theta, (size_t)M.n_params_cap * 4, cudaMemcpyDeviceToHost, st);
    if (h_heights && e == cudaSuccess)
        e = cudaMemcpyAsync(h_heights, M.h, (size_t)M.n_params_cap * 4, cudaMemcpyDeviceToHost, st);
    if (h_sample && e == cudaSuccess)
        e = cudaMemcpyAsync(h_sample, M.sample, (size_t)M.S * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    return to_status(e);
}

void raduls_model_free(raduls_model *m)
{
    if (!m)
        return;
    if (m->m.buf.p)
        cudaFree(m->m.buf.p);
    delete m;
}

int raduls_sort_batched(void *in, void *tmp, const uint64_t *d_seg_offsets, uint32_t n_segs, uint32_t rec_bytes,
                        uint32_t key_bytes, void *stream)
{
    int rc = check_args(in, tmp, 0, rec_bytes, key_bytes);
    if (rc)
        return rc;
    if (n_segs == 0)
        return RADULS_OK;
    if (!d_seg_offsets || !in || !tmp)
        return RADULS_ERR_INVALID_ARG;
    if (((uintptr_t)d_seg_offsets & 7u) || ((uintptr_t)in & 15u) || ((uintptr_t)tmp & 15u))
        return RADULS_ERR_MISALIGNED;
    Ctx *c = current_ctx(&rc);
    if (!c)
        return rc;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaStream_t st = (cudaStream_t)stream;
    // the total record count sizes the workspace: read the last offset
    u64 n = 0;
    cudaError_t e = cudaMemcpyAsync(&n, d_seg_offsets + n_segs, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return to_status(e);
    rc = check_args(in, tmp, n, rec_bytes, key_bytes);
    if (rc)
        return rc;
    if (n <= 1)
        return RADULS_OK;
    std::lock_guard<std::mutex> g(c->mu);
    e = ctx_init(*c);
    if (e != cudaSuccess)
        return to_status(e);
    return run_batched(*c, dev, (u64 *)in, (u64 *)tmp, (const u64 *)d_seg_offsets, n_segs, n, rec_bytes / 8u,
                       key_bytes / 8u, st);
}

int raduls_autotune(void *in, void *tmp, uint64_t n_recs, uint32_t rec_bytes, uint32_t key_bytes,
                    const uint64_t *d_seg_offsets, uint32_t n_segs, raduls_tuning *out, void *stream)
{
    int rc = check_args(in, tmp, n_recs, rec_bytes, key_bytes);
    if (rc)
        return rc;
    if (n_recs < 2 || (d_seg_offsets && n_segs == 0))
        return RADULS_ERR_INVALID_ARG;
    if (d_seg_offsets && ((uintptr_t)d_seg_offsets & 7u))
        return RADULS_ERR_MISALIGNED;
    Ctx *c = current_ctx(&rc);
    if (!c)
        return rc;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= TUNE_DEVICES || rec_bytes / 8u > 32u)
        return RADULS_ERR_UNSUPPORTED;
    const bool batched = d_seg_offsets != nullptr;
    const u32 rw = rec_bytes / 8u, kw = key_bytes / 8u;
    cudaStream_t st = (cudaStream_t)stream;
    // Candidates, one setting at a time from the defaults (coordinate descent):
    // every distribution variant of this record width, the widest digit of a
    // distribution pass (12 down to 8 bits), the sub-bin size the digit widths
    // aim at, the on-chip class at its full and half size, the mid-size class
    // full / half / off.  A later candidate must beat the current choice by
    // more than TIE_FRAC: within timing noise the default, larger size classes
    // stay, which suits inputs less regular than the tuner's seeded records.
    Tuned none{};
    g_force = &none;
    const Shape base = choose_shape(rw, kw, batched);
    g_force = nullptr;
    constexpr float TIE_FRAC = 0.01f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return RADULS_ERR_CUDA;
    }
    Tuned best{};
    best.valid = true;
    best.scat_var = base.scat_var;
    best.cap_b = base.cap_b;
    best.bucket_max = base.bucket_max;
    best.wmax = base.wmax;
    best.leaf = base.leaf;
    float best_ms = 0.f;
    bool have_best = false;
    u32 timed = 0;
    rc = RADULS_OK;
    auto time_one = [&](const Tuned &t, float &ms_min) {
        for (int rep = 0; rep < 2 && rc == RADULS_OK; ++rep) {
            tune_fill_kernel<<<1024, 256, 0, st>>>((u64 *)in, n_recs * rw, 0x5241445553ull + rep);
            if (cudaGetLastError() != cudaSuccess) {
                rc = RADULS_ERR_CUDA;
                break;
            }
            g_force = &t;
            cudaEventRecord(e0, st);
            {
                std::lock_guard<std::mutex> g(c->mu);
                cudaError_t e = ctx_init(*c);
                if (e != cudaSuccess) {
                    rc = to_status(e);
                } else if (batched) {
                    rc = run_batched(*c, dev, (u64 *)in, (u64 *)tmp, (const u64 *)d_seg_offsets, n_segs, n_recs, rw,
                                     kw, st);
                } else {
                    SortJob j{};
                    j.in = (u64 *)in;
                    j.tmp = (u64 *)tmp;
                    j.n = n_recs;
                    j.rw = rw;
                    j.kw = kw;
                    j.mode = 1;
                    j.train_steps = 16u;
                    rc = run_sort(*c, c->main, j, st);
                }
            }
            g_force = nullptr;
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                cudaGetLastError();
                rc = RADULS_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms_min = (rep == 0 || ms < ms_min) ? ms : ms_min;
        }
        if (rc == RADULS_OK) {
            const int srt = raduls_stream_status(stream);
            if (srt != RADULS_OK)
                rc = srt;
        }
        if (rc != RADULS_OK)
            return;
        ++timed;
        if (!have_best || ms_min < best_ms * (1.f - TIE_FRAC)) {
            best = t;
            best_ms = ms_min;
            have_best = true;
        }
    };
    float ms = 0.f;
    // untimed sorts first: the GPU leaves its idle clocks and the workspace is
    // allocated before anything is compared
    {
        const Tuned warm = best;
        for (int i = 0; i < 3 && rc == RADULS_OK; ++i) {
            time_one(warm, ms);
            have_best = false;
            timed = 0;
        }
    }
    time_one(best, ms);
    const Tuned base_t = best;
    for (int v = 0; v < 16 && rc == RADULS_OK; ++v) {
        if (v == base.scat_var || !scatter_variant_fits(v, rw) || ((v == 3 || v == 4) && rw <= 4))
            continue;
        Tuned t = best;
        t.scat_var = v;
        if ((1u << t.wmax) > wscatter_kmax_of(v))
            t.wmax = 8;
        time_one(t, ms);
    }
    for (u32 wm = WIDE_MAX; wm >= 8u && rc == RADULS_OK; --wm) {
        if (wm == best.wmax || (1u << wm) > wscatter_kmax_of(best.scat_var))
            continue;
        Tuned t = best;
        t.wmax = wm;
        time_one(t, ms);
    }
    const u32 leaves[2] = {base.cap_b / 2u, WARP_BIN / 2u};
    for (int li = 0; li < 2 && rc == RADULS_OK; ++li) {
        if (leaves[li] == best.leaf || leaves[li] < 16u)
            continue;
        Tuned t = best;
        t.leaf = leaves[li];
        time_one(t, ms);
    }
    if (rc == RADULS_OK && rw == 2 && !batched && base.bins_var < 0) {
        // the on-chip class at twice the size
        Tuned t = best;
        t.cap_b = block_cap_of(5);
        if (t.bucket_max && t.bucket_max <= t.cap_b)
            t.bucket_max = 0;
        t.leaf = 0;
        time_one(t, ms);
    }
    if (rc == RADULS_OK && base.cap_b / 2u > WARP_BIN) {
        Tuned t = best;
        t.cap_b = base.cap_b / 2u;
        if (t.leaf > t.cap_b)
            t.leaf = t.cap_b / 2u;
        if (t.bucket_max && t.bucket_max <= t.cap_b)
            t.bucket_max = 0;
        time_one(t, ms);
    }
    if (rc == RADULS_OK && base.bins_var >= 0) {
        // the general on-chip kernel alone (the streamed bin sort off)
        Tuned t = best;
        t.bins = 2;
        t.cap_b = 0;
        t.leaf = 0;
        time_one(t, ms);
    }
    // the mid-size class: at half size and off when it is on by default, at
    // full and half size when it is off
    const u32 bfull = base.bucket_var < 0 ? 0u : 640u * 1024u / (rw * 8u);
    const u32 bmaxes[2] = {base.bucket_max ? base.bucket_max / 2u : (bfull < BUCKET_IDX_MAX ? bfull : BUCKET_IDX_MAX),
                           base.bucket_max ? 0u : bfull / 2u};
    for (int bi = 0; bi < 2 && base.bucket_var >= 0 && rc == RADULS_OK; ++bi) {
        Tuned t = best;
        t.bucket_max = bmaxes[bi] > t.cap_b ? bmaxes[bi] : 0u;
        if (t.bucket_max == best.bucket_max)
            continue;
        time_one(t, ms);
    }
    // the winner against the default once more, alternating, best of three
    // each: the default stays unless the winner is clearly faster
    if (rc == RADULS_OK && (best.scat_var != base_t.scat_var || best.wmax != base_t.wmax ||
                            best.leaf != base_t.leaf || best.cap_b != base_t.cap_b ||
                            best.bucket_max != base_t.bucket_max || best.bins != base_t.bins)) {
        const Tuned win = best;
        float mw = 1e30f, mb = 1e30f;
        for (int i = 0; i < 3 && rc == RADULS_OK; ++i) {
            float x = 0.f;
            have_best = false;
            time_one(win, x);
            mw = x < mw ? x : mw;
            have_best = false;
            time_one(base_t, x);
            mb = x < mb ? x : mb;
        }
        if (mw < mb * (1.f - TIE_FRAC)) {
            best = win;
            best_ms = mw;
        } else {
            best = base_t;
            best_ms = mb;
        }
    }
    g_force = nullptr;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != RADULS_OK)
        return rc;
    {
        std::lock_guard<std::mutex> g(g_tuned_mu);
        g_tuned[dev][batched ? 1 : 0][rw] = best;
    }
    if (out) {
        out->scatter_variant = best.scat_var;
        out->scatter_tile = wscatter_tile_of(best.scat_var);
        out->block_cap = best.cap_b;
        out->bucket_max = best.bucket_max;
        out->best_ms = best_ms;
        out->candidates = timed;
        out->digit_bits = best.wmax;
        out->leaf = best.leaf;
        out->bin_sort = best.bins == 2 ? 0u : (base.bins_var >= 0 ? 1u : 0u);
    }
    return RADULS_OK;
}

int raduls_autotune_reset(void)
{
    std::lock_guard<std::mutex> g(g_tuned_mu);
    for (auto &d : g_tuned)
        for (auto &k : d)
            for (auto &r : k)
                r = Tuned{};
    return RADULS_OK;
}

int raduls_histogram(const void *in, uint64_t n_recs, uint32_t rec_bytes, uint32_t key_bytes, uint32_t digit,
                     uint64_t *d_hist_out, void *stream)
{
    if (rec_bytes % 8u || key_bytes % 8u || key_bytes < 8u || key_bytes > rec_bytes || digit >= key_bytes)
        return RADULS_ERR_INVALID_ARG;
    if (rec_bytes > 256u)
        return RADULS_ERR_UNSUPPORTED;
    if (!d_hist_out || (n_recs > 0 && !in))
        return RADULS_ERR_INVALID_ARG;
    if (((uintptr_t)in & 15u) || ((uintptr_t)d_hist_out & 7u))
        return RADULS_ERR_MISALIGNED;
    int rc = 0;
    Ctx *c = current_ctx(&rc);
    if (!c)
        return rc;
    if (n_recs == 0) {
        cudaError_t e = cudaMemsetAsync(d_hist_out, 0, RADIX * 8, (cudaStream_t)stream);
        return to_status(e);
    }
    std::lock_guard<std::mutex> g(c->mu);
    cudaError_t e = ctx_init(*c);
    if (e != cudaSuccess)
        return to_status(e);
    SortJob j{};
    j.in = (u64 *)in;
    j.tmp = (u64 *)in;
    j.n = n_recs;
    j.rw = rec_bytes / 8u;
    j.kw = key_bytes / 8u;
    j.digit = digit;
    j.hist_out = reinterpret_cast<u64 *>(d_hist_out);
    j.mode = 1;
    return run_sort(*c, c->main, j, (cudaStream_t)stream);
}

int raduls_distribution_pass(const void *in, void *out, uint64_t n_recs, uint32_t rec_bytes, uint32_t key_bytes,
                             uint32_t digit, void *stream)
{
    int rc = check_args(in, out, n_recs, rec_bytes, key_bytes);
    if (rc)
        return rc;
    if (digit >= key_bytes)
        return RADULS_ERR_INVALID_ARG;
    if (n_recs == 0)
        return RADULS_OK;
    if (n_recs == 1) {
        cudaError_t e = cudaMemcpyAsync(out, in, rec_bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
        return to_status(e);
    }
    Ctx *c = current_ctx(&rc);
    if (!c)
        return rc;
    std::lock_guard<std::mutex> g(c->mu);
    cudaError_t e = ctx_init(*c);
    if (e != cudaSuccess)
        return to_status(e);
    SortJob j{};
    j.in = (u64 *)in;
    j.tmp = (u64 *)out;
    j.n = n_recs;
    j.rw = rec_bytes / 8u;
    j.kw = key_bytes / 8u;
    j.digit = digit;
    j.single_pass = 1;
    j.mode = 1;
    return run_sort(*c, c->main, j, (cudaStream_t)stream);
}

int raduls_stream_status(void *stream)
{
    int rc = 0;
    Ctx *c = current_ctx(&rc);
    if (!c)
        return rc;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess)
        return RADULS_ERR_CUDA;
    std::lock_guard<std::mutex> g(c->mu);
    if (!c->inited)
        return RADULS_OK;
    u32 v = 0;
    e = cudaMemcpy(&v, c->dev_status, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return RADULS_ERR_CUDA;
    if (v) {
        e = cudaMemset(c->dev_status, 0, 4);
        if (e != cudaSuccess)
            return RADULS_ERR_CUDA;
    }
    return (int)v;
}

const char *raduls_status_string(int status)
{
    switch (status) {
    case RADULS_OK: return "ok";
    case RADULS_ERR_INVALID_ARG: return "invalid argument";
    case RADULS_ERR_MISALIGNED: return "buffer misaligned or overlapping";
    case RADULS_ERR_UNSUPPORTED: return "unsupported shape or mode";
    case RADULS_ERR_CUDA: return "CUDA runtime error";
    case RADULS_ERR_OOM: return "out of device memory for the workspace";
    case RADULS_ERR_TIMEOUT: return "device-side wait timed out";
    case RADULS_ERR_INTERNAL: return "internal capacity check failed on the device";
    default: return "unknown status";
    }
}

int raduls_debug_inject(uint32_t kind, uint64_t tile)
{
    std::lock_guard<std::mutex> g(g_setting_mu);
    if (kind == 0) {
        g_inject_tile = ~0u;
        return RADULS_OK;
    }
    if (kind == 1 && tile < 0xffffffffull) {
        g_inject_tile = (u32)tile;
        return RADULS_OK;
    }
    if (kind == 2 && tile < 0xffffffffull) {
        g_withhold_push = (u32)tile;
        return RADULS_OK;
    }
    return RADULS_ERR_INVALID_ARG;
}

int raduls_set_wait_limit_ns(uint64_t ns)
{
    if (ns == 0)
        return RADULS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(g_setting_mu);
    g_wait_ns = ns;
    return RADULS_OK;
}

}  // extern "C"
