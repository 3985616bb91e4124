// driver.cu -- host driver and C ABI of the sorter (see include/raduls.h).
//
// The driver plays the part of the paper's scheduler (Fig. 1-3) with GPU work
// lists instead of threads and queues: it runs one MSD level at a time --
// histograms of every big bin, on-device planning, one device-wide
// distribution launch for all big bins of the level -- until no bin is bigger
// than what one CTA sorts on chip, then copies back finished bins left in the
// scratch buffer and runs the on-chip sorts of all small-bin runs.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "../../include/raduls.h"
#include "kernels.h"

namespace raduls {

u32 scatter_tile_of(int var);
u32 block_cap_of(int var);

Shape choose_shape(u32 rw, u32 key_words)
{
    Shape s{};
    s.rw = rw;
    s.key_words = key_words;
    s.tile_h = 16384;
    s.tile_c = 65536;
    if (rw == 1) {
        s.scat_var = 0;
        s.block_var = 0;
    } else if (rw == 2) {
        s.scat_var = 1;
        s.block_var = 1;
    } else if (rw == 4) {
        s.scat_var = 2;
        s.block_var = 2;
    } else if (rw <= 8) {
        s.scat_var = 3;
        s.block_var = 3;
    } else {
        s.scat_var = 4;
        s.block_var = 4;
    }
    s.tile_s = scatter_tile_of(s.scat_var);
    s.cap_b = block_cap_of(s.block_var);
    return s;
}

namespace {

constexpr int MAX_DEVICES = 64;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct Ctx {
    std::mutex mu;
    bool inited = false;
    Counters *ctrs = nullptr;      // device
    Counters *h_ctrs = nullptr;    // pinned host mirror
    u32 *dev_status = nullptr;     // device: sticky status word of this device
    DevBuf lists, hist, status, tiles;
    u32 epoch = 0;
    u64 wait_ns = 2000000000ull;
    u32 inject_tile = ~0u;
    cudaEvent_t ev[1024] = {};
    bool have_events = false;
};

Ctx g_ctx[MAX_DEVICES];

std::mutex g_setting_mu;
u64 g_wait_ns = 2000000000ull;
u32 g_inject_tile = ~0u;

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
    WorkItem *blocks;
    WorkItem *copies;
    u32 *tile_hist;
    u32 *tile_copy;
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

cudaError_t ctx_init(Ctx &c)
{
    if (c.inited)
        return cudaSuccess;
    cudaError_t e = cudaMalloc(&c.ctrs, sizeof(Counters));
    if (e != cudaSuccess)
        return e;
    e = cudaMalloc(&c.dev_status, 256);
    if (e != cudaSuccess)
        return e;
    e = cudaMemset(c.dev_status, 0, 256);
    if (e != cudaSuccess)
        return e;
    e = cudaMallocHost(&c.h_ctrs, sizeof(Counters));
    if (e != cudaSuccess)
        return e;
    c.inited = true;
    return cudaSuccess;
}

// Sizes every list for a problem of n records (upper bounds, see below).
cudaError_t ctx_lists(Ctx &c, const Shape &s, u64 n, Lists &L)
{
    const u64 W = s.key_words;
    const u64 grid_cap = n / ((u64)s.cap_b + 1) + 2;                 // grid bins hold > cap_b records each
    const u64 hist_tiles = n / s.tile_h + grid_cap + 2;
    const u64 copy_cap = 8 * W * grid_cap + 2;                        // one per finished big bin
    const u64 copy_tiles = n / s.tile_c + copy_cap + 2;
    u64 block_cap = 2 * n / s.cap_b + 2 * 8 * W * grid_cap + 4;       // full runs + runs cut by big bins/parents
    if (block_cap > n + 4)
        block_cap = n + 4;
    if (grid_cap > 0xffffffffull || hist_tiles > 0xffffffffull || copy_tiles > 0xffffffffull)
        return cudaErrorInvalidValue;
    size_t off = 0, o_grid0, o_grid1, o_scat, o_blocks, o_copies, o_th, o_tc;
    o_grid0 = off; off = align256(off + grid_cap * sizeof(WorkItem));
    o_grid1 = off; off = align256(off + grid_cap * sizeof(WorkItem));
    o_scat = off; off = align256(off + grid_cap * sizeof(WorkItem));
    o_blocks = off; off = align256(off + block_cap * sizeof(WorkItem));
    o_copies = off; off = align256(off + copy_cap * sizeof(WorkItem));
    o_th = off; off = align256(off + hist_tiles * 4);
    o_tc = off; off = align256(off + copy_tiles * 4);
    cudaError_t e = ensure(c.lists, off, false);
    if (e != cudaSuccess)
        return e;
    char *b = (char *)c.lists.p;
    L.grid[0] = (WorkItem *)(b + o_grid0);
    L.grid[1] = (WorkItem *)(b + o_grid1);
    L.scat = (WorkItem *)(b + o_scat);
    L.blocks = (WorkItem *)(b + o_blocks);
    L.copies = (WorkItem *)(b + o_copies);
    L.tile_hist = (u32 *)(b + o_th);
    L.tile_copy = (u32 *)(b + o_tc);
    L.caps.grid = (u32)grid_cap;
    L.caps.hist_tiles = (u32)hist_tiles;
    L.caps.copy = (u32)copy_cap;
    L.caps.copy_tiles = (u32)copy_tiles;
    L.caps.block = block_cap;
    L.caps.scat_tiles = 0;
    return cudaSuccess;
}

// Per-level buffers: histogram rows of the current big bins and the look-back
// status words of this level's distribution tiles.
cudaError_t ctx_level(Ctx &c, const Shape &s, u64 n, u32 n_grid, u64 **hist, u64 **orand, u64 **status,
                      u32 **tile_scat, Caps &caps, cudaStream_t st)
{
    const u64 rows = (u64)n_grid + 1;
    cudaError_t e = ensure(c.hist, align256(rows * RADIX * 8) + rows * 16, false);
    if (e != cudaSuccess)
        return e;
    *hist = (u64 *)c.hist.p;
    *orand = (u64 *)((char *)c.hist.p + align256(rows * RADIX * 8));
    const u64 st_tiles = n / s.tile_s + n_grid + 2;
    if (st_tiles > 0xffffffffull)
        return cudaErrorInvalidValue;
    bool grew = false;
    e = ensure(c.status, st_tiles * RADIX * 8, true, &grew, st);
    if (e != cudaSuccess)
        return e;
    if (grew)
        c.epoch = 0;
    e = ensure(c.tiles, st_tiles * 4, false);
    if (e != cudaSuccess)
        return e;
    *status = (u64 *)c.status.p;
    *tile_scat = (u32 *)c.tiles.p;
    caps.scat_tiles = (u32)(c.status.bytes / (RADIX * 8));
    if ((u64)caps.scat_tiles * 4 > c.tiles.bytes)
        caps.scat_tiles = (u32)(c.tiles.bytes / 4);
    return cudaSuccess;
}

u32 next_epoch(Ctx &c, cudaStream_t st)
{
    c.epoch += 1;
    if (c.epoch >= LB_EPOCH_MASK) {
        cudaMemsetAsync(c.status.p, 0, c.status.bytes, st);
        c.epoch = 1;
    }
    return c.epoch;
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

int run_sort(Ctx &c, const SortJob &j, cudaStream_t st)
{
    const Shape s = choose_shape(j.rw, j.kw);
    Lists L{};
    CK(ctx_lists(c, s, j.n, L));
    Recorder rec;
    rec.c = &c;
    rec.st = st;
    if (j.stats) {
        CK(ctx_events(c));
        rec.timing = true;
    }
    const u32 top = 8u * j.kw - 1u;
    const bool step_api = j.single_pass || j.hist_out;
    TIMED(RADULS_K_SETUP, launch_init(c.ctrs, L.grid[0], L.blocks, L.tile_hist, j.n, step_api ? j.digit : top,
                                      s.cap_b, s.tile_h, step_api ? 1u : 0u, st));
    {
        std::lock_guard<std::mutex> g(g_setting_mu);
        c.wait_ns = g_wait_ns;
        c.inject_tile = g_inject_tile;
        g_inject_tile = ~0u;
    }
    int cur = 0;
    u32 n_grid = (step_api || j.n > s.cap_b) ? 1u : 0u;
    for (u32 level = 0; n_grid > 0; ++level) {
        u64 *hist, *orand, *status;
        u32 *tile_scat;
        CK(ctx_level(c, s, j.n, n_grid, &hist, &orand, &status, &tile_scat, L.caps, st));
        TIMED(RADULS_K_SETUP, launch_prep(hist, orand, c.ctrs, n_grid, st));
        TIMED(RADULS_K_HIST, launch_hist(s, j.in, j.tmp, L.grid[cur], L.tile_hist, hist, orand, c.ctrs, st));
        if (j.hist_out) {
            CK(cudaMemcpyAsync(j.hist_out, hist, RADIX * 8, cudaMemcpyDeviceToDevice, st));
            break;
        }
        PlanArgs a{};
        a.grid_cur = L.grid[cur];
        a.grid_next = L.grid[cur ^ 1];
        a.scat = L.scat;
        a.blocks = L.blocks;
        a.copies = L.copies;
        a.hist = hist;
        a.orand = orand;
        a.tile_hist = L.tile_hist;
        a.tile_scat = tile_scat;
        a.tile_copy = L.tile_copy;
        a.ctrs = c.ctrs;
        a.caps = L.caps;
        a.key_words = j.kw;
        a.rw = j.rw;
        a.cap_b = s.cap_b;
        a.tile_h = s.tile_h;
        a.tile_s = s.tile_s;
        a.tile_c = s.tile_c;
        a.single_pass = j.single_pass ? 1u : 0u;
        TIMED(RADULS_K_PLAN, launch_plan(a, n_grid, st));
        const u32 epoch = next_epoch(c, st);
        TIMED(RADULS_K_SCATTER, launch_scatter(s, j.in, j.tmp, L.scat, tile_scat, hist, status, c.ctrs, epoch,
                                               c.wait_ns, c.inject_tile, st));
        c.inject_tile = ~0u;
        TIMED(RADULS_K_SETUP, launch_advance(c.ctrs, st));
        if (j.single_pass)
            break;
        CK(cudaMemcpyAsync(c.h_ctrs, c.ctrs, sizeof(Counters), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (c.h_ctrs->err)
            break;
        n_grid = c.h_ctrs->grid_cur;
        cur ^= 1;
    }
    if (!step_api) {
        TIMED(RADULS_K_COPY, launch_copy(s, j.in, j.tmp, L.copies, L.tile_copy, c.ctrs, st));
        TIMED(RADULS_K_BLOCK, launch_block_sort(s, j.in, j.tmp, L.blocks, c.ctrs, st));
    }
    CK(rec.begin(RADULS_K_SETUP));
    fold_status_kernel<<<1, 1, 0, st>>>(c.ctrs, c.dev_status);
    CK(cudaGetLastError());
    CK(rec.end());
    if (j.stats) {
        CK(cudaMemcpyAsync(c.h_ctrs, c.ctrs, sizeof(Counters), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const Counters &h = *c.h_ctrs;
        raduls_stats &o = *j.stats;
        o.grid_passes = h.grid_passes;
        o.levels = h.levels;
        o.hist_bytes_read = h.hist_bytes;
        o.scatter_bytes = h.scatter_bytes;
        o.block_bytes = h.block_bytes;
        o.block_items = h.block;
        o.skipped_digits = h.skipped;
        o.gpu_launches = rec.total;
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

using namespace raduls;

extern "C" {

int raduls_sort_ex(void *in, void *tmp, uint64_t n_recs, uint32_t rec_bytes, uint32_t key_bytes,
                   const raduls_opts *opts, void *stream)
{
    int rc = check_args(in, tmp, n_recs, rec_bytes, key_bytes);
    if (rc)
        return rc;
    if (opts && opts->mode > 2u)
        return RADULS_ERR_INVALID_ARG;
    if (opts && opts->mode == 2u)
        return RADULS_ERR_UNSUPPORTED;
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
    return run_sort(*c, j, (cudaStream_t)stream);
}

int raduls_sort(void *in, void *tmp, uint64_t n_recs, uint32_t rec_bytes, uint32_t key_bytes, void *stream)
{
    return raduls_sort_ex(in, tmp, n_recs, rec_bytes, key_bytes, nullptr, stream);
}

int raduls_sort_batched(void *in, void *tmp, const uint64_t *d_seg_offsets, uint32_t n_segs, uint32_t rec_bytes,
                        uint32_t key_bytes, void *stream)
{
    (void)in;
    (void)tmp;
    (void)d_seg_offsets;
    (void)n_segs;
    (void)rec_bytes;
    (void)key_bytes;
    (void)stream;
    return RADULS_ERR_UNSUPPORTED;
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
    return run_sort(*c, j, (cudaStream_t)stream);
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
    return run_sort(*c, j, (cudaStream_t)stream);
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
