// noalloc.cu -- a digit histogram that allocates nothing.
//
// raduls_histogram() keeps its scratch (work counters, the work item, the
// tile map and the histogram row) in the library's per-device workspace,
// which is allocated with cudaMalloc on first use and grown on demand.  Some
// callers cannot let a library allocate: an application whose memory is all
// reserved up front by its own allocator (cudaMalloc would fail or fragment
// its pool), a latency-critical loop that cannot afford the device-wide
// synchronisation cudaMalloc/cudaFree imply, or code running while a stream
// is being captured, where allocation calls are not allowed.
// raduls_histogram_static() serves them: its scratch is the fixed array below,
// which every GPU that loads the library holds until the process exits.
#include <mutex>

#include "raduls.h"
#include "kernels.h"

namespace raduls {
namespace {

// Scratch of raduls_histogram_static(): counters (256 B), one work item
// (256 B), the histogram row and OR/AND words (4 KiB), then one u32 per
// histogram tile.  1 MiB in all.
constexpr size_t STATIC_SCRATCH_BYTES = 1u << 20;
constexpr size_t OFF_CTRS = 0, OFF_ITEM = 256, OFF_HIST = 512, OFF_ORAND = OFF_HIST + RADIX * 8,
                 OFF_LIGHT = OFF_ORAND + 256, OFF_TILES = OFF_LIGHT + RADIX * 8;
static_assert(sizeof(Counters) <= OFF_ITEM - OFF_CTRS, "counters fit");
constexpr u64 STATIC_MAX_TILES = (STATIC_SCRATCH_BYTES - OFF_TILES) / 4;
// Records per histogram tile of this entry point: fixed (not the tuned shape's
// tile), so its size limit is the documented one: 260,928 tiles x 16,384.
constexpr u32 STATIC_TILE = 16384;
static_assert(STATIC_MAX_TILES == 260928, "documented tile limit");

static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

constexpr int MAX_DEV = 64;
std::mutex g_static_mu;
unsigned char *g_static_ptr[MAX_DEV] = {};

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).  In host code the array's name is
// only a host-side handle, never a device address.
int static_scratch(unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) {
        cudaGetLastError();
        return RADULS_ERR_CUDA;
    }
    std::lock_guard<std::mutex> g(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return RADULS_ERR_CUDA;
        }
        g_static_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_static_ptr[dev];
    return RADULS_OK;
}

}  // namespace
}  // namespace raduls

using namespace raduls;

extern "C" int raduls_histogram_static(const void *in, uint64_t n_recs, uint32_t rec_bytes, uint32_t key_bytes,
                                       uint32_t digit, uint64_t *d_hist_out, void *stream)
{
    if (rec_bytes % 8u || key_bytes % 8u || key_bytes < 8u || key_bytes > rec_bytes || digit >= key_bytes)
        return RADULS_ERR_INVALID_ARG;
    if (rec_bytes > 256u)
        return RADULS_ERR_UNSUPPORTED;
    if (!d_hist_out || (n_recs > 0 && !in))
        return RADULS_ERR_INVALID_ARG;
    if (((uintptr_t)in & 15u) || ((uintptr_t)d_hist_out & 7u))
        return RADULS_ERR_MISALIGNED;
    // the tile map is the only part that grows with n: reject what does not fit
    if ((n_recs + STATIC_TILE - 1) / STATIC_TILE > STATIC_MAX_TILES)
        return RADULS_ERR_UNSUPPORTED;
    Shape s = choose_shape(rec_bytes / 8u, key_bytes / 8u);
    s.tile_h = STATIC_TILE;
    cudaStream_t st = (cudaStream_t)stream;
    if (n_recs == 0) {
        const cudaError_t e = cudaMemsetAsync(d_hist_out, 0, RADIX * 8, st);
        return e == cudaSuccess ? RADULS_OK : RADULS_ERR_CUDA;
    }
    unsigned char *base = nullptr;
    int rc = static_scratch(&base);
    if (rc)
        return rc;
    Counters *ctrs = reinterpret_cast<Counters *>(base + OFF_CTRS);
    WorkItem *item = reinterpret_cast<WorkItem *>(base + OFF_ITEM);
    u64 *hist = reinterpret_cast<u64 *>(base + OFF_HIST);
    u64 *orand = reinterpret_cast<u64 *>(base + OFF_ORAND);
    u32 *tiles = reinterpret_cast<u32 *>(base + OFF_TILES);
    // every scratch field is rewritten before it is read: init writes the
    // counters, the work item and the tile map; prep zeroes the row
    cudaError_t e = launch_init(ctrs, item, item, tiles, n_recs, digit, s.cap_b, s.tile_h, 1u, nullptr, 0u, nullptr, 0u, 0u,
                                st);
    if (e == cudaSuccess)
        e = launch_prep(hist, orand, ctrs, 1u, 1u, st);
    if (e == cudaSuccess)
        e = launch_hist(s, (const u64 *)in, (const u64 *)in, item, tiles, hist, orand, ctrs, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_hist_out, hist, RADIX * 8, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return RADULS_ERR_CUDA;
    }
    return RADULS_OK;
}
