// passes.cu -- the histogram-only traversal: the first traversal of Sec. 1's
// counting split (the digit histogram of a byte of the key) on its own, for
// raduls_histogram() and raduls_histogram_static().  The sort's own passes
// count and distribute in wide.cu.
#include "kernels.h"

namespace raduls {

// ----------------------------------------------------------------- histogram

template <int THREADS, int UNROLL>
__global__ void __launch_bounds__(THREADS)
hist_kernel(const u64 *__restrict__ in, const u64 *__restrict__ tmp, const WorkItem *__restrict__ items,
            const u32 *__restrict__ tile_item, u64 *__restrict__ hist, u64 *__restrict__ orand,
            Counters *__restrict__ ctrs, u32 tile_recs, u32 rw, u32 key_words)
{
    constexpr int NW = THREADS / 32;
    __shared__ u32 cnt[NW][RADIX + 1];
    __shared__ u64 red_or[NW], red_and[NW];
    __shared__ u32 s_tile;
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    const u32 n_tiles = ctrs->grid_cur_tiles;
    for (u32 i = lane; i < RADIX + 1; i += 32)
        cnt[w][i] = 0;
    // Counts, OR / AND and bytes accumulate over consecutive tiles of the same
    // bin and go to global memory when the bin changes (or at the end): the
    // tiles of one big bin would otherwise all hit the same few counters.
    u32 cur_row = ~0u;
    u64 vor = 0, vand = ~0ull, bytes = 0;
    for (;;) {
        if (tid == 0)
            s_tile = atomicAdd(&ctrs->tile_ctr[0], 1u);
        __syncthreads();
        const u32 t = s_tile;
        const u32 next_row = t < n_tiles ? items[tile_item[t]].row : ~0u;
        if (next_row != cur_row && cur_row != ~0u) {
            if (tid < RADIX) {
                u32 s = 0;
#pragma unroll
                for (int ww = 0; ww < NW; ++ww)
                    s += cnt[ww][tid];
                if (s)
                    atomicAdd(&hist[(u64)cur_row * RADIX + tid], (u64)s);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                vor |= __shfl_xor_sync(FULL_MASK, vor, o);
                vand &= __shfl_xor_sync(FULL_MASK, vand, o);
            }
            if (lane == 0) {
                red_or[w] = vor;
                red_and[w] = vand;
            }
            __syncthreads();
            if (tid == 0) {
                u64 o2 = 0, a2 = ~0ull;
#pragma unroll
                for (int i = 0; i < NW; ++i) {
                    o2 |= red_or[i];
                    a2 &= red_and[i];
                }
                atomicOr(&orand[2ull * cur_row], o2);
                atomicAnd(&orand[2ull * cur_row + 1], a2);
                atomicAdd(&ctrs->hist_bytes, bytes);
            }
            for (u32 i = lane; i < RADIX + 1; i += 32)
                cnt[w][i] = 0;
            vor = 0;
            vand = ~0ull;
            bytes = 0;
            __syncthreads();
        }
        if (t >= n_tiles)
            break;
        const WorkItem item = items[tile_item[t]];
        cur_row = item.row;
        const u64 lo = item.begin + (u64)(t - item.tile_base) * tile_recs;
        const u64 hi = min(item.begin + item.count, lo + tile_recs);
        const u64 *src = (item.flags & ITEM_IN_TMP) ? tmp : in;
        // digit p: byte p % 8 of key word W - 1 - p / 8
        const u32 word = key_words - 1u - item.digit / 8u, sh = 8u * (item.digit % 8u);
        bytes += (hi - lo) * (u64)min(rw * 8u, 32u);
        for (u64 base = lo; base < hi; base += (u64)THREADS * UNROLL) {
            u64 key[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const u64 i = base + (u64)u * THREADS + tid;
                key[u] = i < hi ? __ldcs(src + i * rw + word) : 0ull;
            }
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const u64 i = base + (u64)u * THREADS + tid;
                const bool valid = i < hi;
                const u32 d = valid ? (u32)(key[u] >> sh) & 0xffu : (u32)RADIX;
                if (valid) {
                    vor |= key[u];
                    vand &= key[u];
                }
                // one add for a warp whose lanes share a digit (skewed data), else one per lane
                const u32 d0 = __shfl_sync(FULL_MASK, d, 0);
                if (__all_sync(FULL_MASK, d == d0)) {
                    if (lane == 0)
                        cnt[w][d0] += 32u;
                } else {
                    atomicAdd(&cnt[w][d], 1u);
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------- launch

namespace {

template <typename KernelT>
u32 persistent_grid(KernelT kernel, int threads, size_t smem)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (per_sm < 1)
        per_sm = 1;
    return (u32)(sms * per_sm);
}

constexpr int HIST_THREADS = 512, HIST_UNROLL = 8;

}  // namespace

u32 hist_grid(const Shape &)
{
    return persistent_grid(hist_kernel<HIST_THREADS, HIST_UNROLL>, HIST_THREADS, 0);
}

cudaError_t launch_hist(const Shape &s, const u64 *in, const u64 *tmp, const WorkItem *items, const u32 *tile_item,
                        u64 *hist, u64 *orand, Counters *ctrs, cudaStream_t st)
{
    static thread_local int cached_dev = -1;
    static thread_local u32 grid = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != cached_dev) {
        grid = hist_grid(s);
        cached_dev = dev;
    }
    hist_kernel<HIST_THREADS, HIST_UNROLL><<<grid, HIST_THREADS, 0, st>>>(in, tmp, items, tile_item, hist, orand, ctrs,
                                                                         s.tile_h, s.rw, s.key_words);
    return cudaGetLastError();
}

}  // namespace raduls
