// passes.cu -- the two device-wide kernels of one MSD distribution pass.
//
// A pass over a bin on digit p follows the counting split of Sec. 1: a first
// traversal builds the bin's digit histogram (hist_kernel), an exclusive prefix
// turns it into the start of every digit's sub-bin (plan.cu), and a second
// traversal distributes whole records stably (scatter_kernel).  Sec. 3.2-3.3
// run this split with many threads on one big bin; here every CTA takes the
// next tile of a bin, ranks the tile's records by digit on chip, and learns
// where its records of each digit go from a single-pass decoupled look-back
// over the tiles of the same bin (Merrill & Garland, "Single-pass Parallel
// Prefix Scan with Decoupled Look-back", 2016; own implementation).  The tile
// is regrouped by digit in shared memory before it is written, so each
// digit's records leave as one contiguous run: the GPU counterpart of the
// paper's write-combining buffers (Sec. 2, Sec. 3.2).
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
    __shared__ u32 s_tile;
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    const u32 n_tiles = ctrs->grid_cur_tiles;
    for (;;) {
        if (tid == 0)
            s_tile = atomicAdd(&ctrs->tile_ctr[0], 1u);
        for (u32 i = lane; i < RADIX + 1; i += 32)
            cnt[w][i] = 0;
        __syncthreads();
        const u32 t = s_tile;
        if (t >= n_tiles)
            break;
        const WorkItem item = items[tile_item[t]];
        const u64 lo = item.begin + (u64)(t - item.tile_base) * tile_recs;
        const u64 hi = min(item.begin + item.count, lo + tile_recs);
        const u64 *src = (item.flags & ITEM_IN_TMP) ? tmp : in;
        const u32 wi = key_words - 1u - item.digit / 8u, sh = 8u * (item.digit % 8u);
        u64 vor = 0, vand = ~0ull;
        for (u64 base = lo; base < hi; base += (u64)THREADS * UNROLL) {
            u64 key[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const u64 i = base + (u64)u * THREADS + tid;
                key[u] = i < hi ? __ldcs(src + i * rw + wi) : 0ull;
            }
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const u64 i = base + (u64)u * THREADS + tid;
                const bool valid = i < hi;
                const u32 d = valid ? digit_of_word(key[u], sh) : (u32)RADIX;
                if (valid) {
                    vor |= key[u];
                    vand &= key[u];
                }
                const u32 peers = __match_any_sync(FULL_MASK, d);
                if ((peers & lanemask_lt()) == 0)
                    cnt[w][d] += __popc(peers);
                __syncwarp();
            }
        }
        __syncthreads();
        if (tid < RADIX) {
            u32 s = 0;
#pragma unroll
            for (int ww = 0; ww < NW; ++ww)
                s += cnt[ww][tid];
            if (s)
                atomicAdd(&hist[(u64)item.row * RADIX + tid], (u64)s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vor |= __shfl_xor_sync(FULL_MASK, vor, o);
            vand &= __shfl_xor_sync(FULL_MASK, vand, o);
        }
        if (lane == 0) {
            atomicOr(&orand[2ull * item.row], vor);
            atomicAnd(&orand[2ull * item.row + 1], vand);
        }
        if (tid == 0)
            atomicAdd(&ctrs->hist_bytes, (hi - lo) * (u64)min(rw * 8u, 32u));
        __syncthreads();
    }
}

// -------------------------------------------------------------- distribution

template <int THREADS, int K>
struct ScatterSmem {
    RankSmem<THREADS> rank;
    u64 goff[RADIX];              // global start of each digit's run, minus its tile start
    unsigned short perm[THREADS * K];  // tile-sorted slot -> element
    u32 tile;
    u32 abort;
};

constexpr size_t round16(size_t x) { return (x + 15) & ~(size_t)15; }

template <int THREADS, int K>
constexpr size_t scatter_smem_bytes(u32 rw)
{
    return round16(sizeof(ScatterSmem<THREADS, K>)) + ((size_t)THREADS * K * rw + 2) * 8;
}

template <int THREADS, int K, int RW>
__global__ void __launch_bounds__(THREADS)
scatter_kernel(u64 *__restrict__ in, u64 *__restrict__ tmp, const WorkItem *__restrict__ items,
               const u32 *__restrict__ tile_item, const u64 *__restrict__ bases, u64 *__restrict__ status,
               Counters *__restrict__ ctrs, u32 rw_rt, u32 key_words, u32 epoch, u64 wait_ns, u32 inject_tile)
{
    constexpr u32 TILE = THREADS * K;
    static_assert(TILE <= 65536, "tile slots are 16-bit");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScatterSmem<THREADS, K> &sm = *reinterpret_cast<ScatterSmem<THREADS, K> *>(smem_raw);
    u64 *const recs_base = reinterpret_cast<u64 *>(smem_raw + round16(sizeof(ScatterSmem<THREADS, K>)));
    const u32 rw = RW ? (u32)RW : rw_rt;
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    const u32 n_tiles = ctrs->scatter_tiles;
    const u32 ep = epoch & LB_EPOCH_MASK;

    for (;;) {
        if (tid == 0) {
            sm.tile = atomicAdd(&ctrs->tile_ctr[1], 1u);
            sm.abort = 0;
        }
        __syncthreads();
        const u32 t = sm.tile;
        if (t >= n_tiles)
            break;
        const WorkItem item = items[tile_item[t]];
        const u32 j = t - item.tile_base;
        const u64 lo = item.begin + (u64)j * TILE;
        const u32 m = (u32)min((u64)TILE, item.begin + item.count - lo);
        const u64 *src = (item.flags & ITEM_IN_TMP) ? tmp : in;
        u64 *dst = (item.flags & ITEM_IN_TMP) ? in : tmp;
        const u32 wi = key_words - 1u - item.digit / 8u, sh = 8u * (item.digit % 8u);
        // keep shared and global 16-byte phases equal so the bulk moves as vectors
        const u32 s0 = (u32)((lo * rw) & 1u);
        u64 *recs = recs_base + s0;
        load_words<THREADS>(recs, src + lo * rw, (u64)m * rw);
        __syncthreads();

        // rank the tile's records by digit, stably (warp-contiguous layout)
        u32 dig[K], rk[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const u32 e = w * 32u * K + (u32)k * 32u + lane;
            dig[k] = e < m ? digit_of_word(recs[(u64)e * rw + wi], sh) : (u32)RADIX;
        }
        warp_rank<THREADS, K>(sm.rank, dig, rk);
        __syncthreads();
        u32 total = 0;
        if (tid < RADIX) {
            total = warp_offsets<THREADS>(sm.rank, tid);
            // publish this tile's count of digit tid (inclusive if first tile of the bin)
            if (t != inject_tile)
                st_relaxed_u64(&status[(u64)t * RADIX + tid], lb_pack(j == 0 ? LB_INC : LB_AGG, ep, total));
        }
        scan_totals<THREADS>(sm.rank, total);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const u32 d = dig[k];
            if (d < (u32)RADIX) {
                const u32 e = w * 32u * K + (u32)k * 32u + lane;
                sm.perm[sm.rank.tstart[d] + sm.rank.cnt[w][d] + rk[k]] = (unsigned short)e;
            }
        }
        // decoupled look-back: sum predecessor tiles of the same bin until an inclusive value
        if (tid < RADIX) {
            u64 excl = 0;
            bool ok = (t != inject_tile);
            if (ok && j > 0) {
                u64 pred = (u64)t - 1;
                u64 t0 = 0;
                u32 spins = 0;
                for (;;) {
                    const u64 v = ld_relaxed_u64(&status[pred * RADIX + tid]);
                    const u32 flag = (u32)(v >> 62);
                    if (flag != 0 && (u32)((v >> 40) & LB_EPOCH_MASK) == ep) {
                        excl += v & LB_VAL_MASK;
                        if (flag == LB_INC)
                            break;
                        --pred;
                        continue;
                    }
                    if ((++spins & 31u) == 0) {
                        const u64 now = global_timer_ns();
                        if (t0 == 0) {
                            t0 = now;
                        } else if (now - t0 > wait_ns) {
                            ok = false;
                            set_error(ctrs, ST_TIMEOUT);
                            break;
                        }
                        if (ld_relaxed_u32(&ctrs->err) != 0) {
                            ok = false;
                            break;
                        }
                    }
                }
            }
            if (t != inject_tile)
                st_relaxed_u64(&status[(u64)t * RADIX + tid], lb_pack(LB_INC, ep, excl + total));
            if (!ok)
                sm.abort = 1;
            sm.goff[tid] = bases[(u64)item.row * RADIX + tid] + excl - sm.rank.tstart[tid];
        }
        if (tid == 0 && ld_relaxed_u32(&ctrs->err) != 0)
            sm.abort = 1;
        __syncthreads();
        if (!sm.abort) {
            for (u32 s = tid; s < m; s += THREADS) {
                const u32 e = sm.perm[s];
                const u64 *r = recs + (u64)e * rw;
                const u32 d = digit_of_word(r[wi], sh);
                copy_record<RW>(dst + (sm.goff[d] + s) * rw, r, rw);
            }
            if (tid == 0)
                atomicAdd(&ctrs->scatter_bytes, 2ull * m * rw * 8u);
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

// distribution variants: {threads, K, RW}
#define SCATTER_VARIANTS(X) \
    X(0, 512, 16, 1)        \
    X(1, 512, 8, 2)         \
    X(2, 512, 4, 4)         \
    X(3, 512, 4, 0)         \
    X(4, 256, 1, 0)

template <int THREADS, int K, int RW>
cudaError_t prepare_scatter(u32 rw, size_t *smem)
{
    *smem = scatter_smem_bytes<THREADS, K>(rw);
    return cudaFuncSetAttribute(scatter_kernel<THREADS, K, RW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)*smem);
}

}  // namespace

u32 scatter_tile_of(int var)
{
    switch (var) {
#define X(v, T, K, RW) \
    case v:            \
        return T * K;
        SCATTER_VARIANTS(X)
#undef X
    }
    return 0;
}

u32 hist_grid(const Shape &)
{
    return persistent_grid(hist_kernel<HIST_THREADS, HIST_UNROLL>, HIST_THREADS, 0);
}

u32 scatter_grid(const Shape &s)
{
    switch (s.scat_var) {
#define X(v, T, K, RW)                                                             \
    case v: {                                                                      \
        size_t smem = 0;                                                           \
        prepare_scatter<T, K, RW>(s.rw, &smem);                                    \
        return persistent_grid(scatter_kernel<T, K, RW>, T, smem);                 \
    }
        SCATTER_VARIANTS(X)
#undef X
    }
    return 0;
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
    hist_kernel<HIST_THREADS, HIST_UNROLL><<<grid, HIST_THREADS, 0, st>>>(in, tmp, items, tile_item, hist, orand,
                                                                         ctrs, s.tile_h, s.rw, s.key_words);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const Shape &s, u64 *in, u64 *tmp, const WorkItem *items, const u32 *tile_item,
                           const u64 *bases, u64 *status, Counters *ctrs, u32 epoch, u64 wait_ns, u32 inject_tile,
                           cudaStream_t st)
{
    const u32 grid = scatter_grid(s);
    switch (s.scat_var) {
#define X(v, T, K, RW)                                                                                   \
    case v: {                                                                                            \
        size_t smem = 0;                                                                                 \
        cudaError_t e = prepare_scatter<T, K, RW>(s.rw, &smem);                                          \
        if (e != cudaSuccess)                                                                            \
            return e;                                                                                    \
        scatter_kernel<T, K, RW><<<grid, T, smem, st>>>(in, tmp, items, tile_item, bases, status, ctrs, \
                                                        s.rw, s.key_words, epoch, wait_ns, inject_tile); \
        return cudaGetLastError();                                                                       \
    }
        SCATTER_VARIANTS(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

}  // namespace raduls
