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
            u64 *__restrict__ dlight, Counters *__restrict__ ctrs, u32 tile_recs, u32 rw, u32 key_words,
            const Model *__restrict__ model)
{
    constexpr int NW = THREADS / 32;
    __shared__ u32 cnt[NW][RADIX + 1];
    __shared__ u32 light[RADIX];         // records per digit whose key is not heavy (model low digit only)
    __shared__ u64 red_or[NW], red_and[NW];
    __shared__ u32 s_tile;
    extern __shared__ u64 heavy[];       // the model's heavy keys (dynamic: HEAVY_MAX words with a model)
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    const u32 n_tiles = ctrs->grid_cur_tiles;
    const u32 n_heavy = model ? model->n_heavy : 0u;
    for (u32 i = tid; i < n_heavy; i += THREADS)
        heavy[i] = model->heavy[i];
    for (u32 i = lane; i < RADIX + 1; i += 32)
        cnt[w][i] = 0;
    if (tid < RADIX)
        light[tid] = 0;
    // Counts, OR / AND and bytes accumulate over consecutive tiles of the same
    // bin and go to global memory when the bin changes (or at the end): the
    // tiles of one big bin would otherwise all hit the same few counters.
    u32 cur_row = ~0u, cur_learned = 0;
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
                if (cur_learned == 2 && light[tid])
                    atomicAdd(&dlight[(u64)cur_row * RADIX + tid], (u64)light[tid]);
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
            if (tid < RADIX)
                light[tid] = 0;
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
        const DigitSel sel = digit_sel(item.digit, key_words);
        cur_learned = sel.learned;
        bytes += (hi - lo) * (u64)min(rw * 8u, 32u);
        for (u64 base = lo; base < hi; base += (u64)THREADS * UNROLL) {
            u64 key[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const u64 i = base + (u64)u * THREADS + tid;
                key[u] = i < hi ? __ldcs(src + i * rw + sel.word) : 0ull;
            }
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const u64 i = base + (u64)u * THREADS + tid;
                const bool valid = i < hi;
                const u32 d = valid ? digit_of_key(sel, key[u], model) : (u32)RADIX;
                if (valid) {
                    vor |= key[u];
                    vand &= key[u];
                    if (sel.learned == 2 && !is_heavy(heavy, n_heavy, key[u]))
                        atomicAdd(&light[d], 1u);
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

// -------------------------------------------------------------- distribution

template <int THREADS, int K>
struct ScatterSmem {
    RankSmem<THREADS> rank;
    u64 goff[RADIX];              // global start of each digit's run, minus its tile start
    u64 excl[RADIX];              // records of each digit in earlier tiles of the bin
    u32 total[RADIX];             // this tile's records of each digit
    u32 perm[THREADS * K];        // tile-sorted slot -> element | digit << 16
    WorkItem item;                // the item of the tile in hand (thread 0 copies it in)
    u32 item_idx;                 // its index in the item list (~0u: none yet)
    u32 tile;
    u32 abort;
};

constexpr size_t round16(size_t x) { return (x + 15) & ~(size_t)15; }

template <int THREADS, int K>
constexpr size_t scatter_smem_bytes(u32 rw)
{
    return round16(sizeof(ScatterSmem<THREADS, K>)) + ((size_t)THREADS * K * rw + 2) * 8;
}

// Decoupled look-back for digit d of tile t (index j > 0 inside its bin, whose
// first tile is `first`): sum the counts published by earlier tiles of the bin,
// up to LB of them per round trip, until one carries an inclusive value.
// Bounded by wait_ns; returns false on timeout or when another CTA reported an
// error.
template <int LB>
__device__ __forceinline__ bool lookback(const u64 *status, Counters *ctrs, u64 t, u64 first, u32 d, u32 ep,
                                         u64 wait_ns, u64 &excl)
{
    u64 pred = t - 1;
    u64 t0 = 0;
    u32 spins = 0;
    for (;;) {
        const u64 avail = pred - first + 1;
        const u32 nb = avail < (u64)LB ? (u32)avail : (u32)LB;
        u64 v[LB];
#pragma unroll
        for (int i = 0; i < LB; ++i)
            v[i] = ((u32)i < nb) ? ld_relaxed_u64(&status[(pred - i) * RADIX + d]) : 0ull;
        u32 used = nb;
        bool done = false;
#pragma unroll
        for (int i = 0; i < LB; ++i) {
            if ((u32)i >= used || done)
                continue;
            const u32 flag = (u32)(v[i] >> 62);
            if (flag == 0 || (u32)((v[i] >> 40) & LB_EPOCH_MASK) != ep) {
                used = (u32)i;
                continue;
            }
            excl += v[i] & LB_VAL_MASK;
            if (flag == LB_INC)
                done = true;
        }
        if (done)
            return true;
        pred -= used;
        if (used < nb && (++spins & 7u) == 0) {
            const u64 now = global_timer_ns();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > wait_ns) {
                set_error(ctrs, ST_TIMEOUT);
                return false;
            }
            if (ld_relaxed_u32(&ctrs->err) != 0)
                return false;
        }
    }
}

template <int THREADS, int K, int RW>
__global__ void __launch_bounds__(THREADS, THREADS >= 512 ? 2 : 4)
scatter_kernel(u64 *__restrict__ in, u64 *__restrict__ tmp, const WorkItem *__restrict__ items,
               const u32 *__restrict__ tile_item, const u64 *__restrict__ bases, u64 *__restrict__ status,
               Counters *__restrict__ ctrs, u32 rw_rt, u32 key_words, const u32 *__restrict__ epoch, u64 wait_ns,
               u32 inject_tile, const Model *__restrict__ model)
{
    constexpr u32 TILE = THREADS * K;
    static_assert(TILE <= 65536, "tile slots are 16-bit");
    static_assert(THREADS >= 2 * RADIX, "digit totals and look-back run on separate warps");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScatterSmem<THREADS, K> &sm = *reinterpret_cast<ScatterSmem<THREADS, K> *>(smem_raw);
    u64 *const recs_base = reinterpret_cast<u64 *>(smem_raw + round16(sizeof(ScatterSmem<THREADS, K>)));
    const u32 rw = RW ? (u32)RW : rw_rt;
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    const u32 n_tiles = ctrs->scatter_tiles;
    const u32 ep = *epoch & LB_EPOCH_MASK;

    if (tid == 0)
        sm.item_idx = ~0u;
    u32 err_seen = 0;  // thread 0: the error word as read when the tile was taken
    for (;;) {
        if (tid == 0) {
            // the tile and its item; consecutive tiles of a CTA mostly belong to
            // the same big bin, whose item is then already in shared memory
            const u32 t0 = atomicAdd(&ctrs->tile_ctr[1], 1u);
            sm.tile = t0;
            sm.abort = 0;
            err_seen = ld_relaxed_u32(&ctrs->err);  // read early: the answer is needed only before the writes
            if (t0 < n_tiles) {
                const u32 idx = tile_item[t0];
                if (idx != sm.item_idx) {
                    sm.item = items[idx];
                    sm.item_idx = idx;
                }
            }
        }
        __syncthreads();
        const u32 t = sm.tile;
        if (t >= n_tiles)
            break;
        const WorkItem item = sm.item;
        const u32 j = t - item.tile_base;
        const u64 lo = item.begin + (u64)j * TILE;
        const u32 m = (u32)min((u64)TILE, item.begin + item.count - lo);
        const u64 *src = (item.flags & ITEM_IN_TMP) ? tmp : in;
        u64 *dst = (item.flags & ITEM_IN_TMP) ? in : tmp;
        const DigitSel sel = digit_sel(item.digit, key_words);
        // keep shared and global 16-byte phases equal so the bulk moves as vectors
        const u32 s0 = (u32)((lo * rw) & 1u);
        u64 *recs = recs_base + s0;
        load_words<THREADS>(recs, src + lo * rw, (u64)m * rw);
        __syncthreads();

        // rank the tile's records by digit, stably (warp-contiguous layout)
        u32 dr[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const u32 e = w * 32u * K + (u32)k * 32u + lane;
            dr[k] = e < m ? digit_of(sel, recs + (u64)e * rw, model) : (u32)(RADIX - 1);
        }
        warp_rank<THREADS, K>(sm.rank, dr);
        __syncthreads();
        if (tid < RADIX) {
            u32 total = warp_offsets<THREADS>(sm.rank, tid);
            if (tid == RADIX - 1)
                total -= TILE - m;  // padding elements of a partial tile
            sm.total[tid] = total;
            // publish this tile's count of digit tid (inclusive if first tile of the bin)
            if (t != inject_tile)
                st_relaxed_u64(&status[(u64)t * RADIX + tid], lb_pack(j == 0 ? LB_INC : LB_AGG, ep, total));
        }
        __syncthreads();
        if (tid < RADIX) {
            // warps 0-7: prefix of the digit totals inside the tile
            scan_totals_256<THREADS>(sm.rank, sm.total[tid]);
        } else if (tid < 2 * RADIX) {
            // warps 8-15, meanwhile: where earlier tiles of the bin left off, per digit
            const u32 d = tid - RADIX;
            u64 excl = 0;
            bool ok = (t != inject_tile);
            if (ok && j > 0)
                ok = lookback<8>(status, ctrs, t, item.tile_base, d, ep, wait_ns, excl);
            if (t != inject_tile)
                st_relaxed_u64(&status[(u64)t * RADIX + d], lb_pack(LB_INC, ep, excl + sm.total[d]));
            if (!ok)
                sm.abort = 1;
            sm.excl[d] = excl;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const u32 e = w * 32u * K + (u32)k * 32u + lane;
            if (e < m) {
                const u32 d = dr[k] & 0xffu;
                sm.perm[sm.rank.tstart[d] + sm.rank.cnt[w][d] + (dr[k] >> 8)] = e | (d << 16);
            }
        }
        if (tid < RADIX)
            sm.goff[tid] = bases[(u64)item.row * RADIX + tid] + sm.excl[tid] - sm.rank.tstart[tid];
        if (tid == 0 && err_seen != 0)  // another CTA failed: leave the rest of the pass alone
            sm.abort = 1;
        __syncthreads();
        if (!sm.abort) {
            for (u32 s = tid; s < m; s += THREADS) {
                const u32 pe = sm.perm[s];
                copy_record<RW>(dst + (sm.goff[pe >> 16] + s) * rw, recs + (u64)(pe & 0xffffu) * rw, rw);
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
    X(4, 512, 1, 0)         \
    X(5, 512, 10, 2)        \
    X(6, 1024, 8, 2)        \
    X(7, 768, 8, 2)

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
                        u64 *hist, u64 *orand, u64 *dlight, Counters *ctrs, const Model *model, cudaStream_t st)
{
    static thread_local int cached_dev = -1;
    static thread_local u32 grid = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != cached_dev) {
        grid = hist_grid(s);
        cached_dev = dev;
    }
    const size_t dyn = model ? (size_t)HEAVY_MAX * 8 : 0;
    if (model) {
        const cudaError_t e = cudaFuncSetAttribute(hist_kernel<HIST_THREADS, HIST_UNROLL>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess)
            return e;
    }
    hist_kernel<HIST_THREADS, HIST_UNROLL><<<grid, HIST_THREADS, dyn, st>>>(in, tmp, items, tile_item, hist, orand,
                                                                           dlight, ctrs, s.tile_h, s.rw, s.key_words,
                                                                           model);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const Shape &s, u64 *in, u64 *tmp, const WorkItem *items, const u32 *tile_item,
                           const u64 *bases, u64 *status, Counters *ctrs, const u32 *epoch, u64 wait_ns,
                           u32 inject_tile, const Model *model, cudaStream_t st)
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
                                                        s.rw, s.key_words, epoch, wait_ns, inject_tile,  \
                                                        model);                                          \
        return cudaGetLastError();                                                                       \
    }
        SCATTER_VARIANTS(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

}  // namespace raduls
