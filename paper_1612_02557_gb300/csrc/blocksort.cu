// blocksort.cu -- on-chip stable sort of small bins (Sec. 3.4-3.5).
//
// Work items come in two kinds:
//   * a RUN: consecutive small sub-bins (at most WARP_MAX records each) of one
//     parent bin, split on the parent's digit, or consecutive small arrays of
//     a batched call.  The run is loaded into one CTA's shared memory with
//     coalesced loads, its sub-bin boundaries are read off a histogram of that
//     digit (or the array offsets), and every sub-bin is then sorted by one
//     warp on its own, without block-wide barriers (warp_sort_bin);
//   * a single bin of up to CAP records (or a whole small input), sorted by
//     the whole CTA (block_path).
// The sorts themselves are in onchip.cuh.
#include "onchip.cuh"

namespace raduls {

// ------------------------------------------------------------------ kernel

template <int THREADS, int K, int RW>
__global__ void __launch_bounds__(THREADS, THREADS >= 512 ? 2 : 4)
block_sort_kernel(u64 *__restrict__ in, const u64 *__restrict__ tmp, const WorkItem *__restrict__ blocks,
                  Counters *__restrict__ ctrs, u32 rw_rt, u32 key_words, const u64 *__restrict__ seg_off)
{
    constexpr u32 CAP = THREADS * K;
    constexpr int NW = THREADS / 32;
    static_assert(CAP <= 65536 && CAP < (1u << 23), "record indices are 16-bit");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BlockSmem<THREADS, K> &sm = *reinterpret_cast<BlockSmem<THREADS, K> *>(smem_raw);
    u64 *const recs_base = reinterpret_cast<u64 *>(smem_raw + round16b(sizeof(BlockSmem<THREADS, K>)));
    const u32 rw = RW ? (u32)RW : rw_rt;
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    const u64 n_items = ctrs->block;

    for (;;) {
        if (tid == 0) {
            sm.item = atomicAdd(&ctrs->tile_ctr[3], 1u);
            sm.big_group = 0;
        }
        __syncthreads();
        const u64 ii = sm.item;
        if (ii >= n_items)
            break;
        const WorkItem item = blocks[ii];
        if (item.count > CAP) {  // planner guard: never overrun shared memory
            if (tid == 0)
                set_error(ctrs, ST_INTERNAL);
            __syncthreads();
            continue;
        }
        const u32 m = (u32)item.count;
        const u64 *src = (item.flags & ITEM_IN_TMP) ? tmp : in;
        const u32 s0 = (u32)((item.begin * rw) & 1u);
        u64 *recs = recs_base + s0;
        u64 *out = in + item.begin * rw;
        if (tid < RADIX)
            sm.chist[tid] = 0;
        load_words<THREADS>(recs, src + item.begin * rw, (u64)m * rw);
        __syncthreads();

        if (item.flags & ITEM_RUN) {
            // sub-bin boundaries: a run of one parent's sub-bins is grouped by the
            // parent's split digit p; a run of arrays takes them from the offsets
            const bool segs = (item.flags & ITEM_SEG) != 0;
            const u32 p = item.digit;
            const u32 p_word = segs ? 0u : key_words - 1u - p / 8u;
            const u32 p_byte = segs ? 8u : p % 8u;  // bytes of p_word below the split digit that may vary
            if (!segs) {
                for (u32 e0 = w * 32u; e0 < m; e0 += THREADS) {
                    const u32 e = e0 + lane;
                    const u32 d = e < m ? digit_of_word(recs[(u64)e * rw + p_word], 8u * p_byte) : (u32)RADIX;
                    const u32 d0 = __shfl_sync(FULL_MASK, d, 0);
                    const u32 same = __ballot_sync(FULL_MASK, d == d0);
                    if (same == FULL_MASK) {
                        if (lane == 0 && d0 < (u32)RADIX)
                            atomicAdd(&sm.chist[d0], 32u);
                    } else if (d < (u32)RADIX) {
                        atomicAdd(&sm.chist[d], 1u);
                    }
                }
            }
            // key digits below p that vary anywhere in the run
            varying_digits_below<THREADS, K>(sm, recs, rw, m, p_word, p_byte, key_words);
            if (segs) {
                // arrays [tile_base, tile_base + row) of the offset table (row <= 256)
                const u64 o0 = seg_off[item.tile_base];
                if (tid < item.row) {
                    const u64 a = seg_off[item.tile_base + tid], b = seg_off[item.tile_base + tid + 1];
                    sm.cbeg[tid] = (unsigned short)(a - o0);
                    sm.ccnt[tid] = (unsigned short)(b - a);
                }
                if (tid == 0)
                    sm.nchild = item.row;
                __syncthreads();
            } else {
                u32 packed = 0;
                if (tid < RADIX)
                    packed = (sm.chist[tid] << 9) | (sm.chist[tid] ? 1u : 0u);
                scan_totals<THREADS>(sm.rank, packed);
                if (tid < RADIX && sm.chist[tid]) {
                    const u32 ex = sm.rank.tstart[tid];
                    const u32 slot = ex & 511u;
                    sm.cbeg[slot] = (unsigned short)(ex >> 9);
                    sm.ccnt[slot] = (unsigned short)sm.chist[tid];
                }
                if (tid == RADIX - 1)
                    sm.nchild = ((sm.rank.tstart[tid] + packed) & 511u);
                __syncthreads();
            }
            const u32 nchild = sm.nchild, nv = sm.nv;
            for (u32 ci = w; ci < nchild; ci += NW) {
                const u32 c = sm.ccnt[ci];
                if (c > WARP_MAX) {
                    if (lane == 0)
                        set_error(ctrs, ST_INTERNAL);
                    continue;
                }
                warp_sort_bin<RW>(sm.rank.cnt[w], sm.xidx, sm.xcode, sm.xnew, recs, rw, sm.cbeg[ci], c, sm.vword,
                                  sm.vshift, nv, p_word, key_words, out);
            }
        } else {
            u32 id[K];
            const u32 kv = (m + THREADS - 1) / THREADS;
            block_path<THREADS, K>(sm, recs, rw, m, kv, item.digit, key_words, id);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const u32 pos = w * 32u * kv + (u32)k * 32u + lane;
                if ((u32)k < kv && pos < m)
                    copy_record<RW>(out + (u64)pos * rw, recs + (u64)id[k] * rw, rw);
            }
        }
        if (tid == 0)
            atomicAdd(&ctrs->block_bytes, 2ull * m * rw * 8u);
        __syncthreads();
    }
}

namespace {

// on-chip sort variants: {id, threads, K, RW}
#define BLOCK_VARIANTS(X) \
    X(0, 512, 8, 1)       \
    X(1, 512, 8, 2)       \
    X(2, 512, 4, 4)       \
    X(3, 512, 2, 0)       \
    X(4, 256, 1, 0)

template <int THREADS, int K, int RW>
cudaError_t prepare_block(u32 rw, size_t *smem)
{
    *smem = block_smem_bytes<THREADS, K>(rw);
    return cudaFuncSetAttribute(block_sort_kernel<THREADS, K, RW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)*smem);
}

}  // namespace

u32 block_cap_of(int var)
{
    switch (var) {
#define X(v, T, K, RW) \
    case v:            \
        return T * K;
        BLOCK_VARIANTS(X)
#undef X
    }
    return 0;
}

u32 block_grid(const Shape &s)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    switch (s.block_var) {
#define X(v, T, K, RW)                                                                           \
    case v: {                                                                                    \
        size_t smem = 0;                                                                         \
        prepare_block<T, K, RW>(s.rw, &smem);                                                    \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, block_sort_kernel<T, K, RW>, T, smem); \
        break;                                                                                   \
    }
        BLOCK_VARIANTS(X)
#undef X
    }
    return (u32)(sms * (per_sm < 1 ? 1 : per_sm));
}

cudaError_t launch_block_sort(const Shape &s, u64 *in, const u64 *tmp, const WorkItem *blocks, Counters *ctrs,
                              const u64 *seg_off, cudaStream_t st)
{
    const u32 grid = block_grid(s);
    switch (s.block_var) {
#define X(v, T, K, RW)                                                                              \
    case v: {                                                                                       \
        size_t smem = 0;                                                                            \
        cudaError_t e = prepare_block<T, K, RW>(s.rw, &smem);                                       \
        if (e != cudaSuccess)                                                                       \
            return e;                                                                               \
        block_sort_kernel<T, K, RW><<<grid, T, smem, st>>>(in, tmp, blocks, ctrs, s.rw, s.key_words,  \
                                                           seg_off);                              \
        return cudaGetLastError();                                                                  \
    }
        BLOCK_VARIANTS(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

}  // namespace raduls
