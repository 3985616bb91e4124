// blocksort.cu -- on-chip stable sort of small bins (Sec. 3.4-3.5).
//
// The paper finishes bins that fit in cache with an unbuffered counting
// split and tiny bins with comparison sorts (Sec. 3.4, 3.5).  Its comparison
// sorts (introsort, Shell sort) are not stable; the sort here is defined as
// stable, so a run of small bins is instead loaded into one CTA's shared
// memory and sorted there by LSD counting passes (Sec. 1) over the key digits
// that actually vary inside the run -- digits on which all its records agree
// are found from the OR and AND of the key words and skipped.  Each pass is
// the same stable warp multi-split ranking as the distribution kernel.  The
// records themselves stay in place in shared memory: only (key word, record
// index) pairs move between passes, and the final order is written to `in`
// with coalesced stores.
#include "kernels.h"

namespace raduls {

template <int THREADS, int K>
struct BlockSmem {
    RankSmem<THREADS> rank;
    u64 xkey[THREADS * K];             // exchange buffer: key words
    unsigned short xidx[THREADS * K];  // exchange buffer: record indices
    u64 red_or[THREADS / 32];
    u64 red_and[THREADS / 32];
    u32 item;
};

constexpr size_t round16b(size_t x) { return (x + 15) & ~(size_t)15; }

template <int THREADS, int K>
constexpr size_t block_smem_bytes(u32 rw)
{
    return round16b(sizeof(BlockSmem<THREADS, K>)) + ((size_t)THREADS * K * rw + 2) * 8;
}

template <int THREADS, int K, int RW>
__global__ void __launch_bounds__(THREADS)
block_sort_kernel(u64 *__restrict__ in, const u64 *__restrict__ tmp, const WorkItem *__restrict__ blocks,
                  Counters *__restrict__ ctrs, u32 rw_rt, u32 key_words)
{
    constexpr u32 CAP = THREADS * K;
    constexpr int NW = THREADS / 32;
    static_assert(CAP <= 65536, "record indices are 16-bit");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BlockSmem<THREADS, K> &sm = *reinterpret_cast<BlockSmem<THREADS, K> *>(smem_raw);
    u64 *const recs_base = reinterpret_cast<u64 *>(smem_raw + round16b(sizeof(BlockSmem<THREADS, K>)));
    const u32 rw = RW ? (u32)RW : rw_rt;
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    const u64 n_items = ctrs->block;

    for (;;) {
        if (tid == 0)
            sm.item = atomicAdd(&ctrs->tile_ctr[3], 1u);
        __syncthreads();
        const u64 ii = sm.item;
        if (ii >= n_items)
            break;
        const WorkItem item = blocks[ii];
        if (item.count > CAP) {  // planner bug guard: never overrun shared memory
            if (tid == 0)
                set_error(ctrs, ST_INTERNAL);
            __syncthreads();
            continue;
        }
        const u32 m = (u32)item.count;
        const u64 *src = (item.flags & ITEM_IN_TMP) ? tmp : in;
        const u32 s0 = (u32)((item.begin * rw) & 1u);
        u64 *recs = recs_base + s0;
        load_words<THREADS>(recs, src + item.begin * rw, (u64)m * rw);
        __syncthreads();

        // element slots, warp-contiguous: slot k of lane l in warp w is position w*32K + 32k + l
        u32 id[K];
#pragma unroll
        for (int k = 0; k < K; ++k)
            id[k] = w * 32u * K + (u32)k * 32u + lane;

        const u32 top_word = key_words - 1u - item.digit / 8u;
        for (int wi = (int)key_words - 1; wi >= (int)top_word && m > 1; --wi) {
            // which bytes of this key word vary inside the run
            u64 vor = 0, vand = ~0ull;
            for (u32 e = tid; e < m; e += THREADS) {
                const u64 v = recs[(u64)e * rw + wi];
                vor |= v;
                vand &= v;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                vor |= __shfl_xor_sync(FULL_MASK, vor, o);
                vand &= __shfl_xor_sync(FULL_MASK, vand, o);
            }
            if (lane == 0) {
                sm.red_or[w] = vor;
                sm.red_and[w] = vand;
            }
            __syncthreads();
            u64 diff = 0;
            {
                u64 o2 = 0, a2 = ~0ull;
#pragma unroll
                for (int i = 0; i < NW; ++i) {
                    o2 |= sm.red_or[i];
                    a2 &= sm.red_and[i];
                }
                diff = o2 ^ a2;
            }
            if (wi == (int)top_word && (item.digit % 8u) != 7u)
                diff &= (2ull << (8u * (item.digit % 8u) + 7u)) - 1ull;  // bytes above the run's digit are shared
            __syncthreads();
            if (diff == 0)
                continue;
            u64 key[K];
#pragma unroll
            for (int k = 0; k < K; ++k)
                key[k] = id[k] < m ? recs[(u64)id[k] * rw + wi] : 0ull;
            for (u32 b = 0; b < 8u; ++b) {
                if (((diff >> (8u * b)) & 0xffu) == 0)
                    continue;
                u32 dig[K], rk[K];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const u32 pos = w * 32u * K + (u32)k * 32u + lane;
                    dig[k] = pos < m ? digit_of_word(key[k], 8u * b) : (u32)RADIX;
                }
                warp_rank<THREADS, K>(sm.rank, dig, rk);
                __syncthreads();
                u32 total = 0;
                if (tid < RADIX)
                    total = warp_offsets<THREADS>(sm.rank, tid);
                scan_totals<THREADS>(sm.rank, total);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const u32 d = dig[k];
                    if (d < (u32)RADIX) {
                        const u32 np = sm.rank.tstart[d] + sm.rank.cnt[w][d] + rk[k];
                        sm.xkey[np] = key[k];
                        sm.xidx[np] = (unsigned short)id[k];
                    }
                }
                __syncthreads();
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const u32 pos = w * 32u * K + (u32)k * 32u + lane;
                    if (pos < m) {
                        key[k] = sm.xkey[pos];
                        id[k] = sm.xidx[pos];
                    }
                }
                __syncthreads();
            }
        }
        // write the run in its final order
        u64 *out = in + item.begin * rw;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const u32 pos = w * 32u * K + (u32)k * 32u + lane;
            if (pos < m)
                copy_record<RW == 2 || RW == 4 ? 0 : RW>(out + (u64)pos * rw, recs + (u64)id[k] * rw, rw);
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
                              cudaStream_t st)
{
    const u32 grid = block_grid(s);
    switch (s.block_var) {
#define X(v, T, K, RW)                                                                              \
    case v: {                                                                                       \
        size_t smem = 0;                                                                            \
        cudaError_t e = prepare_block<T, K, RW>(s.rw, &smem);                                       \
        if (e != cudaSuccess)                                                                       \
            return e;                                                                               \
        block_sort_kernel<T, K, RW><<<grid, T, smem, st>>>(in, tmp, blocks, ctrs, s.rw, s.key_words); \
        return cudaGetLastError();                                                                  \
    }
        BLOCK_VARIANTS(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

}  // namespace raduls
