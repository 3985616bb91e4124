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
__global__ void __launch_bounds__(THREADS, THREADS >= 1024 ? 1 : THREADS >= 512 ? 2 : 4)
block_sort_kernel(u64 *__restrict__ in, const u64 *__restrict__ tmp, const WorkItem *__restrict__ blocks,
                  Counters *__restrict__ ctrs, u32 rw_rt, u32 key_words, const u64 *__restrict__ seg_off, u32 fb)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BlockSmem<THREADS, K> &sm = *reinterpret_cast<BlockSmem<THREADS, K> *>(smem_raw);
    if (cta_failed(ctrs))
        return;
    // the on-chip list, or the items the streamed bin sort left to this kernel
    const u64 n_items = fb ? ctrs->block_fb : ctrs->block;
    u32 *const ctr = fb ? &ctrs->fb_ctr : &ctrs->tile_ctr[3];
    for (;;) {
        if (threadIdx.x == 0)
            sm.item = atomicAdd(ctr, 1u);
        __syncthreads();
        const u64 ii = sm.item;
        if (ii >= n_items)
            break;
        const WorkItem item = blocks[ii];
        block_item<THREADS, K, RW>(smem_raw, in, tmp, ctrs, rw_rt, key_words, seg_off, item);
    }
}


namespace {

// on-chip sort variants: {id, threads, K, RW}
#define BLOCK_VARIANTS(X) \
    X(0, 512, 8, 1)       \
    X(1, 512, 8, 2)       \
    X(2, 512, 4, 4)       \
    X(3, 512, 2, 0)       \
    X(4, 256, 1, 0)       \
    X(5, 1024, 8, 2)

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
                              const u64 *seg_off, cudaStream_t st, bool fb)
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
                                                           seg_off, fb ? 1u : 0u);                \
        return cudaGetLastError();                                                                  \
    }
        BLOCK_VARIANTS(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

}  // namespace raduls
