// sq_queue_dispatch.cuh -- instantiate the queue kernels (sq_queue.cuh) for
// one precision and every supported region half-width m, and launch them by
// runtime m.  Included by exactly one translation unit per precision.
#pragma once
#include "sq_queue.cuh"

namespace sq {

template <typename T>
struct QueueDispatch {
    template <int M>
    static const void* fn(int which)
    {
        constexpr bool DB = fits_double_buffer<T, M>();
        return which == 0 ? (const void*)moments_queue_kernel<T, M, DB> : (const void*)lanczos_queue_kernel<T, M, DB>;
    }
    // Resident CTAs per SM and dynamic shared memory with `extra` bytes after
    // the region vectors (the largest need of the group's systems).
    template <int M>
    static int config(int which, size_t extra, int* blocks_per_sm, size_t* smem)
    {
        const size_t bytes = region_smem<T, M>() + extra;
        const void* f = fn<M>(which);
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, f) != cudaSuccess) {
            cudaGetLastError();
            return SQ_ECUDA;
        }
        if ((int)bytes > fa.maxDynamicSharedSizeBytes &&
            cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
            cudaGetLastError();
            return SQ_EUNSUPPORTED;
        }
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, Geo<M>::NT, bytes) != cudaSuccess) {
            cudaGetLastError();
            return SQ_ECUDA;
        }
        *blocks_per_sm = occ;
        *smem = bytes;
        return occ > 0 ? SQ_OK : SQ_EUNSUPPORTED;
    }
    template <int M>
    static int launch(int which, const QueueArgs<T>& q, size_t extra, int blocks, cudaStream_t st)
    {
        constexpr bool DB = fits_double_buffer<T, M>();
        const size_t bytes = region_smem<T, M>() + extra;
        if (which == 0) moments_queue_kernel<T, M, DB><<<blocks, Geo<M>::NT, bytes, st>>>(q);
        else lanczos_queue_kernel<T, M, DB><<<blocks, Geo<M>::NT, bytes, st>>>(q);
        return cudaGetLastError() == cudaSuccess ? SQ_OK : SQ_ECUDA;
    }
};

}  // namespace sq
