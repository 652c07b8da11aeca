// sq_force_region_dispatch.cuh -- instantiate the region-form force kernel
// (sq_force_region.cuh) for one precision and every supported region
// half-width m, and launch it by runtime m.  Included by exactly one
// translation unit per precision.
#pragma once
#include "sq_force_region.cuh"

namespace sq {

template <typename T>
struct ForceRegionDispatch {
    // Resident CTAs per SM and dynamic shared memory with `extra` bytes after
    // the region vectors.
    template <int M>
    static int config(size_t extra, int* blocks_per_sm, size_t* smem)
    {
        constexpr bool DB = fits_double_buffer<T, M>();
        const size_t bytes = region_smem<T, M>() + extra;
        const void* f = (const void*)force_region_kernel<T, M, DB>;
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
    static int launch(const ForceRegionArgs<T>& f, size_t extra, int blocks, cudaStream_t st)
    {
        constexpr bool DB = fits_double_buffer<T, M>();
        force_region_kernel<T, M, DB><<<blocks, Geo<M>::NT, region_smem<T, M>() + extra, st>>>(f);
        return cudaGetLastError() == cudaSuccess ? SQ_OK : SQ_ECUDA;
    }
};

}  // namespace sq
