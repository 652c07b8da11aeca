// sq_region_dispatch.cuh -- instantiate the region kernels for one precision
// and every supported region half-width m, and launch them by runtime m.
// Included by exactly one translation unit per precision with SQ_T and
// SQ_MMAX defined.
#pragma once
#include "sq_region.cuh"

namespace sq {

template <typename T>
struct RegionDispatch {
    template <int M>
    static int config(int which, size_t extra, int* blocks_per_sm, size_t* smem)
    {
        constexpr bool DB = fits_double_buffer<T, M>();
        size_t bytes = region_smem<T, M>() + extra;
        const void* fn = which == 0 ? (const void*)moments_kernel<T, M, DB> : (const void*)lanczos_kernel<T, M, DB>;
        // the limit only ever grows: contexts that share this kernel (with
        // different projector-table sizes) may launch in any order later,
        // e.g. from one captured graph
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
            cudaGetLastError();
            return SQ_ECUDA;
        }
        if ((int)bytes > fa.maxDynamicSharedSizeBytes &&
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
            cudaGetLastError();
            return SQ_EUNSUPPORTED;
        }
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, Geo<M>::NT, bytes) != cudaSuccess)
            return SQ_ECUDA;
        *blocks_per_sm = occ;
        *smem = bytes;
        return occ > 0 ? SQ_OK : SQ_EUNSUPPORTED;
    }
    template <int M>
    static int launch(int which, const RegionArgs<T>& a, size_t extra, int blocks, cudaStream_t st)
    {
        constexpr bool DB = fits_double_buffer<T, M>();
        size_t bytes = region_smem<T, M>() + extra;
        if (which == 0) moments_kernel<T, M, DB><<<blocks, Geo<M>::NT, bytes, st>>>(a);
        else lanczos_kernel<T, M, DB><<<blocks, Geo<M>::NT, bytes, st>>>(a);
        return cudaGetLastError() == cudaSuccess ? SQ_OK : SQ_ECUDA;
    }
};

}  // namespace sq

#define SQ_REGION_CASE(M, CALL)  case M: return CALL<M>
