// sq_cluster_dispatch.cuh -- instantiate the FP32 cluster region kernels
// (sq_cluster.cuh) for a range of region half-widths and launch them by
// runtime m.  Each m has one cluster size, the smallest of 2, 4, 8 whose
// slab, projector entries and candidate tables fit a CTA's shared memory for
// the candidate counts of FCC-Al-like atom densities; a context whose
// candidates do not fit uses the single-CTA kernels.  Included by the two
// translation units sq_cluster_lo.cu (m = 3..9) and sq_cluster_hi.cu
// (m = 10..15), which compile in parallel.
#pragma once
#include "sq_cluster.cuh"

namespace sq {

// cluster size per region half-width m (0: the single-CTA kernels)
__host__ __device__ constexpr inline int cluster_size_for(int m) { return m < 3 ? 0 : (m <= 8 ? 2 : (m <= 14 ? 4 : 8)); }

namespace {

template <int M>
struct ClDispatch {
    static constexpr int NC = cluster_size_for(M) > 0 ? cluster_size_for(M) : 2;
    using G = CGeo<M, NC>;
    static const void* fn(int which)
    {
        return which == 0 ? (const void*)cl_moments_kernel<M, NC> : (const void*)cl_lanczos_kernel<M, NC>;
    }
    static int config(int which, int ccap, int npl, int* clusters, size_t* smem)
    {
        const size_t bytes = cl_layout(G::S, G::NZMAX, ccap, which == 0 ? npl : 0).total;
        const void* f = fn(which);
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, f) != cudaSuccess) {
            cudaGetLastError();
            return SQ_ECUDA;
        }
        int dev = 0, optin = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
            cudaGetLastError();
            return SQ_ECUDA;
        }
        if (bytes + fa.sharedSizeBytes > (size_t)optin) return SQ_EUNSUPPORTED;
        if ((int)bytes > fa.maxDynamicSharedSizeBytes &&
            cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
            cudaGetLastError();
            return SQ_EUNSUPPORTED;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(NC, 1, 1);
        cfg.blockDim = dim3(G::NT, 1, 1);
        cfg.dynamicSmemBytes = bytes;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, f, &cfg) != cudaSuccess) {
            cudaGetLastError();
            return SQ_ECUDA;
        }
        if (n < 1) return SQ_EUNSUPPORTED;
        *clusters = n;
        *smem = bytes;
        return SQ_OK;
    }
    static int launch(int which, const RegionArgs<float>& a, int clusters, size_t smem, cudaStream_t st)
    {
        if (which == 0) cl_moments_kernel<M, NC><<<clusters * NC, G::NT, smem, st>>>(a);
        else cl_lanczos_kernel<M, NC><<<clusters * NC, G::NT, smem, st>>>(a);
        return cudaGetLastError() == cudaSuccess ? SQ_OK : SQ_ECUDA;
    }
};

}  // namespace

}  // namespace sq
