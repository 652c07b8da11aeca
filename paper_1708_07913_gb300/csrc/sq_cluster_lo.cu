// sq_cluster_lo.cu -- FP32 cluster region kernels for m = 3..9 (see sq_cluster_dispatch.cuh).
#include "sq_cluster_dispatch.cuh"

namespace sq {

int cluster_nc(int m) { return (m >= 0 && m <= MAX_M) ? cluster_size_for(m) : 0; }

int cluster_config_f32_lo(int m, int which, int ccap, int npl, int* clusters, size_t* smem)
{
    switch (m) {
#define C(M) case M: return ClDispatch<M>::config(which, ccap, npl, clusters, smem);
        C(3) C(4) C(5) C(6) C(7) C(8) C(9)
#undef C
    }
    return SQ_EUNSUPPORTED;
}

int cluster_launch_f32_lo(int m, int which, const RegionArgs<float>& a, int clusters, size_t smem, cudaStream_t st)
{
    switch (m) {
#define C(M) case M: return ClDispatch<M>::launch(which, a, clusters, smem, st);
        C(3) C(4) C(5) C(6) C(7) C(8) C(9)
#undef C
    }
    return SQ_EUNSUPPORTED;
}
}  // namespace sq
