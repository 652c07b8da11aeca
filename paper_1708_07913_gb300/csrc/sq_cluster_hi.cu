// sq_cluster_hi.cu -- FP32 cluster region kernels for m = 10..15 (see sq_cluster_dispatch.cuh).
#include "sq_cluster_dispatch.cuh"

namespace sq {

int cluster_config_f32_hi(int m, int which, int ccap, int npl, int* clusters, size_t* smem)
{
    switch (m) {
#define C(M) case M: return ClDispatch<M>::config(which, ccap, npl, clusters, smem);
        C(10) C(11) C(12) C(13) C(14) C(15)
#undef C
    }
    return SQ_EUNSUPPORTED;
}

int cluster_launch_f32_hi(int m, int which, const RegionArgs<float>& a, int clusters, size_t smem, cudaStream_t st)
{
    switch (m) {
#define C(M) case M: return ClDispatch<M>::launch(which, a, clusters, smem, st);
        C(10) C(11) C(12) C(13) C(14) C(15)
#undef C
    }
    return SQ_EUNSUPPORTED;
}
}  // namespace sq
