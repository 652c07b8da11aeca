// Region-form force kernel, FP32 recurrence, D and projector sums (FP64 coefficients and contraction).
#include "sq_force_region_dispatch.cuh"

namespace sq {
using FR_f32 = ForceRegionDispatch<float>;

int force_region_config_f32(int m, size_t extra, int* bps, size_t* smem)
{
    switch (m) {
#define C(M) case M: return FR_f32::config<M>(extra, bps, smem);
        C(0) C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12) C(13) C(14) C(15)
#undef C
    }
    return SQ_EUNSUPPORTED;
}

int force_region_launch_f32(int m, const ForceRegionArgs<float>& f, size_t extra, int blocks, cudaStream_t st)
{
    switch (m) {
#define C(M) case M: return FR_f32::launch<M>(f, extra, blocks, st);
        C(0) C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12) C(13) C(14) C(15)
#undef C
    }
    return SQ_EUNSUPPORTED;
}
}  // namespace sq
