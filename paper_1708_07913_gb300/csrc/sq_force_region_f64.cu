// Region-form force kernel, FP64 (regions up to 25^3).
#include "sq_force_region_dispatch.cuh"

namespace sq {
using FR_f64 = ForceRegionDispatch<double>;

int force_region_config_f64(int m, size_t extra, int* bps, size_t* smem)
{
    switch (m) {
#define C(M) case M: return FR_f64::config<M>(extra, bps, smem);
        C(0) C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12)
#undef C
    }
    return SQ_EUNSUPPORTED;
}

int force_region_launch_f64(int m, const ForceRegionArgs<double>& f, size_t extra, int blocks, cudaStream_t st)
{
    switch (m) {
#define C(M) case M: return FR_f64::launch<M>(f, extra, blocks, st);
        C(0) C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12)
#undef C
    }
    return SQ_EUNSUPPORTED;
}
}  // namespace sq
