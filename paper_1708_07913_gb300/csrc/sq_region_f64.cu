// FP64 recurrence and Lanczos.  Regions above 25^3 do not fit one CTA's
// shared memory in FP64 and are rejected with SQ_EUNSUPPORTED.
#include "sq_region_dispatch.cuh"

namespace sq {
using D64 = RegionDispatch<double>;

int region_config_f64(int m, int which, size_t extra, int* bps, size_t* smem)
{
    switch (m) {
#define C(M) case M: return D64::config<M>(which, extra, bps, smem);
        C(0) C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12)
#undef C
    }
    return SQ_EUNSUPPORTED;
}

int region_launch_f64(int m, int which, const RegionArgs<double>& a, size_t extra, int blocks, cudaStream_t st)
{
    switch (m) {
#define C(M) case M: return D64::launch<M>(which, a, extra, blocks, st);
        C(0) C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12)
#undef C
    }
    return SQ_EUNSUPPORTED;
}
}  // namespace sq
