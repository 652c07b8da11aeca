// Queue kernels, FP32 recurrence / Lanczos vectors (moments and Lanczos
// coefficients in FP64).
#include "sq_queue_dispatch.cuh"

namespace sq {
using Q32 = QueueDispatch<float>;

int queue_config_f32(int m, int which, size_t extra, int* bps, size_t* smem)
{
    switch (m) {
#define C(M) case M: return Q32::config<M>(which, extra, bps, smem);
        C(0) C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12) C(13) C(14) C(15)
#undef C
    }
    return SQ_EUNSUPPORTED;
}

int queue_launch_f32(int m, int which, const QueueArgs<float>& q, size_t extra, int blocks, cudaStream_t st)
{
    switch (m) {
#define C(M) case M: return Q32::launch<M>(which, q, extra, blocks, st);
        C(0) C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12) C(13) C(14) C(15)
#undef C
    }
    return SQ_EUNSUPPORTED;
}
}  // namespace sq
