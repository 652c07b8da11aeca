// Queue kernels, FP64 (regions up to 25^3, as for the single-system kernels).
#include "sq_queue_dispatch.cuh"

namespace sq {
using Q64 = QueueDispatch<double>;

int queue_config_f64(int m, int which, size_t extra, int* bps, size_t* smem)
{
    switch (m) {
#define C(M) case M: return Q64::config<M>(which, extra, bps, smem);
        C(0) C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12)
#undef C
    }
    return SQ_EUNSUPPORTED;
}

int queue_launch_f64(int m, int which, const QueueArgs<double>& q, size_t extra, int blocks, cudaStream_t st)
{
    switch (m) {
#define C(M) case M: return Q64::launch<M>(which, q, extra, blocks, st);
        C(0) C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12)
#undef C
    }
    return SQ_EUNSUPPORTED;
}
}  // namespace sq
