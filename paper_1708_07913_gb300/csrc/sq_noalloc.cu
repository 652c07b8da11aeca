// sq_noalloc.cu -- sq_density_energy_noalloc: the density / band energy /
// entropy step for callers that must not allocate device memory.
//
// Some host programs own all device memory themselves -- an application that
// reserves the GPU's memory up front for its own pool, or one whose memory
// budget is settled at start-up -- and do not let a library call cudaMalloc.
// For them this entry point allocates nothing: the caller passes inputs and
// outputs, the quadrature weights are recomputed per node on the fly instead
// of being stored, and the few bytes of scratch the reduction needs
// (per-block partial sums, a completion counter, the three totals) live in
// one file-scope __device__ array of fixed size.
//
// The array's name is only a host-side stand-in in host code; its device
// address is obtained once per device with cudaGetSymbolAddress (the first
// call on each device does this, with that device current) and passed to the
// kernel.  Every call shares the array and it keeps the last call's contents:
// each call clears the counter it depends on before use, and calls whose
// execution overlaps on the GPU (different streams, or threads) race on it.
#include <math.h>
#include <mutex>

#include "sq_internal.cuh"

namespace {

constexpr int NA_MAX_BLOCKS = 2048;       // grid size cap of the reduction
constexpr int NA_THREADS = 256;
constexpr int NA_MAX_DEVICES = 64;

// partials[3 * NA_MAX_BLOCKS] | counter (as 8 bytes) | totals[3]
constexpr size_t NA_SCRATCH_BYTES = sizeof(double) * (3 * NA_MAX_BLOCKS + 1 + 3);
static __device__ __align__(256) unsigned char g_na_scratch[NA_SCRATCH_BYTES];

std::mutex g_na_mutex;
void* g_na_ptr[NA_MAX_DEVICES] = {nullptr};

__global__ void density_noalloc_kernel(const double* __restrict__ mom, const double* __restrict__ chi,
                                       const double* __restrict__ zeta, long long Nd, int K, double mu,
                                       double kT, double h, double* __restrict__ rho, double* scratch)
{
    extern __shared__ double na_sh[];                 // [K] nodes x_k, then [K][K] T_j(x_k) when it fits
    double* xk = na_sh;
    double* Ttab = na_sh + K;
    const bool table = (size_t)(K + K * K) * sizeof(double) <= 96 * 1024;
    double* partials = scratch;
    unsigned* counter = reinterpret_cast<unsigned*>(scratch + 3 * NA_MAX_BLOCKS);
    double* totals = scratch + 3 * NA_MAX_BLOCKS + 1;
    __shared__ double red[3][32];
    __shared__ bool last;

    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double x = cos(M_PI * (k + 0.5) / K);
        xk[k] = x;
        if (table) {
            double tm = 1.0, t = x;
            Ttab[k] = 1.0;
            if (K > 1) Ttab[K + k] = x;
            for (int j = 2; j < K; ++j) {
                double tn = 2.0 * x * t - tm;
                tm = t;
                t = tn;
                Ttab[j * K + k] = t;
            }
        }
    }
    __syncthreads();
    const double h3 = h * h * h;
    double acc[3] = {0.0, 0.0, 0.0};
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < Nd;
         q += (long long)gridDim.x * blockDim.x) {
        const double* r = mom + q * K;
        const double c = chi[q], z = zeta[q];
        double rq = 0.0, eb = 0.0, es = 0.0;
        for (int k = 0; k < K; ++k) {
            // weight W_qk = (2/K)(rho^0/2 + sum_j rho^j T_j(x_k)), recomputed here
            double s = 0.5 * r[0];
            if (table) {
                for (int j = 1; j < K; ++j) s += r[j] * Ttab[j * K + k];
            } else {
                double tm = 1.0, t = xk[k];
                for (int j = 1; j < K; ++j) {
                    s += r[j] * t;
                    double tn = 2.0 * xk[k] * t - tm;
                    tm = t;
                    t = tn;
                }
            }
            const double wk = 2.0 / K * s;
            const double E = c + z * xk[k];
            const double t = (E - mu) / kT;
            if (t > 40.0) continue;
            if (t < -40.0) {
                rq += wk;
                eb += 2.0 * wk * E;
                continue;
            }
            const double g = 1.0 / (1.0 + exp(t));
            const double gm = 1.0 / (1.0 + exp(-t));
            rq += wk * g;
            eb += 2.0 * wk * E * g;
            double sf = 0.0;
            if (g > 0.0) sf += g * log(g);
            if (gm > 0.0) sf += gm * log(gm);
            es += 2.0 * kT * wk * sf;
        }
        const double rho_q = 2.0 / h3 * rq;
        rho[q] = rho_q;
        acc[0] += eb;
        acc[1] += es;
        acc[2] += h3 * rho_q;
    }
    // fixed-order block reduction, then the last block adds block partials in order
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        double v = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[i][w] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < 3; ++i) {
            double t = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[i][k];
            partials[3 * blockIdx.x + i] = t;
        }
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) {
            s0 += ((volatile double*)partials)[3 * b + 0];
            s1 += ((volatile double*)partials)[3 * b + 1];
            s2 += ((volatile double*)partials)[3 * b + 2];
        }
        totals[0] = s0;
        totals[1] = s1;
        totals[2] = s2;
        *counter = 0;
    }
}

bool is_device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
int scratch_address(double** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SQ_ECUDA;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return SQ_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SQ_ECUDA;
        }
        g_na_ptr[dev] = p;
    }
    *out = static_cast<double*>(g_na_ptr[dev]);
    return SQ_OK;
}

}  // namespace

extern "C" int sq_density_energy_noalloc(int n1, int n2, int n3, double h, int npl, const double* moments,
                                         const double* chi, const double* zeta, double mu, double kT,
                                         double* rho, double* e_band_host, double* e_ent_host,
                                         double* n_elec_host, void* cuda_stream)
{
    if (n1 < 1 || n2 < 1 || n3 < 1 || (long long)n1 * n2 * n3 > (1LL << 31)) return SQ_EINVAL;
    if (!(h > 0.0) || !isfinite(h) || !(kT > 0.0) || !isfinite(kT) || !isfinite(mu)) return SQ_EINVAL;
    if (npl < 4 || npl > sq::MAX_NPL || npl % 4 != 0) return SQ_EINVAL;
    if (!is_device_ptr(moments) || !is_device_ptr(chi) || !is_device_ptr(zeta) || !is_device_ptr(rho))
        return SQ_EINVAL;
    double* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SQ_ECUDA;
    const long long Nd = (long long)n1 * n2 * n3;
    const int K = npl + 1;
    long long want = (Nd + NA_THREADS - 1) / NA_THREADS;
    int blocks = (int)(want < 4LL * sms ? want : 4LL * sms);
    if (blocks > NA_MAX_BLOCKS) blocks = NA_MAX_BLOCKS;
    const size_t tab = (size_t)(K + K * K) * sizeof(double);
    const size_t smem = tab <= 96 * 1024 ? tab : (size_t)K * sizeof(double);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(density_noalloc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return SQ_ECUDA;
    // the completion counter must start at zero (an earlier call may have been cut short)
    if (cudaMemsetAsync(scratch + 3 * NA_MAX_BLOCKS, 0, sizeof(double), st) != cudaSuccess) return SQ_ECUDA;
    density_noalloc_kernel<<<blocks, NA_THREADS, smem, st>>>(moments, chi, zeta, Nd, K, mu, kT, h, rho, scratch);
    if (cudaGetLastError() != cudaSuccess) return SQ_ECUDA;
    double totals[3];
    if (cudaMemcpyAsync(totals, scratch + 3 * NA_MAX_BLOCKS + 1, sizeof(totals), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SQ_ECUDA;
    if (e_band_host) *e_band_host = totals[0];
    if (e_ent_host) *e_ent_host = totals[1];
    if (n_elec_host) *n_elec_host = totals[2];
    return SQ_OK;
}
