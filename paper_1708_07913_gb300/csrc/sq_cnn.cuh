// sq_cnn.cuh -- kernels of the learned SCF warm start: a 3-D convolutional
// network on the periodic grid that maps the 9^3 patch of the effective
// potential around each node to the node's density,
//
//   x0 = (V - v_shift) / v_scale
//   a1 = silu(conv5(x0; W1) + b1)      1 -> 32 channels, 5^3 kernel
//   a2 = silu(conv3(a1; W2) + b2)      32 -> 32 channels, 3^3 kernel
//   y  = conv3(a2; W3) + b3            32 -> 1 channel, 3^3 kernel
//   rho = rho_scale softplus(y)
//
// conv_k(x; W)[o](p) = sum_i sum_{d in [-r,r]^3} W[d][i][o] x[i](p + d)
// (periodic cross-correlation), its two adjoints for training, the loss
// mean((rho - rho_ref)^2)/rho_scale^2 and Adam.  Weights and activations
// are stored in T (bfloat16 or float); every sum accumulates in FP32;
// biases, pre-activations, gradients, master weights and Adam moments are
// FP32.  Layouts: activations node-major, channel fastest ([p][c]);
// weights tap-major ([d][i][o], d = (dz+r) k^2 + (dy+r) k + (dx+r)).
//
// CUDA cores, one thread per (node, channel) for the data passes; weight
// gradients are per-chunk partial sums added in chunk order, so everything
// repeats bit for bit.  Block barriers and plain loads/stores only.
#pragma once
#include <stdint.h>
#include <string.h>
#include <cuda_runtime.h>

namespace sq {

constexpr int CNN_C = 32;            // hidden channels
constexpr int CNN_NT = 256;          // threads per block
constexpr int CNN_CHUNK = 512;       // nodes per partial sum of a weight gradient

// bfloat16 storage (round to nearest even from FP32; NaN stays NaN)
struct Bf16 {
    uint16_t u;
};

__host__ __device__ inline float bits_f(uint32_t b)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float f;
    memcpy(&f, &b, 4);
    return f;
#endif
}

__host__ __device__ inline uint32_t f_bits(float f)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
#endif
}

__host__ __device__ inline float ldv(float v) { return v; }
__host__ __device__ inline float ldv(Bf16 v) { return bits_f((uint32_t)v.u << 16); }
__host__ __device__ inline void stv(float& d, float v) { d = v; }
__host__ __device__ inline void stv(Bf16& d, float v)
{
    uint32_t u = f_bits(v);
    if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x7fffffu)) {
        d.u = (uint16_t)((u >> 16) | 0x40u);
        return;
    }
    u += 0x7fffu + ((u >> 16) & 1u);
    d.u = (uint16_t)(u >> 16);
}

__device__ inline float cnn_sigmoid(float z) { return 1.0f / (1.0f + expf(-z)); }
__device__ inline float cnn_silu(float z) { return z * cnn_sigmoid(z); }
__device__ inline float cnn_silu_grad(float z)
{
    const float s = cnn_sigmoid(z);
    return s * (1.0f + z * (1.0f - s));
}

__device__ inline int cnn_wrap(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

struct CnnGrid {
    int n1, n2, n3;
    long long N;
};

// node index of p + d on the periodic grid
__device__ inline long long cnn_nb(const CnnGrid& g, int i, int j, int k, int dx, int dy, int dz)
{
    return (long long)cnn_wrap(i + dx, g.n1) +
           (long long)g.n1 * ((long long)cnn_wrap(j + dy, g.n2) + (long long)g.n2 * cnn_wrap(k + dz, g.n3));
}

__device__ inline void cnn_ijk(const CnnGrid& g, long long p, int& i, int& j, int& k)
{
    i = (int)(p % g.n1);
    j = (int)((p / g.n1) % g.n2);
    k = (int)(p / ((long long)g.n1 * g.n2));
}

// x0 = (V - shift) / scale, stored in T
template <typename T>
__global__ void cnn_input_kernel(CnnGrid g, const double* __restrict__ V, double shift, double scale, T* __restrict__ x0)
{
    for (long long p = blockIdx.x * (long long)CNN_NT + threadIdx.x; p < g.N; p += (long long)gridDim.x * CNN_NT)
        stv(x0[p], (float)((V[p] - shift) / scale));
}

// z[p][o] = b[o] + sum_d sum_i W[d][i][o] x[p + d][i]; a = silu(z) in T.
// CI input channels (1 or 32), K kernel edge, C outputs.
template <typename T, int CI, int K>
__global__ void __launch_bounds__(CNN_NT) cnn_conv_fwd_kernel(CnnGrid g, const T* __restrict__ x,
                                                              const T* __restrict__ W, const float* __restrict__ b,
                                                              float* __restrict__ z, T* __restrict__ a)
{
    constexpr int R = (K - 1) / 2;
    for (long long t = blockIdx.x * (long long)CNN_NT + threadIdx.x; t < g.N * CNN_C;
         t += (long long)gridDim.x * CNN_NT) {
        const long long p = t / CNN_C;
        const int o = (int)(t % CNN_C);
        int i, j, k;
        cnn_ijk(g, p, i, j, k);
        float acc = 0.0f;
        int d = 0;
        for (int dz = -R; dz <= R; ++dz)
            for (int dy = -R; dy <= R; ++dy)
                for (int dx = -R; dx <= R; ++dx, ++d) {
                    const T* xs = x + cnn_nb(g, i, j, k, dx, dy, dz) * CI;
                    const T* w = W + ((size_t)d * CI) * CNN_C + o;
                    for (int c = 0; c < CI; ++c) acc += ldv(w[(size_t)c * CNN_C]) * ldv(xs[c]);
                }
        const float zz = acc + b[o];
        z[t] = zz;
        stv(a[t], cnn_silu(zz));
    }
}

// Output layer: y[p] = b3 + sum_d sum_i W3[d][i] a2[p + d][i]; rho = rs softplus(y).
template <typename T>
__global__ void __launch_bounds__(CNN_NT) cnn_out_fwd_kernel(CnnGrid g, const T* __restrict__ a2,
                                                             const T* __restrict__ W3, const float* __restrict__ b3,
                                                             double rho_scale, float* __restrict__ y,
                                                             double* __restrict__ rho)
{
    for (long long p = blockIdx.x * (long long)CNN_NT + threadIdx.x; p < g.N; p += (long long)gridDim.x * CNN_NT) {
        int i, j, k;
        cnn_ijk(g, p, i, j, k);
        float acc = 0.0f;
        int d = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx, ++d) {
                    const T* xs = a2 + cnn_nb(g, i, j, k, dx, dy, dz) * CNN_C;
                    const T* w = W3 + (size_t)d * CNN_C;
                    for (int c = 0; c < CNN_C; ++c) acc += ldv(w[c]) * ldv(xs[c]);
                }
        const float yy = acc + b3[0];
        y[p] = yy;
        const float sp = fmaxf(yy, 0.0f) + log1pf(expf(-fabsf(yy)));
        rho[p] = rho_scale * (double)sp;
    }
}

// Loss partials and dL/dy: diff = rho - ref, part[block] = sum diff^2 (tree
// in shared memory), gy = 2 diff / (N rs^2) * rs * sigmoid(y).
__global__ void __launch_bounds__(CNN_NT) cnn_loss_kernel(CnnGrid g, const double* __restrict__ rho,
                                                          const double* __restrict__ ref, const float* __restrict__ y,
                                                          double rho_scale, float* __restrict__ gy,
                                                          double* __restrict__ part)
{
    __shared__ double s[CNN_NT];
    double acc = 0.0;
    const double cg = 2.0 / ((double)g.N * rho_scale);
    for (long long p = blockIdx.x * (long long)CNN_NT + threadIdx.x; p < g.N; p += (long long)gridDim.x * CNN_NT) {
        const double dlt = rho[p] - ref[p];
        acc += dlt * dlt;
        gy[p] = (float)(cg * dlt) * cnn_sigmoid(y[p]);
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = CNN_NT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// part[block] = sum of rho over the block's nodes (tree in shared memory).
__global__ void __launch_bounds__(CNN_NT) cnn_sum_kernel(CnnGrid g, const double* __restrict__ rho,
                                                         double* __restrict__ part)
{
    __shared__ double s[CNN_NT];
    double acc = 0.0;
    for (long long p = blockIdx.x * (long long)CNN_NT + threadIdx.x; p < g.N; p += (long long)gridDim.x * CNN_NT)
        acc += rho[p];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = CNN_NT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// out[0] = (sum_b part[b]) / (N rs^2), in block order (one thread).
__global__ void cnn_loss_sum_kernel(const double* __restrict__ part, int nb, double norm, double* __restrict__ out)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b];
    out[0] = s * norm;
}

// Data gradient through a conv layer: gx[p][i] = (sum_d sum_o W[d][i][o]
// gz[p - d][o]) * silu'(zx[p][i]).  CO = outputs of the layer (1 or 32).
template <typename T, int CO, int K>
__global__ void __launch_bounds__(CNN_NT) cnn_conv_bwd_data_kernel(CnnGrid g, const float* __restrict__ gz,
                                                                   const T* __restrict__ W,
                                                                   const float* __restrict__ zx,
                                                                   float* __restrict__ gx)
{
    constexpr int R = (K - 1) / 2;
    for (long long t = blockIdx.x * (long long)CNN_NT + threadIdx.x; t < g.N * CNN_C;
         t += (long long)gridDim.x * CNN_NT) {
        const long long p = t / CNN_C;
        const int ci = (int)(t % CNN_C);
        int i, j, k;
        cnn_ijk(g, p, i, j, k);
        float acc = 0.0f;
        int d = 0;
        for (int dz = -R; dz <= R; ++dz)
            for (int dy = -R; dy <= R; ++dy)
                for (int dx = -R; dx <= R; ++dx, ++d) {
                    const float* gs = gz + cnn_nb(g, i, j, k, -dx, -dy, -dz) * CO;
                    const T* w = W + ((size_t)d * CNN_C + ci) * CO;
                    for (int o = 0; o < CO; ++o) acc += ldv(w[o]) * gs[o];
                }
        gx[t] = acc * cnn_silu_grad(zx[t]);
    }
}

// Weight-gradient partials: block (chunk, d) adds, over the nodes of its
// chunk, G[p][o] A[p + d][i] into part[chunk][d][i][o] (CI x CO outputs);
// the extra tap d = K^3 is the bias (A = 1, one input).
template <typename T, int CI, int CO, int K>
__global__ void __launch_bounds__(CNN_NT) cnn_wgrad_kernel(CnnGrid g, const float* __restrict__ G,
                                                           const T* __restrict__ A, float* __restrict__ part)
{
    constexpr int R = (K - 1) / 2;
    constexpr int TAPS = K * K * K;
    constexpr int NOUT = CI * CO;
    constexpr int PER = (NOUT + CNN_NT - 1) / CNN_NT;
    const int d = blockIdx.y;
    const long long chunk = blockIdx.x;
    const long long p0 = chunk * CNN_CHUNK;
    const long long p1 = p0 + CNN_CHUNK < g.N ? p0 + CNN_CHUNK : g.N;
    const int dz = d / (K * K) - R, dy = (d / K) % K - R, dx = d % K - R;
    const bool bias = d == TAPS;
    float acc[PER];
    for (int u = 0; u < PER; ++u) acc[u] = 0.0f;
    for (long long p = p0; p < p1; ++p) {
        int i, j, k;
        cnn_ijk(g, p, i, j, k);
        const long long q = bias ? p : cnn_nb(g, i, j, k, dx, dy, dz);
        for (int u = 0; u < PER; ++u) {
            const int e = threadIdx.x + u * CNN_NT;
            if (e >= NOUT) break;
            const int ci = e / CO, o = e % CO;
            if (bias && ci > 0) continue;
            const float av = bias ? 1.0f : ldv(A[q * CI + ci]);
            acc[u] += G[p * CO + o] * av;
        }
    }
    float* out = part + ((size_t)chunk * (TAPS + 1) + d) * NOUT;
    for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + u * CNN_NT;
        if (e < NOUT) out[e] = acc[u];
    }
}

// grad[d][e] = sum over chunks (in order) of part[chunk][d][e], for the
// TAPS + 1 taps of one layer; the bias (tap TAPS) keeps its first CO entries.
__global__ void cnn_wgrad_sum_kernel(const float* __restrict__ part, int nchunk, int taps1, int nout, int co,
                                     float* __restrict__ gw, float* __restrict__ gb, int accumulate)
{
    const long long n = (long long)taps1 * nout;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int c = 0; c < nchunk; ++c) s += part[(size_t)c * n + t];
        const long long d = t / nout;
        const int e = (int)(t % nout);
        if (d < taps1 - 1) {
            gw[t] = accumulate ? gw[t] + s : s;
        } else if (e < co) {
            gb[e] = accumulate ? gb[e] + s : s;
        }
    }
}

// Adam on the FP32 master weights (flat), then the compute copy in T:
// m = b1 m + (1-b1) g s, v = b2 v + (1-b2) (g s)^2, w -= lr (m c1) / (sqrt(v c2) + eps)
// with s the gradient scale and c1, c2 the bias corrections 1/(1 - b^t).
__global__ void cnn_adam_kernel(long long n, float* __restrict__ w, const float* __restrict__ gr,
                                float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float eps,
                                float c1, float c2, float gscale)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const float gg = gr[t] * gscale;
        const float mm = b1 * m[t] + (1.0f - b1) * gg;
        const float vv = b2 * v[t] + (1.0f - b2) * gg * gg;
        m[t] = mm;
        v[t] = vv;
        w[t] -= lr * (mm * c1) / (sqrtf(vv * c2) + eps);
    }
}

// Compute copies of the weights: dst[t] = T(src[t]).
template <typename T>
__global__ void cnn_cast_kernel(long long n, const float* __restrict__ src, T* __restrict__ dst)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        stv(dst[t], src[t]);
}

}  // namespace sq
