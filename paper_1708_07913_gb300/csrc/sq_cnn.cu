// sq_cnn.cu -- host side of the learned-warm-start network (include/sq.h,
// sq_cnn_*): parameter layouts, device buffers, and the launch sequences of
// the forward pass, the backward pass and the Adam step (kernels in
// sq_cnn.cuh).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/sq.h"
#include "sq_cnn.cuh"
#include "sq_cnn_tc.cuh"

using namespace sq;

namespace {

constexpr int C = CNN_C;
constexpr int T1 = 125, T2 = 27, T3 = 27;                 // taps of the three kernels
// flat parameter layout on the device (FP32 master, gradients, Adam moments)
constexpr long long OW1 = 0, OB1 = OW1 + (long long)T1 * C, OW2 = OB1 + C, OB2 = OW2 + (long long)T2 * C * C,
                    OW3 = OB2 + C, OB3 = OW3 + (long long)T3 * C, NPARAM = OB3 + 1;

bool dev_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename P>
int alloc(P** p, size_t bytes)
{
    *p = nullptr;
    if (cudaMalloc((void**)p, std::max<size_t>(bytes, 256)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return SQ_ENOMEM;
    }
    return SQ_OK;
}

}  // namespace

struct sq_cnn {
    int bf16 = 1;
    cudaStream_t st = nullptr;
    int sm = 1;
    double v_shift = 0.0, v_scale = 1.0, rho_scale = 1.0;
    double shift = 0.0;               // extra input shift (sq_cnn_set_shift)
    long long t = 0;                  // Adam steps taken
    bool have_params = false, have_grads = false;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    void* wt = nullptr;               // compute copy of w (bf16 or float)
    // activations and gradients for up to cap nodes
    long long cap = 0;
    void *x0 = nullptr, *a1 = nullptr, *a2 = nullptr;
    float *z1 = nullptr, *z2 = nullptr, *y = nullptr, *gy = nullptr, *gz1 = nullptr, *gz2 = nullptr;
    float* part = nullptr;
    double* lpart = nullptr;
    double* lout = nullptr;
    // bfloat16 networks run the middle layer's forward on the tensor cores
    // (sq_cnn_tc.cuh) unless SQ_CNN_TENSOR=0 was set when the network was
    // created; its latched wait-expiry bit lives here
    int tensor = 1;
    unsigned* err = nullptr;
};

namespace {

void free_bufs(sq_cnn* n)
{
    void* p[] = {n->x0, n->a1, n->a2, n->z1, n->z2, n->y, n->gy, n->gz1, n->gz2, n->part, n->lpart, n->lout};
    for (void* q : p)
        if (q) cudaFree(q);
    n->x0 = n->a1 = n->a2 = nullptr;
    n->z1 = n->z2 = n->y = n->gy = n->gz1 = n->gz2 = n->part = nullptr;
    n->lpart = n->lout = nullptr;
    n->cap = 0;
}

constexpr int LOSS_BLOCKS = 1024;

long long nchunks(long long N) { return (N + CNN_CHUNK - 1) / CNN_CHUNK; }

int ensure(sq_cnn* n, long long N)
{
    if (N <= n->cap) return SQ_OK;
    if (cudaStreamSynchronize(n->st) != cudaSuccess) return SQ_ECUDA;
    free_bufs(n);
    const size_t ts = n->bf16 ? sizeof(Bf16) : sizeof(float);
    const size_t NC = (size_t)N * C;
    const size_t part = (size_t)nchunks(N) * std::max({(size_t)(T1 + 1) * C, (size_t)(T2 + 1) * C * C,
                                                       (size_t)(T3 + 1) * C});
    int rc;
    if ((rc = alloc(&n->x0, ts * N)) || (rc = alloc(&n->a1, ts * NC)) || (rc = alloc(&n->a2, ts * NC)) ||
        (rc = alloc(&n->z1, 4 * NC)) || (rc = alloc(&n->z2, 4 * NC)) || (rc = alloc(&n->y, 4 * (size_t)N)) ||
        (rc = alloc(&n->gy, 4 * (size_t)N)) || (rc = alloc(&n->gz1, 4 * NC)) || (rc = alloc(&n->gz2, 4 * NC)) ||
        (rc = alloc(&n->part, 4 * part)) || (rc = alloc(&n->lpart, 8 * LOSS_BLOCKS)) || (rc = alloc(&n->lout, 8))) {
        free_bufs(n);
        return rc;
    }
    n->cap = N;
    return SQ_OK;
}

int grid_for(long long work, int sm)
{
    long long b = (work + CNN_NT - 1) / CNN_NT;
    return (int)std::max<long long>(1, std::min<long long>(b, (long long)sm * 16));
}

template <typename T>
int forward_t(sq_cnn* n, const CnnGrid& g, const double* V, double* rho)
{
    const T* wt = (const T*)n->wt;
    T* x0 = (T*)n->x0;
    T* a1 = (T*)n->a1;
    T* a2 = (T*)n->a2;
    const int gN = grid_for(g.N, n->sm), gNC = grid_for(g.N * C, n->sm);
    cnn_input_kernel<T><<<gN, CNN_NT, 0, n->st>>>(g, V, n->v_shift + n->shift, n->v_scale, x0);
    cnn_conv_fwd_kernel<T, 1, 5><<<gNC, CNN_NT, 0, n->st>>>(g, x0, wt + OW1, n->w + OB1, n->z1, a1);
    if constexpr (sizeof(T) == sizeof(Bf16)) {
        if (n->tensor) {
            static bool attr = false;        // the kernel's shared memory exceeds the 48 KB default
            if (!attr) {
                if (cudaFuncSetAttribute(cnn_conv2_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM) !=
                    cudaSuccess)
                    return SQ_ECUDA;
                attr = true;
            }
            const long long tiles = (g.N + TC_M - 1) / TC_M;
            const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, (long long)n->sm));
            cnn_conv2_tc_kernel<<<grid, 128, TC_SMEM, n->st>>>(g, (const Bf16*)a1, (const Bf16*)(wt + OW2),
                                                               n->w + OB2, n->z2, (Bf16*)a2, n->err);
        } else {
            cnn_conv_fwd_kernel<T, C, 3><<<gNC, CNN_NT, 0, n->st>>>(g, a1, wt + OW2, n->w + OB2, n->z2, a2);
        }
    } else {
        cnn_conv_fwd_kernel<T, C, 3><<<gNC, CNN_NT, 0, n->st>>>(g, a1, wt + OW2, n->w + OB2, n->z2, a2);
    }
    cnn_out_fwd_kernel<T><<<gN, CNN_NT, 0, n->st>>>(g, a2, wt + OW3, n->w + OB3, n->rho_scale, n->y, rho);
    return cudaGetLastError() == cudaSuccess ? SQ_OK : SQ_ECUDA;
}

// After a synchronisation: SQ_ETIMEOUT (and the bit cleared) if a tensor-core
// wait expired since the last check.
int take_tc_error(sq_cnn* n)
{
    unsigned e = 0;
    if (cudaMemcpy(&e, n->err, sizeof(e), cudaMemcpyDeviceToHost) != cudaSuccess) return SQ_ECUDA;
    if (!e) return SQ_OK;
    if (cudaMemset(n->err, 0, sizeof(unsigned)) != cudaSuccess) return SQ_ECUDA;
    return SQ_ETIMEOUT;
}

template <typename T>
int backward_t(sq_cnn* n, const CnnGrid& g, const double* ref, const double* rho, int accumulate)
{
    const T* wt = (const T*)n->wt;
    const int gN = std::min(grid_for(g.N, n->sm), LOSS_BLOCKS), gNC = grid_for(g.N * C, n->sm);
    cnn_loss_kernel<<<gN, CNN_NT, 0, n->st>>>(g, rho, ref, n->y, n->rho_scale, n->gy, n->lpart);
    cnn_loss_sum_kernel<<<1, 32, 0, n->st>>>(n->lpart, gN, 1.0 / ((double)g.N * n->rho_scale * n->rho_scale),
                                             n->lout);
    const int nc = (int)nchunks(g.N);
    // output layer: weights, then the data gradient into the second layer
    cnn_wgrad_kernel<T, C, 1, 3><<<dim3(nc, T3 + 1), CNN_NT, 0, n->st>>>(g, n->gy, (const T*)n->a2, n->part);
    cnn_wgrad_sum_kernel<<<grid_for((long long)(T3 + 1) * C, n->sm), CNN_NT, 0, n->st>>>(
        n->part, nc, T3 + 1, C, 1, n->g + OW3, n->g + OB3, accumulate);
    cnn_conv_bwd_data_kernel<T, 1, 3><<<gNC, CNN_NT, 0, n->st>>>(g, n->gy, wt + OW3, n->z2, n->gz2);
    // second layer
    cnn_wgrad_kernel<T, C, C, 3><<<dim3(nc, T2 + 1), CNN_NT, 0, n->st>>>(g, n->gz2, (const T*)n->a1, n->part);
    cnn_wgrad_sum_kernel<<<grid_for((long long)(T2 + 1) * C * C, n->sm), CNN_NT, 0, n->st>>>(
        n->part, nc, T2 + 1, C * C, C, n->g + OW2, n->g + OB2, accumulate);
    cnn_conv_bwd_data_kernel<T, C, 3><<<gNC, CNN_NT, 0, n->st>>>(g, n->gz2, wt + OW2, n->z1, n->gz1);
    // first layer
    cnn_wgrad_kernel<T, 1, C, 5><<<dim3(nc, T1 + 1), CNN_NT, 0, n->st>>>(g, n->gz1, (const T*)n->x0, n->part);
    cnn_wgrad_sum_kernel<<<grid_for((long long)(T1 + 1) * C, n->sm), CNN_NT, 0, n->st>>>(
        n->part, nc, T1 + 1, C, C, n->g + OW1, n->g + OB1, accumulate);
    return cudaGetLastError() == cudaSuccess ? SQ_OK : SQ_ECUDA;
}

int cast_weights(sq_cnn* n)
{
    const int gb = grid_for(NPARAM, n->sm);
    if (n->bf16) cnn_cast_kernel<Bf16><<<gb, CNN_NT, 0, n->st>>>(NPARAM, n->w, (Bf16*)n->wt);
    else cnn_cast_kernel<float><<<gb, CNN_NT, 0, n->st>>>(NPARAM, n->w, (float*)n->wt);
    return cudaGetLastError() == cudaSuccess ? SQ_OK : SQ_ECUDA;
}

bool grid_ok(int n1, int n2, int n3)
{
    return n1 >= 1 && n2 >= 1 && n3 >= 1 && n1 <= 4096 && n2 <= 4096 && n3 <= 4096 &&
           (long long)n1 * n2 * n3 <= (1LL << 28);
}

// host layout (the network's natural order) <-> device flat layout
//   host: W1 (C,1,5,5,5), b1 (C), W2 (C,C,3,3,3), b2 (C), W3 (1,C,3,3,3), b3 (1)
//   device: W1[tap][o], b1, W2[tap][i][o], b2, W3[tap][i], b3
void host_to_dev(const double* h, std::vector<float>& d)
{
    d.assign(NPARAM, 0.0f);
    const double* hW1 = h;
    const double* hb1 = hW1 + (size_t)C * T1;
    const double* hW2 = hb1 + C;
    const double* hb2 = hW2 + (size_t)C * C * T2;
    const double* hW3 = hb2 + C;
    const double* hb3 = hW3 + (size_t)C * T3;
    for (int o = 0; o < C; ++o)
        for (int t = 0; t < T1; ++t) d[OW1 + (size_t)t * C + o] = (float)hW1[(size_t)o * T1 + t];
    for (int o = 0; o < C; ++o) d[OB1 + o] = (float)hb1[o];
    for (int o = 0; o < C; ++o)
        for (int i = 0; i < C; ++i)
            for (int t = 0; t < T2; ++t) d[OW2 + ((size_t)t * C + i) * C + o] = (float)hW2[((size_t)o * C + i) * T2 + t];
    for (int o = 0; o < C; ++o) d[OB2 + o] = (float)hb2[o];
    for (int i = 0; i < C; ++i)
        for (int t = 0; t < T3; ++t) d[OW3 + (size_t)t * C + i] = (float)hW3[(size_t)i * T3 + t];
    d[OB3] = (float)hb3[0];
}

void dev_to_host(const std::vector<float>& d, double* h)
{
    double* hW1 = h;
    double* hb1 = hW1 + (size_t)C * T1;
    double* hW2 = hb1 + C;
    double* hb2 = hW2 + (size_t)C * C * T2;
    double* hW3 = hb2 + C;
    double* hb3 = hW3 + (size_t)C * T3;
    for (int o = 0; o < C; ++o)
        for (int t = 0; t < T1; ++t) hW1[(size_t)o * T1 + t] = d[OW1 + (size_t)t * C + o];
    for (int o = 0; o < C; ++o) hb1[o] = d[OB1 + o];
    for (int o = 0; o < C; ++o)
        for (int i = 0; i < C; ++i)
            for (int t = 0; t < T2; ++t) hW2[((size_t)o * C + i) * T2 + t] = d[OW2 + ((size_t)t * C + i) * C + o];
    for (int o = 0; o < C; ++o) hb2[o] = d[OB2 + o];
    for (int i = 0; i < C; ++i)
        for (int t = 0; t < T3; ++t) hW3[(size_t)i * T3 + t] = d[OW3 + (size_t)t * C + i];
    hb3[0] = d[OB3];
}

int get_flat(sq_cnn* n, const float* src, double* host)
{
    std::vector<float> d(NPARAM);
    if (cudaMemcpyAsync(d.data(), src, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, n->st) != cudaSuccess ||
        cudaStreamSynchronize(n->st) != cudaSuccess)
        return SQ_ECUDA;
    dev_to_host(d, host);
    return SQ_OK;
}

}  // namespace

extern "C" {

long long sq_cnn_param_count(int channels) { return channels == C ? NPARAM : -1; }

int sq_cnn_create(sq_cnn** out, int channels, int bf16, void* cuda_stream)
{
    if (!out) return SQ_EINVAL;
    *out = nullptr;
    if (channels != C) return SQ_EUNSUPPORTED;
    if (bf16 != 0 && bf16 != 1) return SQ_EINVAL;
    sq_cnn* n = new (std::nothrow) sq_cnn();
    if (!n) return SQ_ENOMEM;
    n->bf16 = bf16;
    n->st = (cudaStream_t)cuda_stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n->sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        delete n;
        return SQ_ECUDA;
    }
    int rc;
    const size_t ts = bf16 ? sizeof(Bf16) : sizeof(float);
    if ((rc = alloc(&n->w, 4 * NPARAM)) || (rc = alloc(&n->g, 4 * NPARAM)) || (rc = alloc(&n->m, 4 * NPARAM)) ||
        (rc = alloc(&n->v, 4 * NPARAM)) || (rc = alloc(&n->wt, ts * NPARAM)) || (rc = alloc(&n->err, 4))) {
        sq_cnn_destroy(n);
        return rc;
    }
    const char* env = getenv("SQ_CNN_TENSOR");
    n->tensor = !(env && strcmp(env, "0") == 0);
    if (cudaMemsetAsync(n->err, 0, sizeof(unsigned), n->st) != cudaSuccess ||
        cudaMemsetAsync(n->g, 0, 4 * NPARAM, n->st) != cudaSuccess ||
        cudaMemsetAsync(n->m, 0, 4 * NPARAM, n->st) != cudaSuccess ||
        cudaMemsetAsync(n->v, 0, 4 * NPARAM, n->st) != cudaSuccess || cudaStreamSynchronize(n->st) != cudaSuccess) {
        cudaGetLastError();
        sq_cnn_destroy(n);
        return SQ_ECUDA;
    }
    *out = n;
    return SQ_OK;
}

int sq_cnn_set_params(sq_cnn* n, const double* params_host, double v_shift, double v_scale, double rho_scale)
{
    if (!n || !params_host || !std::isfinite(v_shift) || !std::isfinite(v_scale) || v_scale == 0.0 ||
        !std::isfinite(rho_scale) || rho_scale <= 0.0)
        return SQ_EINVAL;
    for (long long i = 0; i < NPARAM; ++i)
        if (!std::isfinite(params_host[i])) return SQ_EINVAL;
    std::vector<float> d;
    host_to_dev(params_host, d);
    if (cudaMemcpyAsync(n->w, d.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice, n->st) != cudaSuccess ||
        cudaMemsetAsync(n->m, 0, 4 * NPARAM, n->st) != cudaSuccess ||
        cudaMemsetAsync(n->v, 0, 4 * NPARAM, n->st) != cudaSuccess)
        return SQ_ECUDA;
    int rc = cast_weights(n);
    if (rc) return rc;
    if (cudaStreamSynchronize(n->st) != cudaSuccess) return SQ_ECUDA;
    n->v_shift = v_shift;
    n->v_scale = v_scale;
    n->rho_scale = rho_scale;
    n->shift = 0.0;
    n->t = 0;
    n->have_params = true;
    n->have_grads = false;
    return SQ_OK;
}

int sq_cnn_get_params(sq_cnn* n, double* params_host)
{
    if (!n || !params_host || !n->have_params) return SQ_EINVAL;
    return get_flat(n, n->w, params_host);
}

int sq_cnn_get_grads(sq_cnn* n, double* grads_host)
{
    if (!n || !grads_host || !n->have_grads) return SQ_EINVAL;
    return get_flat(n, n->g, grads_host);
}

int sq_cnn_forward(sq_cnn* n, int n1, int n2, int n3, const double* V, double* rho)
{
    if (!n || !n->have_params || !grid_ok(n1, n2, n3) || !dev_ptr(V) || !dev_ptr(rho)) return SQ_EINVAL;
    CnnGrid g{n1, n2, n3, (long long)n1 * n2 * n3};
    int rc = ensure(n, g.N);
    if (rc) return rc;
    return n->bf16 ? forward_t<Bf16>(n, g, V, rho) : forward_t<float>(n, g, V, rho);
}

int sq_cnn_set_shift(sq_cnn* n, double shift)
{
    if (!n || !std::isfinite(shift)) return SQ_EINVAL;
    n->shift = shift;
    return SQ_OK;
}

int sq_cnn_forward_sum(sq_cnn* n, int n1, int n2, int n3, const double* V, double* rho, double* sum_host)
{
    if (!sum_host) return SQ_EINVAL;
    int rc = sq_cnn_forward(n, n1, n2, n3, V, rho);
    if (rc) return rc;
    CnnGrid g{n1, n2, n3, (long long)n1 * n2 * n3};
    const int gN = std::min(grid_for(g.N, n->sm), LOSS_BLOCKS);
    cnn_sum_kernel<<<gN, CNN_NT, 0, n->st>>>(g, rho, n->lpart);
    cnn_loss_sum_kernel<<<1, 32, 0, n->st>>>(n->lpart, gN, 1.0, n->lout);
    if (cudaGetLastError() != cudaSuccess) return SQ_ECUDA;
    if (cudaMemcpyAsync(sum_host, n->lout, sizeof(double), cudaMemcpyDeviceToHost, n->st) != cudaSuccess ||
        cudaStreamSynchronize(n->st) != cudaSuccess)
        return SQ_ECUDA;
    return take_tc_error(n);
}

int sq_cnn_backward(sq_cnn* n, int n1, int n2, int n3, const double* V, const double* rho_ref, double* rho,
                    int accumulate, double* loss_host)
{
    if (!n || !n->have_params || !grid_ok(n1, n2, n3) || !dev_ptr(V) || !dev_ptr(rho_ref) || !dev_ptr(rho) ||
        (accumulate != 0 && accumulate != 1) || (accumulate && !n->have_grads))
        return SQ_EINVAL;
    CnnGrid g{n1, n2, n3, (long long)n1 * n2 * n3};
    int rc = ensure(n, g.N);
    if (rc) return rc;
    rc = n->bf16 ? forward_t<Bf16>(n, g, V, rho) : forward_t<float>(n, g, V, rho);
    if (rc) return rc;
    rc = n->bf16 ? backward_t<Bf16>(n, g, rho_ref, rho, accumulate) : backward_t<float>(n, g, rho_ref, rho, accumulate);
    if (rc) return rc;
    n->have_grads = true;
    if (loss_host) {
        if (cudaMemcpyAsync(loss_host, n->lout, sizeof(double), cudaMemcpyDeviceToHost, n->st) != cudaSuccess ||
            cudaStreamSynchronize(n->st) != cudaSuccess)
            return SQ_ECUDA;
        return take_tc_error(n);
    }
    return SQ_OK;
}

int sq_cnn_adam_step(sq_cnn* n, double lr, double beta1, double beta2, double eps, double grad_scale)
{
    if (!n || !n->have_grads || !(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) ||
        !(eps >= 0.0) || !std::isfinite(grad_scale))
        return SQ_EINVAL;
    n->t += 1;
    const double c1 = 1.0 / (1.0 - pow(beta1, (double)n->t)), c2 = 1.0 / (1.0 - pow(beta2, (double)n->t));
    cnn_adam_kernel<<<grid_for(NPARAM, n->sm), CNN_NT, 0, n->st>>>(
        NPARAM, n->w, n->g, n->m, n->v, (float)lr, (float)beta1, (float)beta2, (float)eps, (float)c1, (float)c2,
        (float)grad_scale);
    if (cudaGetLastError() != cudaSuccess) return SQ_ECUDA;
    return cast_weights(n);
}

void sq_cnn_destroy(sq_cnn* n)
{
    if (!n) return;
    if (n->st) cudaStreamSynchronize(n->st);
    free_bufs(n);
    void* p[] = {n->w, n->g, n->m, n->v, n->wt, n->err};
    for (void* q : p)
        if (q) cudaFree(q);
    delete n;
}

}  // extern "C"
