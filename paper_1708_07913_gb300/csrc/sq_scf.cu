// sq_scf.cu -- the pieces of the self-consistent field (SCF) loop around the
// SQ path, on the GPU: the electrostatic potential of Eq. (PoissonEqn) on the
// periodic cell by conjugate gradients with the finite-difference Laplacian
// of Eq. (FD:Laplacian) (the paper solves it with AAR; Section 3), the
// effective potential V_loc + phi + v_x with Slater X-alpha exchange (the
// paper uses LDA), and Anderson mixing of the effective potential (the paper
// uses Periodic Pulay mixing; Section 3).
//
// Every reduction is a fixed-order two-pass sum (a tree per block, then the
// block partials added in index order by the last block to finish), so all
// results repeat bit for bit.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "sq_internal.cuh"

using sq::FD_NO;

namespace {

constexpr int T_RED = 256;          // threads per reduction block
constexpr int MAX_RED_BLOCKS = 1024;
constexpr int MAX_HIST = 16;        // Anderson history

// sum over t of A(t) B(t), A = a1 - a0, B = b1 - b0 (a0, b0 may be NULL;
// b1 NULL means B = 1).  Block partials, then the last block adds them in
// index order into *out and resets the counter.
__global__ void dot_kernel(const double* __restrict__ a1, const double* __restrict__ a0,
                           const double* __restrict__ b1, const double* __restrict__ b0, long long n,
                           double* partials, unsigned* counter, double* out)
{
    __shared__ double sh[T_RED / 32];
    __shared__ bool last;
    double s = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const double A = a0 ? a1[t] - a0[t] : a1[t];
        const double B = b1 ? (b0 ? b1[t] - b0[t] : b1[t]) : 1.0;
        s += A * B;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += sh[w];
        partials[blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double tot = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) tot += ((volatile double*)partials)[b];
        *out = tot;
        *counter = 0;
    }
}

// max over t of |a(t) - b(t)|, block maxima then the last block's maximum in
// index order into *out (a maximum does not depend on the order; the form
// matches dot_kernel).
__global__ void maxabs_kernel(const double* __restrict__ a, const double* __restrict__ b, long long n,
                              double* partials, unsigned* counter, double* out)
{
    __shared__ double sh[T_RED / 32];
    __shared__ bool last;
    double s = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        s = fmax(s, fabs(a[t] - b[t]));
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
        partials[blockIdx.x] = m;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double m = 0.0;
        for (unsigned k = 0; k < gridDim.x; ++k) m = fmax(m, ((volatile double*)partials)[k]);
        *out = m;
        *counter = 0;
    }
}

// chi = chi_ref, zeta = zeta_ref + *w (the Weyl widening of sq_widen_bounds).
__global__ void widen_kernel(const double* __restrict__ chi_ref, const double* __restrict__ zeta_ref,
                             const double* w, double* chi, double* zeta, long long n)
{
    const double dw = *w;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        chi[t] = chi_ref[t];
        zeta[t] = zeta_ref[t] + dw;
    }
}

// y = -lap_h x on the periodic grid (x fastest): the d = 0 term of
// Eq. (FD:Laplacian) appears in its six axis terms.
struct FDW {
    double w[FD_NO + 1];
};
__global__ void lap_periodic_kernel(const double* __restrict__ x, double* __restrict__ y, int n1, int n2, int n3,
                                    FDW fw)
{
    const long long n = (long long)n1 * n2 * n3;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % n1), j = (int)((p / n1) % n2), k = (int)(p / ((long long)n1 * n2));
        const long long row = p - i, plane = p - i - (long long)j * n1;
        double acc = 6.0 * fw.w[0] * x[p];
        for (int d = 1; d <= FD_NO; ++d) {
            const int ip = (i + d) % n1, im = ((i - d) % n1 + n1) % n1;
            const int jp = (j + d) % n2, jm = ((j - d) % n2 + n2) % n2;
            const int kp = (k + d) % n3, km = ((k - d) % n3 + n3) % n3;
            const double sx = x[row + ip] + x[row + im];
            const double sy = x[plane + (long long)jp * n1 + i] + x[plane + (long long)jm * n1 + i];
            const double sz = x[((long long)kp * n2 + j) * n1 + i] + x[((long long)km * n2 + j) * n1 + i];
            acc += fw.w[d] * ((sx + sy) + sz);
        }
        y[p] = -acc;
    }
}

__global__ void rhs_kernel(const double* __restrict__ rho, const double* mean, double* __restrict__ b, long long n)
{
    const double m = *mean / (double)n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        b[t] = 4.0 * M_PI * (rho[t] - m);
}

__global__ void shift_kernel(double* __restrict__ x, const double* sum, long long n)
{
    const double m = *sum / (double)n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        x[t] -= m;
}

__global__ void cg_update_kernel(double* __restrict__ phi, double* __restrict__ r, const double* __restrict__ p,
                                 const double* __restrict__ Ap, double alpha, long long n)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        phi[t] += alpha * p[t];
        r[t] -= alpha * Ap[t];
    }
}

__global__ void xpby_kernel(double* __restrict__ p, const double* __restrict__ r, double beta, long long n)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        p[t] = r[t] + beta * p[t];
}

// V_out = V_loc + phi + v_x(rho), v_x = -(3 alpha / 2) (3 rho / pi)^(1/3) (0 for rho <= 0)
__global__ void veff_kernel(const double* __restrict__ vloc, const double* __restrict__ phi,
                            const double* __restrict__ rho, double alpha, double* __restrict__ vout, long long n)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const double r = rho[t];
        const double vx = r > 0.0 ? -1.5 * alpha * cbrt(3.0 * r / M_PI) : 0.0;
        vout[t] = vloc[t] + phi[t] + vx;
    }
}

// Anderson update: out = x + beta f - sum_i g_i ((X_{i+1} - X_i) + beta (F_{i+1} - F_i))
struct MixHist {
    const double* X[MAX_HIST + 1];
    const double* F[MAX_HIST + 1];
    double g[MAX_HIST];
};
__global__ void mix_kernel(MixHist H, int m, double beta, double* __restrict__ out, long long n)
{
    const double* x = H.X[m];
    const double* f = H.F[m];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        double v = x[t] + beta * f[t];
        for (int i = 0; i < m; ++i)
            v -= H.g[i] * ((H.X[i + 1][t] - H.X[i][t]) + beta * (H.F[i + 1][t] - H.F[i][t]));
        out[t] = v;
    }
}

__global__ void sub_kernel(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out,
                           long long n)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        out[t] = a[t] - b[t];
}

// y = -lap_h x + s x on the periodic grid (the operator of the preconditioner)
__global__ void helmholtz_kernel(const double* __restrict__ x, double* __restrict__ y, int n1, int n2, int n3,
                                 FDW fw, double s)
{
    const long long n = (long long)n1 * n2 * n3;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % n1), j = (int)((p / n1) % n2), k = (int)(p / ((long long)n1 * n2));
        const long long row = p - i, plane = p - i - (long long)j * n1;
        double acc = 6.0 * fw.w[0] * x[p];
        for (int d = 1; d <= FD_NO; ++d) {
            const int ip = (i + d) % n1, im = ((i - d) % n1 + n1) % n1;
            const int jp = (j + d) % n2, jm = ((j - d) % n2 + n2) % n2;
            const int kp = (k + d) % n3, km = ((k - d) % n3 + n3) % n3;
            const double sx = x[row + ip] + x[row + im];
            const double sy = x[plane + (long long)jp * n1 + i] + x[plane + (long long)jm * n1 + i];
            const double sz = x[((long long)kp * n2 + j) * n1 + i] + x[((long long)km * n2 + j) * n1 + i];
            acc += fw.w[d] * ((sx + sy) + sz);
        }
        y[p] = s * x[p] - acc;
    }
}

// out = v_in + f - c u (u is read from out)
__global__ void kerker_out_kernel(const double* __restrict__ v_in, const double* __restrict__ f, double c,
                                  double* __restrict__ out, long long n)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        out[t] = v_in[t] + f[t] - c * out[t];
}

// Reduction scratch: partials, a counter and a few result slots.
struct Red {
    double* partials = nullptr;
    unsigned* counter = nullptr;
    double* out = nullptr;       // result slots (device)
    int blocks = 0;
};

int red_alloc(Red& R, int sm_count, int slots)
{
    R.blocks = std::min(MAX_RED_BLOCKS, std::max(1, sm_count * 4));
    if (cudaMalloc(&R.partials, sizeof(double) * R.blocks) != cudaSuccess ||
        cudaMalloc(&R.counter, sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&R.out, sizeof(double) * slots) != cudaSuccess ||
        cudaMemset(R.counter, 0, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return SQ_ENOMEM;
    }
    return SQ_OK;
}

void red_free(Red& R)
{
    if (R.partials) cudaFree(R.partials);
    if (R.counter) cudaFree(R.counter);
    if (R.out) cudaFree(R.out);
    R = Red();
}

int grid_for(long long n, int sm_count)
{
    return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)sm_count * 8));
}

// Enqueue one dot into slot `slot` of R.out.
int enqueue_dot(Red& R, const double* a1, const double* a0, const double* b1, const double* b0, long long n,
                int slot, cudaStream_t st)
{
    dot_kernel<<<R.blocks, T_RED, 0, st>>>(a1, a0, b1, b0, n, R.partials, R.counter, R.out + slot);
    return cudaGetLastError() == cudaSuccess ? SQ_OK : SQ_ECUDA;
}

int read_slots(Red& R, double* host, int count, cudaStream_t st)
{
    if (cudaMemcpyAsync(host, R.out, sizeof(double) * count, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return SQ_ECUDA;
    }
    return SQ_OK;
}

int read_slot(Red& R, int slot, double* host, cudaStream_t st)
{
    if (cudaMemcpyAsync(host, R.out + slot, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return SQ_ECUDA;
    }
    return SQ_OK;
}

bool device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

// Poisson scratch of a context: b, r, p, Ap and a reduction; kept in a
// table keyed by the context (created on first use, released with it).
struct PoissonWS {
    double* buf = nullptr;
    long long n = 0;
    Red red;
};

namespace {
std::mutex g_ws_mutex;
std::unordered_map<const sq_ctx*, PoissonWS*> g_ws;

void ws_free(PoissonWS* w)
{
    if (!w) return;
    if (w->buf) cudaFree(w->buf);
    red_free(w->red);
    delete w;
}

// The context's workspace of 4 N doubles and a reduction (created on first
// use; shared by the Poisson solve and the preconditioner).
int context_ws(sq_ctx* c, PoissonWS** out)
{
    const long long n = c->g.Nd;
    PoissonWS* ws = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_ws_mutex);
        auto it = g_ws.find(c);
        if (it != g_ws.end()) ws = it->second;
    }
    if (!ws) {
        ws = new (std::nothrow) PoissonWS();
        if (!ws) return SQ_ENOMEM;
        int rc = cudaMalloc(&ws->buf, sizeof(double) * 4 * n) == cudaSuccess ? SQ_OK : SQ_ENOMEM;
        if (rc == SQ_OK) rc = red_alloc(ws->red, c->sm_count, 8);
        if (rc) {
            cudaGetLastError();
            ws_free(ws);
            return rc;
        }
        ws->n = n;
        std::lock_guard<std::mutex> lk(g_ws_mutex);
        g_ws[c] = ws;
    }
    *out = ws;
    return SQ_OK;
}
}  // namespace

namespace sq {
// Called when a context is destroyed.
void free_poisson_ws(sq_ctx* c)
{
    std::lock_guard<std::mutex> lk(g_ws_mutex);
    auto it = g_ws.find(c);
    if (it == g_ws.end()) return;
    ws_free(it->second);
    g_ws.erase(it);
}
}  // namespace sq

// ------------------------------------------------------------------------
// Anderson mixer
// ------------------------------------------------------------------------
struct sq_mixer {
    long long n = 0;
    int hist = 0;
    double beta = 0.0;
    int period = 1;              // Pulay extrapolation on every period-th step (1: every step)
    long long steps = 0;         // steps taken (decides the Pulay steps)
    cudaStream_t st = nullptr;
    int sm = 1;
    std::vector<double*> X, F;   // hist + 1 slots each
    std::vector<int> order;      // slot indices, oldest first
    Red red;
};

namespace {

// Cholesky solve of the normal equations G g = c (G symmetric positive
// semidefinite, m x m row-major); false if a pivot falls below 1e-14 of
// the largest diagonal entry (then the history is dropped).
bool chol_solve(int m, std::vector<double> G, std::vector<double> c, double* g)
{
    double dmax = 0.0;
    for (int i = 0; i < m; ++i) dmax = std::max(dmax, G[i * m + i]);
    for (int j = 0; j < m; ++j) {
        double d = G[j * m + j];
        for (int k = 0; k < j; ++k) d -= G[j * m + k] * G[j * m + k];
        if (!(d > 1e-14 * dmax)) return false;
        const double l = sqrt(d);
        G[j * m + j] = l;
        for (int i = j + 1; i < m; ++i) {
            double s = G[i * m + j];
            for (int k = 0; k < j; ++k) s -= G[i * m + k] * G[j * m + k];
            G[i * m + j] = s / l;
        }
    }
    for (int i = 0; i < m; ++i) {                 // L y = c
        double s = c[i];
        for (int k = 0; k < i; ++k) s -= G[i * m + k] * c[k];
        c[i] = s / G[i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) {            // L^T g = y
        double s = c[i];
        for (int k = i + 1; k < m; ++k) s -= G[k * m + i] * g[k];
        g[i] = s / G[i * m + i];
    }
    return true;
}

}  // namespace

extern "C" {

int sq_poisson(sq_ctx* c, const double* rho, double* phi, double tol, int max_iter, int* iters_host,
               double* rel_resid_host)
{
    if (!c || !(tol > 0.0) || !(tol < 1.0) || max_iter < 0) return SQ_EINVAL;
    if (!device_ptr(rho) || !device_ptr(phi)) return SQ_EINVAL;
    const long long n = c->g.Nd;
    cudaStream_t st = c->stream;
    PoissonWS* ws = nullptr;
    int rcw = context_ws(c, &ws);
    if (rcw) return rcw;
    Red& R = ws->red;
    double* b = ws->buf;
    double* r = b + n;
    double* p = r + n;
    double* Ap = p + n;
    const int G = grid_for(n, c->sm_count);
    FDW fw;
    for (int d = 0; d <= FD_NO; ++d) fw.w[d] = c->g.w[d];
    // b = 4 pi (rho - mean(rho)), made exactly mean-free; |b| and |rho|
    int rc = enqueue_dot(R, rho, nullptr, nullptr, nullptr, n, 0, st);
    if (rc) return rc;
    rhs_kernel<<<G, 256, 0, st>>>(rho, R.out + 0, b, n);
    if ((rc = enqueue_dot(R, b, nullptr, nullptr, nullptr, n, 1, st))) return rc;
    shift_kernel<<<G, 256, 0, st>>>(b, R.out + 1, n);
    if ((rc = enqueue_dot(R, b, nullptr, b, nullptr, n, 2, st)) || (rc = enqueue_dot(R, rho, nullptr, rho, nullptr, n, 3, st)))
        return rc;
    c->launches += 6;
    double h4[4];
    if ((rc = read_slots(R, h4, 4, st))) return rc;
    double bnorm = sqrt(h4[2]);
    if (bnorm <= 1e-13 * 4.0 * M_PI * sqrt(h4[3])) bnorm = 0.0;   // neutral up to rounding
    if (cudaMemsetAsync(phi, 0, sizeof(double) * n, st) != cudaSuccess) return SQ_ECUDA;
    int it = 0;
    double rr = bnorm > 0.0 ? h4[2] : 0.0;
    if (bnorm > 0.0) {
        if (cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(p, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return SQ_ECUDA;
        while (sqrt(rr) > tol * bnorm && it < max_iter) {
            lap_periodic_kernel<<<G, 256, 0, st>>>(p, Ap, c->g.n1, c->g.n2, c->g.n3, fw);
            if ((rc = enqueue_dot(R, p, nullptr, Ap, nullptr, n, 4, st))) return rc;
            double pAp, rr_new;
            if ((rc = read_slot(R, 4, &pAp, st))) return rc;
            const double alpha = rr / pAp;
            cg_update_kernel<<<G, 256, 0, st>>>(phi, r, p, Ap, alpha, n);
            if ((rc = enqueue_dot(R, r, nullptr, r, nullptr, n, 5, st))) return rc;
            if ((rc = read_slot(R, 5, &rr_new, st))) return rc;
            xpby_kernel<<<G, 256, 0, st>>>(p, r, rr_new / rr, n);
            c->launches += 5;
            rr = rr_new;
            ++it;
        }
        if ((rc = enqueue_dot(R, phi, nullptr, nullptr, nullptr, n, 6, st))) return rc;   // phi mean-free
        shift_kernel<<<G, 256, 0, st>>>(phi, R.out + 6, n);
        c->launches += 2;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return SQ_ECUDA;
    if (iters_host) *iters_host = it;
    if (rel_resid_host) *rel_resid_host = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
    return (bnorm > 0.0 && sqrt(rr) > tol * bnorm) ? SQ_ENOCONV : SQ_OK;
}

int sq_widen_bounds(sq_ctx* c, const double* V, const double* V_ref, const double* chi_ref, const double* zeta_ref,
                    double* chi, double* zeta, double* w_host)
{
    if (!c) return SQ_EINVAL;
    if (!device_ptr(V) || !device_ptr(V_ref) || !device_ptr(chi_ref) || !device_ptr(zeta_ref) || !device_ptr(chi) ||
        !device_ptr(zeta))
        return SQ_EINVAL;
    PoissonWS* ws = nullptr;
    int rc = context_ws(c, &ws);
    if (rc) return rc;
    const long long n = c->g.Nd;
    maxabs_kernel<<<ws->red.blocks, T_RED, 0, c->stream>>>(V, V_ref, n, ws->red.partials, ws->red.counter,
                                                             ws->red.out);
    widen_kernel<<<grid_for(n, c->sm_count), 256, 0, c->stream>>>(chi_ref, zeta_ref, ws->red.out, chi, zeta, n);
    c->launches += 2;
    if (cudaGetLastError() != cudaSuccess) return SQ_ECUDA;
    double w = 0.0;
    if ((rc = read_slot(ws->red, 0, &w, c->stream))) return rc;
    if (!std::isfinite(w)) return SQ_EINVAL;
    if (w_host) *w_host = w;
    return SQ_OK;
}

int sq_effective_potential(sq_ctx* c, const double* V_loc, const double* phi, const double* rho, double alpha,
                           double* V_out)
{
    if (!c || !(alpha > 0.0) || !(alpha < 10.0)) return SQ_EINVAL;
    if (!device_ptr(V_loc) || !device_ptr(phi) || !device_ptr(rho) || !device_ptr(V_out)) return SQ_EINVAL;
    const long long n = c->g.Nd;
    veff_kernel<<<grid_for(n, c->sm_count), 256, 0, c->stream>>>(V_loc, phi, rho, alpha, V_out, n);
    c->launches++;
    return cudaGetLastError() == cudaSuccess ? SQ_OK : SQ_ECUDA;
}

int sq_kerker(sq_ctx* c, const double* v_in, const double* v_out, double k0, double amin, double tol, int max_iter,
              double* v_pre, double* rel_resid_host, int* iters_host)
{
    if (!c || !(k0 > 0.0) || !(amin > 0.0) || !(amin <= 1.0) || !(tol > 0.0) || !(tol < 1.0) || max_iter < 0)
        return SQ_EINVAL;
    if (!device_ptr(v_in) || !device_ptr(v_out) || !device_ptr(v_pre) || v_pre == v_in || v_pre == v_out)
        return SQ_EINVAL;
    const long long n = c->g.Nd;
    cudaStream_t st = c->stream;
    PoissonWS* ws = nullptr;
    int rc = context_ws(c, &ws);
    if (rc) return rc;
    Red& R = ws->red;
    double* f = ws->buf;
    double* r = f + n;
    double* p = r + n;
    double* Ap = p + n;
    double* u = v_pre;
    const int G = grid_for(n, c->sm_count);
    const double s = k0 * k0;
    FDW fw;
    for (int d = 0; d <= FD_NO; ++d) fw.w[d] = c->g.w[d];
    sub_kernel<<<G, 256, 0, st>>>(v_out, v_in, f, n);
    if ((rc = enqueue_dot(R, f, nullptr, f, nullptr, n, 0, st)) || (rc = enqueue_dot(R, v_out, nullptr, v_out, nullptr, n, 1, st)))
        return rc;
    c->launches += 3;
    double h2[2];
    if ((rc = read_slots(R, h2, 2, st))) return rc;
    const double fnorm = sqrt(h2[0]);
    if (rel_resid_host) *rel_resid_host = h2[1] > 0.0 ? fnorm / sqrt(h2[1]) : 0.0;
    if (cudaMemsetAsync(u, 0, sizeof(double) * n, st) != cudaSuccess ||
        cudaMemcpyAsync(r, f, sizeof(double) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(p, f, sizeof(double) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return SQ_ECUDA;
    double rr = h2[0];
    int it = 0;
    while (fnorm > 0.0 && sqrt(rr) > tol * fnorm && it < max_iter) {
        helmholtz_kernel<<<G, 256, 0, st>>>(p, Ap, c->g.n1, c->g.n2, c->g.n3, fw, s);
        if ((rc = enqueue_dot(R, p, nullptr, Ap, nullptr, n, 4, st))) return rc;
        double pAp, rr_new;
        if ((rc = read_slot(R, 4, &pAp, st))) return rc;
        const double alpha = rr / pAp;
        cg_update_kernel<<<G, 256, 0, st>>>(u, r, p, Ap, alpha, n);
        if ((rc = enqueue_dot(R, r, nullptr, r, nullptr, n, 5, st))) return rc;
        if ((rc = read_slot(R, 5, &rr_new, st))) return rc;
        xpby_kernel<<<G, 256, 0, st>>>(p, r, rr_new / rr, n);
        c->launches += 5;
        rr = rr_new;
        ++it;
    }
    kerker_out_kernel<<<G, 256, 0, st>>>(v_in, f, (1.0 - amin) * s, v_pre, n);
    c->launches++;
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return SQ_ECUDA;
    if (iters_host) *iters_host = it;
    return (fnorm > 0.0 && sqrt(rr) > tol * fnorm) ? SQ_ENOCONV : SQ_OK;
}

int sq_mixer_create(sq_mixer** out, long long n, int history, double beta, void* cuda_stream)
{
    if (!out) return SQ_EINVAL;
    *out = nullptr;
    if (n < 1 || history < 0 || history > MAX_HIST || !(beta > 0.0) || !(beta <= 1.0)) return SQ_EINVAL;
    sq_mixer* m = new (std::nothrow) sq_mixer();
    if (!m) return SQ_ENOMEM;
    m->n = n;
    m->hist = history;
    m->beta = beta;
    m->st = (cudaStream_t)cuda_stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&m->sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return SQ_ECUDA;
    }
    m->X.assign(history + 1, nullptr);
    m->F.assign(history + 1, nullptr);
    int rc = SQ_OK;
    for (int i = 0; i <= history && rc == SQ_OK; ++i)
        if (cudaMalloc(&m->X[i], sizeof(double) * n) != cudaSuccess || cudaMalloc(&m->F[i], sizeof(double) * n) != cudaSuccess)
            rc = SQ_ENOMEM;
    if (rc == SQ_OK) rc = red_alloc(m->red, m->sm, (MAX_HIST + 1) * (MAX_HIST + 2) / 2 + MAX_HIST + 4);
    if (rc) {
        cudaGetLastError();
        sq_mixer_destroy(m);
        return rc;
    }
    *out = m;
    return SQ_OK;
}

int sq_mixer_step(sq_mixer* m, const double* v_in, const double* v_out, double* v_next, double* rel_resid_host)
{
    if (!m || !device_ptr(v_in) || !device_ptr(v_out) || !device_ptr(v_next)) return SQ_EINVAL;
    const long long n = m->n;
    const int G = grid_for(n, m->sm);
    cudaStream_t st = m->st;
    // the newest slot: the oldest one is recycled once the history is full
    int slot;
    if ((int)m->order.size() < m->hist + 1) {
        slot = (int)m->order.size();
    } else {
        slot = m->order.front();
        m->order.erase(m->order.begin());
    }
    m->order.push_back(slot);
    if (cudaMemcpyAsync(m->X[slot], v_in, sizeof(double) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return SQ_ECUDA;
    sub_kernel<<<G, 256, 0, st>>>(v_out, v_in, m->F[slot], n);
    const int k = (int)m->order.size() - 1;      // differences available
    std::vector<const double*> Xo(k + 1), Fo(k + 1);
    for (int i = 0; i <= k; ++i) {
        Xo[i] = m->X[m->order[i]];
        Fo[i] = m->F[m->order[i]];
    }
    const double* f = Fo[k];
    // Periodic Pulay: extrapolate on steps period-1, 2 period-1, ...; simple mixing otherwise
    const bool pulay = (m->steps + 1) % m->period == 0;
    m->steps++;
    const int kd = pulay ? k : 0;                  // differences used
    // |f|^2, |v_out|^2, then dF_i . dF_j (i <= j) and dF_i . f
    int rc;
    if ((rc = enqueue_dot(m->red, f, nullptr, f, nullptr, n, 0, st)) ||
        (rc = enqueue_dot(m->red, v_out, nullptr, v_out, nullptr, n, 1, st)))
        return rc;
    int s = 2;
    for (int i = 0; i < kd; ++i) {
        if ((rc = enqueue_dot(m->red, Fo[i + 1], Fo[i], f, nullptr, n, s++, st))) return rc;
        for (int j = 0; j <= i; ++j)
            if ((rc = enqueue_dot(m->red, Fo[i + 1], Fo[i], Fo[j + 1], Fo[j], n, s++, st))) return rc;
    }
    std::vector<double> h(s);
    if ((rc = read_slots(m->red, h.data(), s, st))) return rc;
    if (rel_resid_host) *rel_resid_host = h[1] > 0.0 ? sqrt(h[0] / h[1]) : sqrt(h[0]);
    MixHist H = {};
    int used = kd;
    if (kd > 0) {
        std::vector<double> Gm(kd * kd), cv(kd);
        int t = 2;
        for (int i = 0; i < kd; ++i) {
            cv[i] = h[t++];
            for (int j = 0; j <= i; ++j) Gm[i * kd + j] = Gm[j * kd + i] = h[t++];
        }
        if (!chol_solve(kd, Gm, cv, H.g)) used = 0;   // drop the history (simple mixing)
    }
    for (int i = 0; i <= k; ++i) {
        H.X[i] = Xo[i];
        H.F[i] = Fo[i];
    }
    if (used == 0) {                                 // only the newest pair
        H.X[0] = Xo[k];
        H.F[0] = Fo[k];
    }
    mix_kernel<<<G, 256, 0, st>>>(H, used, m->beta, v_next, n);
    if (cudaGetLastError() != cudaSuccess) return SQ_ECUDA;
    return SQ_OK;
}

int sq_mixer_set_period(sq_mixer* m, int period, long long steps_done)
{
    if (!m || period < 1 || period > 1000 || steps_done < 0) return SQ_EINVAL;
    m->period = period;
    m->steps = steps_done;
    return SQ_OK;
}

int sq_mixer_history(const sq_mixer* m, int* count_host)
{
    if (!m || !count_host) return SQ_EINVAL;
    *count_host = (int)m->order.size();
    return SQ_OK;
}

int sq_mixer_export(sq_mixer* m, double* X_host, double* F_host)
{
    if (!m || (!m->order.empty() && (!X_host || !F_host))) return SQ_EINVAL;
    const size_t bytes = sizeof(double) * (size_t)m->n;
    for (size_t i = 0; i < m->order.size(); ++i)
        if (cudaMemcpyAsync(X_host + i * m->n, m->X[m->order[i]], bytes, cudaMemcpyDeviceToHost, m->st) != cudaSuccess ||
            cudaMemcpyAsync(F_host + i * m->n, m->F[m->order[i]], bytes, cudaMemcpyDeviceToHost, m->st) != cudaSuccess) {
            cudaGetLastError();
            return SQ_ECUDA;
        }
    if (cudaStreamSynchronize(m->st) != cudaSuccess) return SQ_ECUDA;
    return SQ_OK;
}

int sq_mixer_import(sq_mixer* m, int count, const double* X_host, const double* F_host)
{
    if (!m || count < 0 || count > m->hist + 1 || (count > 0 && (!X_host || !F_host))) return SQ_EINVAL;
    const size_t bytes = sizeof(double) * (size_t)m->n;
    m->order.clear();
    for (int i = 0; i < count; ++i) {
        if (cudaMemcpyAsync(m->X[i], X_host + (size_t)i * m->n, bytes, cudaMemcpyHostToDevice, m->st) != cudaSuccess ||
            cudaMemcpyAsync(m->F[i], F_host + (size_t)i * m->n, bytes, cudaMemcpyHostToDevice, m->st) != cudaSuccess) {
            cudaGetLastError();
            m->order.clear();
            return SQ_ECUDA;
        }
        m->order.push_back(i);
    }
    if (cudaStreamSynchronize(m->st) != cudaSuccess) return SQ_ECUDA;
    return SQ_OK;
}

int sq_mixer_reset(sq_mixer* m)
{
    if (!m) return SQ_EINVAL;
    m->order.clear();
    m->steps = 0;
    return SQ_OK;
}

void sq_mixer_destroy(sq_mixer* m)
{
    if (!m) return;
    for (double* p : m->X)
        if (p) cudaFree(p);
    for (double* p : m->F)
        if (p) cudaFree(p);
    red_free(m->red);
    delete m;
}

}  // extern "C"
