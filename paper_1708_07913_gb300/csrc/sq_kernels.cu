// sq_kernels.cu -- setup and FP64 post-processing kernels of libsq:
//   * potential copy with a periodic halo (Section 3.1 periodic index map)
//   * separable Gaussian projector tables (KB projectors restricted to the
//     region of influence, Section 3.1)
//   * extreme eigenvalues of the Lanczos tridiagonals (Section 3.2)
//   * quadrature weights by discrete orthogonality (Eq. cqj)
//   * Fermi level by bisection on the electron count (Section 3.2)
//   * density, band energy and entropy (Eqs. ElectronDensity, Eband, Entropy)
// Every global sum is deterministic: per-block tree sums in a fixed order,
// then the last block to finish adds the block partials in index order.
#include <math.h>
#include <algorithm>
#include "sq_internal.cuh"

namespace sq {

// ------------------------------------------------------------------------
// Potential with halo: Vp[k'][j'][i'] = V[(k'-m) mod n3][(j'-m) mod n2][(i'-m) mod n1]
// ------------------------------------------------------------------------
template <typename T>
__global__ void vpad_kernel(const double* __restrict__ V, T* __restrict__ Vp, int n1, int n2, int n3, int m,
                            unsigned* err)
{
    const long long tot = (long long)(n1 + 2 * m) * (n2 + 2 * m) * (n3 + 2 * m);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x)
        vpad_elem<T>(V, Vp, n1, n2, n3, m, t, err);
}

int launch_build_vpad(sq_ctx* ctx, const double* V)
{
    const GridParams& g = ctx->g;
    long long tot = (long long)g.P1 * g.P2 * (g.n3 + 2 * g.m);
    int blocks = (int)std::min<long long>((tot + 255) / 256, (long long)ctx->sm_count * 16);
    if (ctx->precision == SQ_FP32)
        vpad_kernel<float><<<blocks, 256, 0, ctx->stream>>>(V, (float*)ctx->Vp, g.n1, g.n2, g.n3, g.m, ctx->d_err);
    else
        vpad_kernel<double><<<blocks, 256, 0, ctx->stream>>>(V, (double*)ctx->Vp, g.n1, g.n2, g.n3, g.m, ctx->d_err);
    ctx->launches++;
    return cudaGetLastError() == cudaSuccess ? SQ_OK : SQ_ECUDA;
}

// ------------------------------------------------------------------------
// Projector tables.  For atom I at R with box start lo (atom-relative grid
// index) the displacement along axis a of box point i is d = (lo_a + i) h - R_a
// (rounded multiply then subtract, no FMA, so the support test below matches a
// plain evaluation of the same expression).  G = exp(-d^2/(2 rc^2)), DG = d G.
// Row (jj,kk) keeps the x-range of points with d_x^2 + d_y^2 + d_z^2 < r_nl^2.
// ------------------------------------------------------------------------
template <typename T>
__global__ void proj_table_kernel(const double* __restrict__ R, const AtomTab* __restrict__ at, int n_atoms,
                                  int lb, double h, double rc, double rnl2, T* G, T* DG, uint8_t* ivl)
{
    const int atom = blockIdx.x;
    if (atom >= n_atoms) return;
    const AtomTab A = at[atom];
    const double two_rc2 = 2.0 * rc * rc;
    for (int t = threadIdx.x; t < 3 * lb; t += blockDim.x) {
        int ax = t / lb, i = t % lb;
        double g = 0.0, dg = 0.0;
        if (i < A.len[ax]) {
            double d = __dadd_rn(__dmul_rn((double)(A.lo[ax] + i), h), -R[3 * atom + ax]);
            g = exp(-__dmul_rn(d, d) / two_rc2);
            dg = d * g;
        }
        G[((size_t)atom * 3 + ax) * lb + i] = (T)g;
        DG[((size_t)atom * 3 + ax) * lb + i] = (T)dg;
    }
    for (int t = threadIdx.x; t < lb * lb; t += blockDim.x) {
        int jj = t / lb, kk = t % lb;
        int xlo = 1, xhi = 0;
        if (jj < A.len[1] && kk < A.len[2]) {
            double dy = __dadd_rn(__dmul_rn((double)(A.lo[1] + jj), h), -R[3 * atom + 1]);
            double dz = __dadd_rn(__dmul_rn((double)(A.lo[2] + kk), h), -R[3 * atom + 2]);
            int first = -1, last = -1;
            for (int ii = 0; ii < A.len[0]; ++ii) {
                double dx = __dadd_rn(__dmul_rn((double)(A.lo[0] + ii), h), -R[3 * atom + 0]);
                double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                if (r2 < rnl2) {
                    if (first < 0) first = ii;
                    last = ii;
                }
            }
            if (first >= 0) { xlo = first; xhi = last; }
        }
        ivl[(((size_t)atom * lb + jj) * lb + kk) * 2 + 0] = (uint8_t)xlo;
        ivl[(((size_t)atom * lb + jj) * lb + kk) * 2 + 1] = (uint8_t)xhi;
    }
}

int launch_proj_tables(sq_ctx* ctx, const double* d_R)
{
    double rnl2 = ctx->rnl * ctx->rnl;
    if (ctx->precision == SQ_FP32)
        proj_table_kernel<float><<<ctx->n_atoms, 256, 0, ctx->stream>>>(
            d_R, ctx->d_atoms, ctx->n_atoms, ctx->lb, ctx->g.h, ctx->rc, rnl2, (float*)ctx->d_G, (float*)ctx->d_DG,
            ctx->d_ivl);
    else
        proj_table_kernel<double><<<ctx->n_atoms, 256, 0, ctx->stream>>>(
            d_R, ctx->d_atoms, ctx->n_atoms, ctx->lb, ctx->g.h, ctx->rc, rnl2, (double*)ctx->d_G, (double*)ctx->d_DG,
            ctx->d_ivl);
    ctx->launches++;
    return cudaGetLastError() == cudaSuccess ? SQ_OK : SQ_ECUDA;
}

// ------------------------------------------------------------------------
// Extreme eigenvalues of the Lanczos tridiagonal T_k by Sturm bisection.
// The count of eigenvalues below x is the number of sign changes of the
// leading principal minors p_0 = 1, p_i = (a_i - x) p_{i-1} - b_{i-1}^2 p_{i-2}
// (an exact zero takes the sign opposite to its predecessor).  Minors are
// rescaled by powers of two to stay in range; no division is needed.
// ------------------------------------------------------------------------
__device__ int sturm_count(int k, const double* a, const double* b, double x)
{
    double pm = 1.0, p = a[0] - x;
    int sprev = 1, cnt = 0;
    int s = (p > 0.0) ? 1 : (p < 0.0 ? -1 : -sprev);
    if (s != sprev) ++cnt;
    sprev = s;
    for (int i = 1; i < k; ++i) {
        double bb = b[i - 1] * b[i - 1];
        double pn = (a[i] - x) * p - bb * pm;
        pm = p;
        p = pn;
        s = (p > 0.0) ? 1 : (p < 0.0 ? -1 : -sprev);
        if (s != sprev) ++cnt;
        sprev = s;
        double ap = fabs(p), am = fabs(pm);
        if (ap > 0x1p+256 || am > 0x1p+256) { p *= 0x1p-256; pm *= 0x1p-256; }
        else if (ap < 0x1p-256 && am < 0x1p-256) { p *= 0x1p+256; pm *= 0x1p+256; }
    }
    return cnt;
}

__global__ void tridiag_bounds_kernel(const double* __restrict__ alpha, const double* __restrict__ beta,
                                      const int* __restrict__ klen, int cap, long long Nd, double margin,
                                      double* __restrict__ chi, double* __restrict__ zeta)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < Nd;
         q += (long long)gridDim.x * blockDim.x) {
        const double* a = alpha + q * cap;
        const double* b = beta + q * cap;
        int k = klen[q];
        double glo = INFINITY, ghi = -INFINITY;
        for (int i = 0; i < k; ++i) {
            double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < k - 1 ? fabs(b[i]) : 0.0);
            glo = fmin(glo, a[i] - r);
            ghi = fmax(ghi, a[i] + r);
        }
        double pad = 1e-12 * (fabs(glo) + fabs(ghi)) + 1e-300;
        glo -= pad;
        ghi += pad;
        double lo = glo, hi = ghi;
        for (int it = 0; it < 200; ++it) {
            double mid = 0.5 * (lo + hi);
            if (mid == lo || mid == hi) break;
            if (sturm_count(k, a, b, mid) >= 1) hi = mid; else lo = mid;
        }
        double tmin = 0.5 * (lo + hi);
        lo = glo;
        hi = ghi;
        for (int it = 0; it < 200; ++it) {
            double mid = 0.5 * (lo + hi);
            if (mid == lo || mid == hi) break;
            if (sturm_count(k, a, b, mid) >= k) hi = mid; else lo = mid;
        }
        double tmax = 0.5 * (lo + hi);
        double width = fmax(tmax - tmin, 1.0);
        double L = tmin - margin * width, H = tmax + margin * width;
        chi[q] = 0.5 * (H + L);
        zeta[q] = 0.5 * (H - L);
    }
}

int launch_tridiag_bounds(sq_ctx* ctx, double margin, double* chi, double* zeta)
{
    long long Nd = ctx->g.Nd;
    int blocks = (int)std::min<long long>((Nd + 127) / 128, (long long)ctx->sm_count * 16);
    tridiag_bounds_kernel<<<blocks, 128, 0, ctx->stream>>>(ctx->d_alpha, ctx->d_beta, ctx->d_klen, ctx->nl_cap,
                                                           Nd, margin, chi, zeta);
    ctx->launches++;
    return cudaGetLastError() == cudaSuccess ? SQ_OK : SQ_ECUDA;
}

// ------------------------------------------------------------------------
// Quadrature weights (Eq. cqj by discrete orthogonality at the zeros x_k of
// T_{npl+1}):  W_qk = (2/K) [ rho^0/2 + sum_{j>=1} rho^j T_j(x_k) ],  K = npl+1.
// T_j(x_k) by the three-term recurrence, tabulated per block in shared memory.
// ------------------------------------------------------------------------
__global__ void weights_kernel(const double* __restrict__ mom, double* __restrict__ W, long long Nd, int K,
                               int use_table)
{
    extern __shared__ double Ttab[];   // [K][K]: Ttab[j*K + k] = T_j(x_k)
    if (use_table) {
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            double x = cos(M_PI * (k + 0.5) / K);
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
        __syncthreads();
    }
    const long long tot = Nd * K;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < tot;
         idx += (long long)gridDim.x * blockDim.x) {
        long long q = idx / K;
        int k = (int)(idx % K);
        const double* r = mom + q * K;
        double s = 0.5 * r[0];
        if (use_table) {
            for (int j = 1; j < K; ++j) s += r[j] * Ttab[j * K + k];
        } else {
            double x = cos(M_PI * (k + 0.5) / K);
            double tm = 1.0, t = x;
            for (int j = 1; j < K; ++j) {
                s += r[j] * t;
                double tn = 2.0 * x * t - tm;
                tm = t;
                t = tn;
            }
        }
        W[idx] = 2.0 / K * s;
    }
}

int launch_weights(sq_ctx* ctx, const double* moments)
{
    int K = ctx->npl + 1;
    long long tot = ctx->g.Nd * K;
    size_t tbytes = (size_t)K * K * sizeof(double);
    int use_table = tbytes <= 96 * 1024;
    if (use_table && tbytes > 48 * 1024) {        // raise only (see the region kernels' dispatch)
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, weights_kernel) != cudaSuccess) return SQ_ECUDA;
        if ((int)tbytes > fa.maxDynamicSharedSizeBytes &&
            cudaFuncSetAttribute(weights_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tbytes) !=
                cudaSuccess)
            return SQ_ECUDA;
    }
    int blocks = (int)std::min<long long>((tot + 255) / 256, (long long)ctx->sm_count * 8);
    weights_kernel<<<blocks, 256, use_table ? tbytes : 0, ctx->stream>>>(moments, ctx->d_W, ctx->g.Nd, K,
                                                                         use_table);
    ctx->launches++;
    return cudaGetLastError() == cudaSuccess ? SQ_OK : SQ_ECUDA;
}

// ------------------------------------------------------------------------
// Deterministic grid reductions (last-block-done pattern).
// ------------------------------------------------------------------------
constexpr int RED_T = 256;

__device__ inline double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum NV doubles over the block; result valid in thread 0.
template <int NV>
__device__ inline void block_reduce(double (&v)[NV], double* sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = warp_sum_d(v[i]);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) sh[i * 32 + w] = v[i];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double t = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[i * 32 + k];
            v[i] = t;
        }
    }
}

// Fermi state layout (doubles)
enum { F_LO = 0, F_HI, F_NE, F_KT, F_NLO, F_NHI, F_DONE, F_ITERS, F_STATUS, F_EB, F_ES, F_NEL, F_NSTATE };
static_assert(F_NSTATE == FERMI_STATE, "Fermi state size");

// min(chi - zeta) - 10 kT and max(chi + zeta) + 10 kT
__global__ void fermi_bracket_kernel(const double* __restrict__ chi, const double* __restrict__ zeta, long long Nd,
                                     double* red, unsigned* count, double* st)
{
    __shared__ double sh[64];
    __shared__ bool last;
    double lo = INFINITY, hi = -INFINITY;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < Nd;
         q += (long long)gridDim.x * blockDim.x) {
        lo = fmin(lo, chi[q] - zeta[q]);
        hi = fmax(hi, chi[q] + zeta[q]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) { sh[threadIdx.x >> 5] = lo; sh[32 + (threadIdx.x >> 5)] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { lo = fmin(lo, sh[k]); hi = fmax(hi, sh[32 + k]); }
        red[2 * blockIdx.x] = lo;
        red[2 * blockIdx.x + 1] = hi;
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double L = INFINITY, H = -INFINITY;
        for (unsigned b = 0; b < gridDim.x; ++b) {
            L = fmin(L, ((volatile double*)red)[2 * b]);
            H = fmax(H, ((volatile double*)red)[2 * b + 1]);
        }
        st[F_LO] = L - 10.0 * st[F_KT];
        st[F_HI] = H + 10.0 * st[F_KT];
        st[F_DONE] = 0.0;
        st[F_ITERS] = 0.0;
        st[F_STATUS] = 0.0;
        *count = 0;
    }
}

// Electron count N(mu) = 2 sum_q sum_k W_qk g((chi_q + zeta_q x_k - mu)/kT).
// mode 0: N(lo); mode 1: N(hi) and bracket check; mode 2: one bisection step.
__global__ void fermi_count_kernel(const double* __restrict__ W, const double* __restrict__ chi,
                                   const double* __restrict__ zeta, long long Nd, int K, int mode, double* red,
                                   unsigned* count, double* st)
{
    __shared__ double sh[32];
    __shared__ bool last;
    const double lo = st[F_LO], hi = st[F_HI], kT = st[F_KT];
    double mu;
    if (mode == 0) mu = lo;
    else if (mode == 1) mu = hi;
    else {
        if (st[F_DONE] != 0.0) return;                 // uniform over the grid
        mu = 0.5 * (lo + hi);
        if (mu == lo || mu == hi) {                    // converged in FP64
            if (blockIdx.x == 0 && threadIdx.x == 0) st[F_DONE] = 1.0;
            return;
        }
    }
    __shared__ double xk[MAX_NPL + 1];
    for (int k = threadIdx.x; k < K; k += blockDim.x) xk[k] = cos(M_PI * (k + 0.5) / K);
    __syncthreads();
    double acc[1] = {0.0};
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < Nd;
         q += (long long)gridDim.x * blockDim.x) {
        const double c = chi[q], z = zeta[q];
        const double* w = W + q * K;
        double s = 0.0;
        for (int k = 0; k < K; ++k) {
            double t = (c + z * xk[k] - mu) / kT;
            // beyond |t| = 40 the Fermi factor is 1.0 exactly in FP64 (t < -40)
            // or below 4.3e-18 (t > 40, dropped: < 1e-16 of any count here)
            if (t > 40.0) continue;
            s += (t < -40.0) ? w[k] : w[k] / (1.0 + exp(t));
        }
        acc[0] += 2.0 * s;
    }
    block_reduce<1>(acc, sh);
    if (threadIdx.x == 0) {
        red[blockIdx.x] = acc[0];
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double N = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) N += ((volatile double*)red)[b];
        const double Ne = st[F_NE];
        if (mode == 0) st[F_NLO] = N;
        else if (mode == 1) {
            st[F_NHI] = N;
            if (!(st[F_NLO] <= Ne && N >= Ne)) { st[F_STATUS] = (double)SQ_ENOCONV; st[F_DONE] = 1.0; }
        } else {
            if (N < Ne) st[F_LO] = mu; else st[F_HI] = mu;
            st[F_ITERS] += 1.0;
            if (st[F_ITERS] >= 200.0) st[F_DONE] = 1.0;
        }
        *count = 0;
    }
}

// Bisection state reset (a kernel rather than a host copy, so the whole
// Fermi-level search can be captured in a CUDA graph).
__global__ void fermi_init_kernel(double* st, double Ne, double kT)
{
    if (threadIdx.x == 0) {
        for (int i = 0; i < F_NSTATE; ++i) st[i] = 0.0;
        st[F_NE] = Ne;
        st[F_KT] = kT;
    }
}

// Enqueue the whole Fermi-level search on ctx->stream (no host wait); the
// result stays in the device state: mu = (st[F_LO] + st[F_HI]) / 2, status
// in st[F_STATUS].
int enqueue_fermi(sq_ctx* ctx, const double* chi, const double* zeta, double Ne, double kT)
{
    const long long Nd = ctx->g.Nd;
    const int K = ctx->npl + 1;
    fermi_init_kernel<<<1, 32, 0, ctx->stream>>>(ctx->d_fermi, Ne, kT);
    ctx->launches++;
    const int blocks = ctx->red_blocks;
    fermi_bracket_kernel<<<blocks, RED_T, 0, ctx->stream>>>(chi, zeta, Nd, ctx->d_red, ctx->d_count, ctx->d_fermi);
    fermi_count_kernel<<<blocks, RED_T, 0, ctx->stream>>>(ctx->d_W, chi, zeta, Nd, K, 0, ctx->d_red, ctx->d_count,
                                                         ctx->d_fermi);
    fermi_count_kernel<<<blocks, RED_T, 0, ctx->stream>>>(ctx->d_W, chi, zeta, Nd, K, 1, ctx->d_red, ctx->d_count,
                                                         ctx->d_fermi);
    ctx->launches += 3;
    for (int it = 0; it < 201; ++it) {
        fermi_count_kernel<<<blocks, RED_T, 0, ctx->stream>>>(ctx->d_W, chi, zeta, Nd, K, 2, ctx->d_red,
                                                             ctx->d_count, ctx->d_fermi);
        ctx->launches++;
    }
    SQ_CUDA_TRY(cudaGetLastError());
    return SQ_OK;
}

int run_fermi(sq_ctx* ctx, const double* chi, const double* zeta, double Ne, double kT, double* mu)
{
    int rc = enqueue_fermi(ctx, chi, zeta, Ne, kT);
    if (rc) return rc;
    double st[F_NSTATE];
    SQ_CUDA_TRY(cudaMemcpyAsync(st, ctx->d_fermi, sizeof(st), cudaMemcpyDeviceToHost, ctx->stream));
    SQ_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (st[F_STATUS] != 0.0) return (int)st[F_STATUS];
    *mu = 0.5 * (st[F_LO] + st[F_HI]);
    return SQ_OK;
}

int fermi_result(const double* st_host, double* mu, double* eb, double* es, double* ne)
{
    if (mu) *mu = 0.5 * (st_host[F_LO] + st_host[F_HI]);
    if (eb) *eb = st_host[F_EB];
    if (es) *es = st_host[F_ES];
    if (ne) *ne = st_host[F_NEL];
    return st_host[F_STATUS] != 0.0 ? (int)st_host[F_STATUS] : SQ_OK;
}

// ------------------------------------------------------------------------
// Density, band energy, entropy, electron count at mu.
// ------------------------------------------------------------------------
__global__ void density_kernel(const double* __restrict__ W, const double* __restrict__ chi,
                               const double* __restrict__ zeta, long long Nd, int K, double mu, double kT, double h,
                               double* __restrict__ rho, double* red, unsigned* count, double* st, int mu_from_state)
{
    __shared__ double sh[96];
    __shared__ bool last;
    __shared__ double xk[MAX_NPL + 1];
    if (mu_from_state) mu = 0.5 * (((volatile double*)st)[F_LO] + ((volatile double*)st)[F_HI]);
    for (int k = threadIdx.x; k < K; k += blockDim.x) xk[k] = cos(M_PI * (k + 0.5) / K);
    __syncthreads();
    const double h3 = h * h * h;
    double acc[3] = {0.0, 0.0, 0.0};   // E_band, E_ent, N
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < Nd;
         q += (long long)gridDim.x * blockDim.x) {
        const double c = chi[q], z = zeta[q];
        const double* w = W + q * K;
        double r = 0.0, eb = 0.0, es = 0.0;
        for (int k = 0; k < K; ++k) {
            double E = c + z * xk[k];
            double t = (E - mu) / kT;
            if (t > 40.0) continue;                    // g < 4.3e-18: no density, energy or entropy
            double wk = w[k];
            if (t < -40.0) {                           // g == 1.0 exactly in FP64, entropy term 0
                r += wk;
                eb += 2.0 * wk * E;
                continue;
            }
            double g = 1.0 / (1.0 + exp(t));
            double gm = 1.0 / (1.0 + exp(-t));
            r += wk * g;
            eb += 2.0 * wk * E * g;
            double sf = 0.0;
            if (g > 0.0) sf += g * log(g);
            if (gm > 0.0) sf += gm * log(gm);
            es += 2.0 * kT * wk * sf;
        }
        double rq = 2.0 / h3 * r;
        rho[q] = rq;
        acc[0] += eb;
        acc[1] += es;
        acc[2] += h3 * rq;
    }
    block_reduce<3>(acc, sh);
    if (threadIdx.x == 0) {
        red[3 * blockIdx.x + 0] = acc[0];
        red[3 * blockIdx.x + 1] = acc[1];
        red[3 * blockIdx.x + 2] = acc[2];
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) {
            s0 += ((volatile double*)red)[3 * b + 0];
            s1 += ((volatile double*)red)[3 * b + 1];
            s2 += ((volatile double*)red)[3 * b + 2];
        }
        st[F_EB] = s0;
        st[F_ES] = s1;
        st[F_NEL] = s2;
        *count = 0;
    }
}

int enqueue_density(sq_ctx* ctx, const double* chi, const double* zeta, double mu, double kT, double* rho,
                    int mu_from_state)
{
    const int blocks = ctx->red_blocks;
    density_kernel<<<blocks, RED_T, 0, ctx->stream>>>(ctx->d_W, chi, zeta, ctx->g.Nd, ctx->npl + 1, mu, kT,
                                                     ctx->g.h, rho, ctx->d_red, ctx->d_count, ctx->d_fermi,
                                                     mu_from_state);
    ctx->launches++;
    SQ_CUDA_TRY(cudaGetLastError());
    return SQ_OK;
}

int run_density(sq_ctx* ctx, const double* chi, const double* zeta, double mu, double kT, double* rho,
                double* eb, double* es, double* ne)
{
    int rc = enqueue_density(ctx, chi, zeta, mu, kT, rho, 0);
    if (rc) return rc;
    double st[F_NSTATE];
    SQ_CUDA_TRY(cudaMemcpyAsync(st, ctx->d_fermi, sizeof(st), cudaMemcpyDeviceToHost, ctx->stream));
    SQ_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (eb) *eb = st[F_EB];
    if (es) *es = st[F_ES];
    if (ne) *ne = st[F_NEL];
    return SQ_OK;
}

}  // namespace sq
