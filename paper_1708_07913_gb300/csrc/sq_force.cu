// sq_force.cu -- host side of sq_nl_forces (include/sq.h): argument checks,
// the per-context force workspace, and the two launches: a per-node force
// kernel (by default the region form of sq_force_region.cuh, which runs the
// recurrence on the region kernels' machinery; the first form of
// sq_force.cuh where the region form does not fit, or with
// SQ_FORCE_KERNEL=legacy in the environment) and the fixed-order sum over
// its CTAs.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "sq_force.cuh"
#include "sq_force_region.cuh"

using namespace sq;

namespace sq {
int launch_build_vpad(sq_ctx* ctx, const double* V);
int force_region_config_f32(int m, size_t extra, int* bps, size_t* smem);
int force_region_config_f64(int m, size_t extra, int* bps, size_t* smem);
int force_region_launch_f32(int m, const ForceRegionArgs<float>& f, size_t extra, int blocks, cudaStream_t st);
int force_region_launch_f64(int m, const ForceRegionArgs<double>& f, size_t extra, int blocks, cudaStream_t st);
}

// Per-context scratch of the force kernel (created on first use, grown when
// needed, released with the context).
struct ForceWS {
    char* buf = nullptr;
    size_t bytes = 0;
};

namespace {

std::mutex g_force_mutex;
std::unordered_map<const sq_ctx*, ForceWS*> g_force_ws;

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

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Byte offsets of the per-CTA slices inside one CTA's part of the workspace.
struct ForceLayout {
    size_t vec, cand, clen, P, rowent, rown, cent, cstart, part, F, total;
};

ForceLayout force_layout(int S, int cap, int n_atoms, size_t tsz)
{
    ForceLayout L;
    const size_t S2 = (size_t)S * S, S3 = S2 * S;
    L.vec = 0;
    L.cand = L.vec + align256(tsz * 4 * S3);
    L.clen = L.cand + align256(sizeof(int4) * cap);
    L.P = L.clen + align256(sizeof(int) * cap);
    L.rowent = L.P + align256(tsz * 4 * cap);
    L.rown = L.rowent + align256(sizeof(int2) * S2 * FORCE_EPR);
    L.cent = L.rown + align256(sizeof(int) * S2);
    L.cstart = L.cent + align256(sizeof(int) * S2 * FORCE_EPR);
    L.part = L.cstart + align256(sizeof(int) * (cap + 1));
    L.F = L.part + align256(tsz * 4 * S2 * FORCE_EPR);
    L.total = L.F + align256(sizeof(double) * 3 * (size_t)n_atoms);
    return L;
}

// The central finite-difference gradient weights of Eq. (FD:Gradient):
//   wt_d = (-1)^{d+1} (n_o!)^2 / (h d (n_o-d)! (n_o+d)!),  d = 1..n_o.
void grad_weights(int no, double h, double* wt)
{
    double f[32];
    f[0] = 1.0;
    for (int i = 1; i < 32; ++i) f[i] = f[i - 1] * i;
    wt[0] = 0.0;
    for (int d = 1; d <= no; ++d) wt[d] = ((d & 1) ? 1.0 : -1.0) / (h * d) * f[no] * f[no] / (f[no - d] * f[no + d]);
}

void ws_release(ForceWS* w)
{
    if (!w) return;
    if (w->buf) cudaFree(w->buf);
    delete w;
}

// Arguments and launch of the force kernel in precision T (the context's
// recurrence precision), then the fixed-order sum over its CTAs.
// Grid and dynamic shared memory of the force kernel in precision T.  By
// default every recurrence vector is in per-CTA global scratch (it stays
// L1/L2 resident and measured faster); SQ_FORCE_SMEM=1 in the environment
// selects the in-place form, which keeps the current vector (S^3 values) in
// shared memory.  The dynamic shared-memory limit of the kernel is only ever
// raised.
template <typename T>
int force_config(sq_ctx* c, long long nq, bool* inplace, size_t* dyn, int* blocks)
{
    const int S = 2 * c->g.m + 1;
    const char* env = getenv("SQ_FORCE_SMEM");
    *inplace = env && env[0] == '1';
    *dyn = *inplace ? sizeof(T) * (size_t)S * S * S : 0;
    const void* fn = *inplace ? (const void*)nl_force_kernel<T, true> : (const void*)nl_force_kernel<T, false>;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
        cudaGetLastError();
        return SQ_ECUDA;
    }
    if ((int)*dyn > fa.maxDynamicSharedSizeBytes &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*dyn) != cudaSuccess) {
        cudaGetLastError();
        return SQ_EUNSUPPORTED;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, FORCE_NT, *dyn) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        return SQ_EUNSUPPORTED;
    }
    *blocks = (int)std::min<long long>(nq, (long long)std::min(occ, 2) * c->sm_count);
    return SQ_OK;
}

template <typename T>
int launch_force(sq_ctx* c, const ForceLayout& L, char* base, int blocks, bool inplace, size_t dyn,
                 const double* chi, const double* zeta, double mu, double kT, const long long* nodes, long long nq,
                 double* forces)
{
    ForceArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.g = c->g;
    a.lap[0] = (T)(-3.0 * c->g.w[0]);
    for (int d = 1; d <= FD_NO; ++d) a.lap[d] = (T)(-0.5 * c->g.w[d]);
    grad_weights(FD_NO, c->g.h, a.grad);
    a.Vp = (const T*)c->Vp;
    a.nl.n_atoms = c->n_atoms;
    a.nl.atoms = c->d_atoms;
    a.nl.lb = c->lb;
    a.nl.G = (const T*)c->d_G;
    a.nl.DG = (const T*)c->d_DG;
    a.nl.ivl = c->d_ivl;
    a.nl.tile_start = c->d_tile_start;
    a.nl.tile_cand = c->d_tile_cand;
    for (int i = 0; i < 3; ++i) a.nl.ntile[i] = c->ntile[i];
    a.nl.ccap = c->ccap;
    a.nl.smem = 0;
    const double h3 = c->g.h * c->g.h * c->g.h;
    const double As2 = pow(M_PI * c->rc * c->rc, -1.5);          // A_s^2
    const double Ap2 = 2.0 / (c->rc * c->rc) * As2;              // A_p^2
    a.nl.cs = (T)(c->has_s ? h3 * c->gamma_s * As2 : 0.0);
    a.nl.cp = (T)(c->has_p ? h3 * c->gamma_p * Ap2 : 0.0);
    a.chi = chi;
    a.zeta = zeta;
    a.mu = mu;
    a.kT = kT;
    a.npl = c->npl;
    a.nodes = nodes;
    a.nq = nq;
    // the per-CTA slices are grouped by kind: all CTAs' vectors, then all
    // candidate lists, ... (each kind contiguous, CTA b at offset b * size)
    a.vec = (T*)(base + L.vec * blocks);
    a.cand = (int4*)(base + L.cand * blocks);
    a.clen = (int*)(base + L.clen * blocks);
    a.P = (T*)(base + L.P * blocks);
    a.rowent = (int2*)(base + L.rowent * blocks);
    a.rown = (int*)(base + L.rown * blocks);
    a.cent = (int*)(base + L.cent * blocks);
    a.cstart = (int*)(base + L.cstart * blocks);
    a.part = (T*)(base + L.part * blocks);
    a.Fcta = (double*)(base + L.F * blocks);
    a.err = c->d_err;
    if (inplace) nl_force_kernel<T, true><<<blocks, FORCE_NT, dyn, c->stream>>>(a);
    else nl_force_kernel<T, false><<<blocks, FORCE_NT, 0, c->stream>>>(a);
    if (cudaGetLastError() != cudaSuccess) return SQ_ECUDA;
    const int n3 = 3 * c->n_atoms;
    force_sum_kernel<<<(n3 + 127) / 128, 128, 0, c->stream>>>(a.Fcta, blocks, n3, forces);
    return cudaGetLastError() == cudaSuccess ? SQ_OK : SQ_ECUDA;
}

// Per-CTA slices of the region form: D (S^3 in T), the (candidate, axis)
// contributions of one node, the CTA's force array.
struct RegionForceLayout {
    size_t D, fpart, F, total;
};

RegionForceLayout region_force_layout(int S, int n_atoms, size_t tsz)
{
    RegionForceLayout L;
    L.D = 0;
    L.fpart = align256(tsz * (size_t)S * S * S);
    L.F = L.fpart + align256(sizeof(double) * 3 * MAX_CAND);
    L.total = L.F + align256(sizeof(double) * 3 * (size_t)n_atoms);
    return L;
}

// Grid of the region form (0: not available for this context).
int region_force_blocks(sq_ctx* c, long long nq, size_t* extra)
{
    if (c->cl_nc > 0 || !c->d_scratch) return 0;        // the cluster kernels keep no per-CTA scratch
    const char* env = getenv("SQ_FORCE_KERNEL");
    if (env && strcmp(env, "legacy") == 0) return 0;
    *extra = force_coef_bytes(c->npl) + c->nl_extra;
    int bps = 0;
    size_t smem = 0;
    const int rc = c->precision == SQ_FP32 ? force_region_config_f32(c->g.m, *extra, &bps, &smem)
                                           : force_region_config_f64(c->g.m, *extra, &bps, &smem);
    if (rc || bps < 1) return 0;
    long long b = std::min<long long>((long long)bps * c->sm_count, c->grid_blocks);
    return (int)std::min<long long>(b, nq);
}

int force_region_launch(int m, const ForceRegionArgs<float>& f, size_t extra, int blocks, cudaStream_t st)
{
    return force_region_launch_f32(m, f, extra, blocks, st);
}
int force_region_launch(int m, const ForceRegionArgs<double>& f, size_t extra, int blocks, cudaStream_t st)
{
    return force_region_launch_f64(m, f, extra, blocks, st);
}

template <typename T>
int launch_force_region(sq_ctx* c, const RegionForceLayout& L, char* base, int blocks, size_t extra,
                        const double* chi, const double* zeta, double mu, double kT, const long long* nodes,
                        long long nq, double* forces)
{
    ForceRegionArgs<T> f;
    memset(&f, 0, sizeof(f));
    f.r = region_args<T>(c);
    f.r.chi = chi;
    f.r.zeta = zeta;
    grad_weights(FD_NO, c->g.h, f.grad);
    f.mu = mu;
    f.kT = kT;
    f.nodes = nodes;
    f.nq = nq;
    f.D = (T*)(base + L.D * blocks);
    f.fpart = (double*)(base + L.fpart * blocks);
    f.Fcta = (double*)(base + L.F * blocks);
    int rc = force_region_launch(c->g.m, f, extra, blocks, c->stream);
    if (rc) return rc;
    const int n3 = 3 * c->n_atoms;
    force_sum_kernel<<<(n3 + 127) / 128, 128, 0, c->stream>>>(f.Fcta, blocks, n3, forces);
    return cudaGetLastError() == cudaSuccess ? SQ_OK : SQ_ECUDA;
}

// The context's force workspace, at least `need` bytes.
int force_workspace(sq_ctx* c, size_t need, ForceWS** out)
{
    ForceWS* ws = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_force_mutex);
        auto it = g_force_ws.find(c);
        if (it != g_force_ws.end()) ws = it->second;
    }
    if (!ws || ws->bytes < need) {
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SQ_ECUDA;
        std::lock_guard<std::mutex> lk(g_force_mutex);
        auto it = g_force_ws.find(c);
        if (it != g_force_ws.end()) {
            ws_release(it->second);
            g_force_ws.erase(it);
        }
        ws = new (std::nothrow) ForceWS();
        if (!ws) return SQ_ENOMEM;
        if (cudaMalloc((void**)&ws->buf, need) != cudaSuccess) {
            cudaGetLastError();
            ws_release(ws);
            return SQ_ENOMEM;
        }
        ws->bytes = need;
        g_force_ws[c] = ws;
    }
    *out = ws;
    return SQ_OK;
}

}  // namespace

namespace sq {
// Called when a context is destroyed.
void free_force_ws(sq_ctx* c)
{
    std::lock_guard<std::mutex> lk(g_force_mutex);
    auto it = g_force_ws.find(c);
    if (it == g_force_ws.end()) return;
    ws_release(it->second);
    g_force_ws.erase(it);
}
}  // namespace sq

namespace {

int nl_forces(sq_ctx* c, const double* V, const double* chi, const double* zeta, double mu, double kT,
              const long long* nodes, long long n_nodes, double* forces)
{
    if (!c || !isfinite(mu) || !isfinite(kT) || kT <= 0.0) return SQ_EINVAL;
    if (!dev_ptr(V) || !dev_ptr(chi) || !dev_ptr(zeta)) return SQ_EINVAL;
    if (c->n_atoms > 0 && !dev_ptr(forces)) return SQ_EINVAL;
    if (nodes) {
        // the node list is checked on the host before anything is enqueued
        if (n_nodes < 1 || n_nodes > c->g.Nd || !dev_ptr(nodes)) return SQ_EINVAL;
        std::vector<long long> h((size_t)n_nodes);
        if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
            cudaMemcpy(h.data(), nodes, sizeof(long long) * n_nodes, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return SQ_ECUDA;
        }
        for (long long q : h)
            if (q < 0 || q >= c->g.Nd) return SQ_EINVAL;
    }
    const long long nq = nodes ? n_nodes : c->g.Nd;
    if (c->n_atoms == 0) return SQ_OK;
    const int n3 = 3 * c->n_atoms;
    if (!c->has_s && !c->has_p)
        return cudaMemsetAsync(forces, 0, sizeof(double) * n3, c->stream) == cudaSuccess ? SQ_OK : SQ_ECUDA;

    const int S = 2 * c->g.m + 1;
    const size_t tsz = c->precision == SQ_FP32 ? sizeof(float) : sizeof(double);
    ForceWS* ws = nullptr;
    int rc;
    size_t extra = 0;
    const int rblocks = region_force_blocks(c, nq, &extra);
    if (rblocks > 0) {
        const RegionForceLayout L = region_force_layout(S, c->n_atoms, tsz);
        if ((rc = force_workspace(c, L.total * (size_t)rblocks, &ws))) return rc;
        if ((rc = launch_build_vpad(c, V))) return rc;
        rc = c->precision == SQ_FP32
                 ? launch_force_region<float>(c, L, ws->buf, rblocks, extra, chi, zeta, mu, kT, nodes, nq, forces)
                 : launch_force_region<double>(c, L, ws->buf, rblocks, extra, chi, zeta, mu, kT, nodes, nq, forces);
    } else {
        const ForceLayout L = force_layout(S, c->ccap, c->n_atoms, tsz);
        bool inplace = true;
        size_t dyn = 0;
        int blocks = 0;
        int rcc = c->precision == SQ_FP32 ? force_config<float>(c, nq, &inplace, &dyn, &blocks)
                                          : force_config<double>(c, nq, &inplace, &dyn, &blocks);
        if (rcc) return rcc;
        if ((rc = force_workspace(c, L.total * (size_t)blocks, &ws))) return rc;
        if ((rc = launch_build_vpad(c, V))) return rc;
        rc = c->precision == SQ_FP32
                 ? launch_force<float>(c, L, ws->buf, blocks, inplace, dyn, chi, zeta, mu, kT, nodes, nq, forces)
                 : launch_force<double>(c, L, ws->buf, blocks, inplace, dyn, chi, zeta, mu, kT, nodes, nq, forces);
    }
    if (rc) return rc;
    c->launches += 2;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SQ_ECUDA;
    unsigned e = 0;
    if (cudaMemcpy(&e, c->d_err, sizeof(e), cudaMemcpyDeviceToHost) != cudaSuccess) return SQ_ECUDA;
    if (e) {
        unsigned z = 0;
        if (cudaMemcpy(c->d_err, &z, sizeof(z), cudaMemcpyHostToDevice) != cudaSuccess) return SQ_ECUDA;
        return (e & ERR_CAPACITY) ? SQ_ECAPACITY : SQ_EBOUNDS;
    }
    return SQ_OK;
}

}  // namespace

extern "C" int sq_nl_forces(sq_ctx* c, const double* V, const double* chi, const double* zeta, double mu, double kT,
                            double* forces)
{
    return nl_forces(c, V, chi, zeta, mu, kT, nullptr, 0, forces);
}

extern "C" int sq_nl_forces_nodes(sq_ctx* c, const double* V, const double* chi, const double* zeta, double mu,
                                  double kT, const long long* nodes, long long n_nodes, double* forces)
{
    if (!nodes) return SQ_EINVAL;
    return nl_forces(c, V, chi, zeta, mu, kT, nodes, n_nodes, forces);
}
