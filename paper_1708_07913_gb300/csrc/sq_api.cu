// sq_api.cu -- host side of the libsq C ABI (include/sq.h): argument
// validation, context set-up (device tables, per-CTA scratch), and the
// enqueueing of the kernels for each step of the Spectral Quadrature path.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "sq_queue.cuh"

namespace sq {
int region_config_f32(int m, int which, size_t extra, int* bps, size_t* smem);
int region_config_f64(int m, int which, size_t extra, int* bps, size_t* smem);
int region_launch_f32(int m, int which, const RegionArgs<float>& a, size_t extra, int blocks, cudaStream_t st);
int region_launch_f64(int m, int which, const RegionArgs<double>& a, size_t extra, int blocks, cudaStream_t st);
int cluster_nc(int m);
int cluster_config_f32_lo(int m, int which, int ccap, int npl, int* clusters, size_t* smem);
int cluster_config_f32_hi(int m, int which, int ccap, int npl, int* clusters, size_t* smem);
int cluster_launch_f32_lo(int m, int which, const RegionArgs<float>& a, int clusters, size_t smem, cudaStream_t st);
int cluster_launch_f32_hi(int m, int which, const RegionArgs<float>& a, int clusters, size_t smem, cudaStream_t st);
int queue_config_f32(int m, int which, size_t extra, int* bps, size_t* smem);
int queue_config_f64(int m, int which, size_t extra, int* bps, size_t* smem);
int queue_launch_f32(int m, int which, const QueueArgs<float>& q, size_t extra, int blocks, cudaStream_t st);
int queue_launch_f64(int m, int which, const QueueArgs<double>& q, size_t extra, int blocks, cudaStream_t st);
}  // namespace sq

using namespace sq;

namespace sq {
void free_poisson_ws(sq_ctx* ctx);   // sq_scf.cu: the context's Poisson workspace
void free_force_ws(sq_ctx* ctx);     // sq_force.cu: the context's force workspace
}

namespace {

bool is_fin(double x) { return std::isfinite(x); }

// A device pointer the GPU can dereference (device or managed memory).
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

// Central finite-difference weights of the paper's Eq. (FD:Laplacian):
//   w_0 = -(1/h^2) sum_{q=1}^{n_o} q^-2,
//   w_d = 2 (-1)^{d+1} (n_o!)^2 / (h^2 d^2 (n_o-d)! (n_o+d)!).
void fd_weights(int no, double h, double* w)
{
    double f[32];
    f[0] = 1.0;
    for (int i = 1; i < 32; ++i) f[i] = f[i - 1] * i;
    double s = 0.0;
    for (int q = 1; q <= no; ++q) s += 1.0 / ((double)q * q);
    w[0] = -s / (h * h);
    for (int d = 1; d <= no; ++d)
        w[d] = ((d & 1) ? 2.0 : -2.0) / (h * h * d * d) * f[no] * f[no] / (f[no - d] * f[no + d]);
}

template <typename P>
int dev_alloc(P** p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 256;
    if (cudaMalloc((void**)p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return SQ_ENOMEM;
    }
    return SQ_OK;
}

void free_ctx(sq_ctx* c)
{
    if (!c) return;
    void* ptrs[] = {c->Vp, c->d_atoms, c->d_G, c->d_DG, c->d_ivl, c->d_tile_start, c->d_tile_cand, c->d_scratch,
                    c->d_alpha, c->d_beta, c->d_klen, c->d_W, c->d_red, c->d_fermi, c->d_count, c->d_err};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    free_poisson_ws(c);
    free_force_ws(c);
    delete c;
}

// Latched device error bits -> status (and clear them).  Synchronises.
int take_device_error(sq_ctx* c)
{
    unsigned e = 0;
    if (cudaMemcpyAsync(&e, c->d_err, sizeof(e), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) return SQ_ECUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SQ_ECUDA;
    if (e == 0) return SQ_OK;
    unsigned z = 0;
    if (cudaMemcpyAsync(c->d_err, &z, sizeof(z), cudaMemcpyHostToDevice, c->stream) != cudaSuccess) return SQ_ECUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SQ_ECUDA;
    if (e & ERR_TIMEOUT) return SQ_ETIMEOUT;
    if (e & ERR_NONFINITE) return SQ_EINVAL;
    if (e & ERR_CAPACITY) return SQ_ECAPACITY;
    return SQ_EBOUNDS;
}

// Projector geometry and tile candidate lists (host integer bookkeeping; the
// Gaussian tables themselves are evaluated on the device).
int setup_projectors(sq_ctx* c, const double* xyz)
{
    const GridParams& g = c->g;
    const int n[3] = {g.n1, g.n2, g.n3};
    const int m = g.m;
    std::vector<AtomTab> at(c->n_atoms);
    for (int I = 0; I < c->n_atoms; ++I) {
        for (int a = 0; a < 3; ++a) {
            double R = xyz[3 * I + a];
            int lo = (int)ceil((R - c->rnl) / g.h);
            int hi = (int)floor((R + c->rnl) / g.h);
            if (hi < lo) hi = lo - 1;
            at[I].lo[a] = lo;
            at[I].len[a] = hi - lo + 1;
            if (at[I].len[a] > NL_BOX) return SQ_EUNSUPPORTED;
            c->lb = std::max(c->lb, at[I].len[a]);
        }
    }
    if (c->lb < 1) c->lb = 1;
    for (int a = 0; a < 3; ++a) c->ntile[a] = (n[a] + TILE - 1) / TILE;
    const long long ntiles = (long long)c->ntile[0] * c->ntile[1] * c->ntile[2];
    // (tile, atom, box start) records; tiles meet a box iff the union of
    // their nodes' regions, [t*TILE - m, t*TILE + TILE - 1 + m], meets it
    struct Rec { long long tile; int atom, bx, by, bz; };
    std::vector<Rec> recs;
    for (int I = 0; I < c->n_atoms; ++I) {
        if (at[I].len[0] <= 0 || at[I].len[1] <= 0 || at[I].len[2] <= 0) continue;
        std::vector<std::pair<int, int>> axis[3];   // (box start, tile)
        for (int a = 0; a < 3; ++a) {
            int E = (m + NL_BOX + TILE) / n[a] + 2;
            for (int e = -E; e <= E; ++e) {
                int b0 = at[I].lo[a] + e * n[a], b1 = b0 + at[I].len[a] - 1;
                for (int t = 0; t < c->ntile[a]; ++t) {
                    int u0 = t * TILE - m, u1 = std::min(t * TILE + TILE, n[a]) - 1 + m;
                    if (b0 <= u1 && b1 >= u0) axis[a].push_back({b0, t});
                }
            }
        }
        for (auto& z : axis[2])
            for (auto& y : axis[1])
                for (auto& x : axis[0]) {
                    long long tile = x.second + (long long)c->ntile[0] * (y.second + (long long)c->ntile[1] * z.second);
                    recs.push_back({tile, I, x.first, y.first, z.first});
                }
    }
    std::vector<int> start(ntiles + 1, 0);
    for (auto& r : recs) start[r.tile + 1]++;
    for (long long t = 0; t < ntiles; ++t) start[t + 1] += start[t];
    std::vector<int4> cand(recs.size());
    std::vector<int> fill(start.begin(), start.end() - 1);
    for (auto& r : recs) cand[fill[r.tile]++] = make_int4(r.atom, r.bx, r.by, r.bz);   // stable: atom order

    // Largest number of candidates of any node: per tile, a 3-D difference
    // array over the tile's node offsets counts, for every node, the boxes
    // that meet its region (node i meets box [b0, b1] iff b0 - m <= i <= b1 + m).
    c->ccap = 0;
    {
        const int W = TILE + 1;
        std::vector<int> D(W * W * W);
        for (int tz = 0; tz < c->ntile[2]; ++tz)
            for (int ty = 0; ty < c->ntile[1]; ++ty)
                for (int tx = 0; tx < c->ntile[0]; ++tx) {
                    long long tile = tx + (long long)c->ntile[0] * (ty + (long long)c->ntile[1] * tz);
                    std::fill(D.begin(), D.end(), 0);
                    const int t0[3] = {tx * TILE, ty * TILE, tz * TILE};
                    for (int k = start[tile]; k < start[tile + 1]; ++k) {
                        const int4 cd = cand[k];
                        const int b0[3] = {cd.y, cd.z, cd.w};
                        int lo[3], hi[3];
                        bool empty = false;
                        for (int a = 0; a < 3; ++a) {
                            int l = std::max(b0[a] - m, t0[a]);
                            int h = std::min(b0[a] + at[cd.x].len[a] - 1 + m, std::min(t0[a] + TILE, n[a]) - 1);
                            lo[a] = l - t0[a];
                            hi[a] = h - t0[a];
                            if (h < l) empty = true;
                        }
                        if (empty) continue;
                        auto add = [&](int x, int y, int z, int v) { D[x + W * (y + W * z)] += v; };
                        add(lo[0], lo[1], lo[2], 1);
                        add(hi[0] + 1, lo[1], lo[2], -1);
                        add(lo[0], hi[1] + 1, lo[2], -1);
                        add(lo[0], lo[1], hi[2] + 1, -1);
                        add(hi[0] + 1, hi[1] + 1, lo[2], 1);
                        add(hi[0] + 1, lo[1], hi[2] + 1, 1);
                        add(lo[0], hi[1] + 1, hi[2] + 1, 1);
                        add(hi[0] + 1, hi[1] + 1, hi[2] + 1, -1);
                    }
                    for (int z = 0; z < W; ++z)              // prefix sums along x, y, z
                        for (int y = 0; y < W; ++y)
                            for (int x = 1; x < W; ++x) D[x + W * (y + W * z)] += D[x - 1 + W * (y + W * z)];
                    for (int z = 0; z < W; ++z)
                        for (int y = 1; y < W; ++y)
                            for (int x = 0; x < W; ++x) D[x + W * (y + W * z)] += D[x + W * (y - 1 + W * z)];
                    for (int z = 1; z < W; ++z)
                        for (int y = 0; y < W; ++y)
                            for (int x = 0; x < W; ++x) D[x + W * (y + W * z)] += D[x + W * (y + W * (z - 1))];
                    for (int z = 0; z < TILE; ++z)
                        for (int y = 0; y < TILE; ++y)
                            for (int x = 0; x < TILE; ++x) c->ccap = std::max(c->ccap, D[x + W * (y + W * z)]);
                }
    }
    if (c->ccap > MAX_CAND) return SQ_ECAPACITY;
    if (c->ccap < 1) c->ccap = 1;

    int rc;
    size_t tsz = c->precision == SQ_FP32 ? sizeof(float) : sizeof(double);
    if ((rc = dev_alloc(&c->d_atoms, sizeof(AtomTab) * at.size()))) return rc;
    if ((rc = dev_alloc(&c->d_G, tsz * 3 * c->lb * at.size()))) return rc;
    if ((rc = dev_alloc(&c->d_DG, tsz * 3 * c->lb * at.size()))) return rc;
    if ((rc = dev_alloc(&c->d_ivl, (size_t)c->lb * c->lb * 2 * at.size()))) return rc;
    if ((rc = dev_alloc(&c->d_tile_start, sizeof(int) * start.size()))) return rc;
    if ((rc = dev_alloc(&c->d_tile_cand, sizeof(int4) * std::max<size_t>(cand.size(), 1)))) return rc;
    double* d_R = nullptr;
    if ((rc = dev_alloc(&d_R, sizeof(double) * 3 * at.size()))) return rc;
    SQ_CUDA_TRY(cudaMemcpy(c->d_atoms, at.data(), sizeof(AtomTab) * at.size(), cudaMemcpyHostToDevice));
    SQ_CUDA_TRY(cudaMemcpy(c->d_tile_start, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice));
    if (!cand.empty())
        SQ_CUDA_TRY(cudaMemcpy(c->d_tile_cand, cand.data(), sizeof(int4) * cand.size(), cudaMemcpyHostToDevice));
    SQ_CUDA_TRY(cudaMemcpy(d_R, xyz, sizeof(double) * 3 * at.size(), cudaMemcpyHostToDevice));
    rc = launch_proj_tables(c, d_R);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    cudaFree(d_R);
    if (rc) return rc;
    return e == cudaSuccess ? SQ_OK : SQ_ECUDA;
}


// FP32 cluster kernels (sq_cluster.cuh) for this context when
// SQ_REGION_KERNEL=cluster is set in the environment, its region size has
// one and its projector candidates fit; otherwise the single-CTA kernels,
// which measure faster on the benchmark workloads.  Sets c->cl_nc (0: none).
int select_cluster_kernels(sq_ctx* c)
{
    c->cl_nc = 0;
    if (c->precision != SQ_FP32 || cluster_nc(c->g.m) == 0) return SQ_OK;
    const char* env = getenv("SQ_REGION_KERNEL");
    if (!env || strcmp(env, "cluster") != 0) return SQ_OK;
    const int ccap = c->ccap;                               // the kernels size their tables by it too
    for (int which = 0; which < 2; ++which) {
        const int rc = c->g.m <= 9 ? cluster_config_f32_lo(c->g.m, which, ccap, c->npl, &c->cl_clusters[which],
                                                           &c->cl_smem[which])
                                   : cluster_config_f32_hi(c->g.m, which, ccap, c->npl, &c->cl_clusters[which],
                                                           &c->cl_smem[which]);
        if (rc == SQ_EUNSUPPORTED) return SQ_OK;           // candidates do not fit: single-CTA kernels
        if (rc) return rc;
    }
    c->cl_nc = cluster_nc(c->g.m);
    return SQ_OK;
}

// Launch a cluster kernel on `blocks` CTAs (rounded down to whole clusters).
int cluster_launch(sq_ctx* c, int which, const RegionArgs<float>& a, int blocks)
{
    const int clusters = std::max(1, blocks / c->cl_nc);
    return c->g.m <= 9 ? cluster_launch_f32_lo(c->g.m, which, a, clusters, c->cl_smem[which], c->stream)
                       : cluster_launch_f32_hi(c->g.m, which, a, clusters, c->cl_smem[which], c->stream);
}

// Dynamic shared memory beyond the region vectors: the moments kernel (which
// = 0) keeps its per-node moment sums there; both keep the projector tables
// there when they fit.
size_t region_extra(const sq_ctx* c, int which)
{
    return (which == 0 ? mom_smem_bytes(c->npl) : 0) + c->nl_extra;
}

int region_blocks(sq_ctx* c, int which, int* blocks)
{
    if (c->cl_nc > 0) {                  // cluster kernels: CTAs of every resident cluster
        long long b = (long long)c->cl_clusters[which] * c->cl_nc;
        if (b > c->g.Nd * c->cl_nc) b = c->g.Nd * c->cl_nc;
        *blocks = (int)b;
        return SQ_OK;
    }
    int bps = 0;
    size_t smem = 0;
    int rc = c->precision == SQ_FP32 ? region_config_f32(c->g.m, which, region_extra(c, which), &bps, &smem)
                                     : region_config_f64(c->g.m, which, region_extra(c, which), &bps, &smem);
    if (rc) return rc;
    long long b = (long long)bps * c->sm_count;
    if (b > c->g.Nd) b = c->g.Nd;
    *blocks = (int)b;
    return SQ_OK;
}

// Lanczos coefficient buffers for n_lanczos steps (allocated outside any
// stream capture).
int ensure_lanczos_buffers(sq_ctx* c, int n_lanczos)
{
    if (n_lanczos <= c->nl_cap) return SQ_OK;
    if (c->d_alpha) cudaFree(c->d_alpha);
    if (c->d_beta) cudaFree(c->d_beta);
    if (c->d_klen) cudaFree(c->d_klen);
    c->d_alpha = c->d_beta = nullptr;
    c->d_klen = nullptr;
    c->nl_cap = 0;
    int rc;
    if ((rc = dev_alloc(&c->d_alpha, sizeof(double) * c->g.Nd * n_lanczos)) ||
        (rc = dev_alloc(&c->d_beta, sizeof(double) * c->g.Nd * n_lanczos)) ||
        (rc = dev_alloc(&c->d_klen, sizeof(int) * c->g.Nd)))
        return rc;
    c->nl_cap = n_lanczos;
    return SQ_OK;
}

// Lanczos kernel on `blocks` CTAs, then the tridiagonal extremes (Vp built).
int enqueue_bounds(sq_ctx* c, int blocks, int n_lanczos, double margin, double* chi, double* zeta)
{
    int rc;
    if (c->precision == SQ_FP32) {
        RegionArgs<float> a = region_args<float>(c);
        a.n_lanczos = n_lanczos; a.nl_cap = c->nl_cap; a.alpha = c->d_alpha; a.beta = c->d_beta; a.klen = c->d_klen;
        rc = c->cl_nc > 0 ? cluster_launch(c, 1, a, blocks)
                          : region_launch_f32(c->g.m, 1, a, region_extra(c, 1), blocks, c->stream);
    } else {
        RegionArgs<double> a = region_args<double>(c);
        a.n_lanczos = n_lanczos; a.nl_cap = c->nl_cap; a.alpha = c->d_alpha; a.beta = c->d_beta; a.klen = c->d_klen;
        rc = region_launch_f64(c->g.m, 1, a, region_extra(c, 1), blocks, c->stream);
    }
    c->launches++;
    if (rc) return rc;
    return launch_tridiag_bounds(c, margin, chi, zeta);
}

// Moments kernel on `blocks` CTAs (Vp built).
int enqueue_moments(sq_ctx* c, int blocks, const double* chi, const double* zeta, double* moments)
{
    int rc;
    if (c->precision == SQ_FP32) {
        RegionArgs<float> a = region_args<float>(c);
        a.chi = chi; a.zeta = zeta; a.moments = moments;
        rc = c->cl_nc > 0 ? cluster_launch(c, 0, a, blocks)
                          : region_launch_f32(c->g.m, 0, a, region_extra(c, 0), blocks, c->stream);
    } else {
        RegionArgs<double> a = region_args<double>(c);
        a.chi = chi; a.zeta = zeta; a.moments = moments;
        rc = region_launch_f64(c->g.m, 0, a, region_extra(c, 0), blocks, c->stream);
    }
    c->launches++;
    return rc;
}

}  // namespace

// ------------------------------------------------------------------------
// Batch of independent systems: the whole SCF-iteration step of every
// context as one CUDA graph, one forked stream per system.
// ------------------------------------------------------------------------
struct sq_batch {
    int n = 0;
    std::vector<sq_ctx*> ctx;
    cudaStream_t stream = nullptr;               // the caller's stream (may be the legacy stream)
    cudaStream_t own = nullptr;                  // the batch's stream: captures and launches (owned)
    std::vector<cudaStream_t> st;                // one per system (owned)
    cudaEvent_t fork = nullptr, ev_in = nullptr, ev_out = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraphExec_t exec = nullptr;
    std::vector<int> blocks;                     // region-kernel grid per system (0: the default)
    bool tuned = false;
    // arguments the instantiated graph was captured with
    std::vector<const void*> key_ptr;
    std::vector<double> key_val;
    int key_nl = 0;
    double key_margin = -1.0;
    std::vector<double> state;                   // host copy of the Fermi/energy states
    // launch plan: requested (SQ_BATCH_AUTO: tuned on the first run) and in use
    int plan_req = SQ_BATCH_AUTO, npi_req = 1;
    int plan = SQ_BATCH_STREAMS, npi = 1;
    long long wait_budget = 2000000000LL;        // SM cycles per queue wait (about a second)
    int wait_unset = 0;
    // queue plan: groups of systems with one region half-width and precision
    struct Group {
        int m = 0, prec = SQ_FP32;
        std::vector<int> sys;                    // batch indices, at most QMAX
        int bl = 0, bm = 0;                      // grids of the Lanczos and moments queue kernels
        size_t xl = 0, xm = 0;                   // their dynamic shared memory beyond the region vectors
        int off_l = 0, n_l = 0, off_m = 0, n_m = 0;   // item ranges in d_items
        std::vector<int> need;                   // QI_VPAD items per system
    };
    std::vector<Group> groups;
    int groups_npi = 0;                          // nodes per item the groups were built for (0: none)
    QItem* d_items = nullptr;
    unsigned* d_ctl = nullptr;                   // per group: 2 counters + QMAX completion counts
    std::vector<cudaEvent_t> gfork;
};

namespace {

void batch_free_graph(sq_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

void batch_free_queue(sq_batch* b)
{
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_ctl) cudaFree(b->d_ctl);
    b->d_items = nullptr;
    b->d_ctl = nullptr;
    for (cudaEvent_t e : b->gfork)
        if (e) cudaEventDestroy(e);
    b->gfork.clear();
    b->groups.clear();
    b->groups_npi = 0;
}

struct BatchArgs {
    const double* const* V;
    double* const* chi;
    double* const* zeta;
    double* const* moments;
    double* const* rho;
    const double* Ne;
    const double* kT;
    int n_lanczos;
    double margin;
};

// Enqueue the whole step of system i on the current stream of its context
// (bl, bm: grids of the Lanczos and moments kernels).
int batch_enqueue_one(sq_batch* b, int i, const BatchArgs& A, int bl, int bm)
{
    sq_ctx* c = b->ctx[i];
    int rc;
    if ((rc = launch_build_vpad(c, A.V[i]))) return rc;
    if ((rc = enqueue_bounds(c, bl, A.n_lanczos, A.margin, A.chi[i], A.zeta[i]))) return rc;
    if ((rc = enqueue_moments(c, bm, A.chi[i], A.zeta[i], A.moments[i]))) return rc;
    if ((rc = launch_weights(c, A.moments[i]))) return rc;
    if ((rc = enqueue_fermi(c, A.chi[i], A.zeta[i], A.Ne[i], A.kT[i]))) return rc;
    return enqueue_density(c, A.chi[i], A.zeta[i], 0.0, A.kT[i], A.rho[i], 1);
}

// Capture every system's step, each on its own stream forked from and
// joined back into b->stream, and instantiate the graph.
int batch_capture_streams(sq_batch* b, const BatchArgs& A, const std::vector<int>& blocks, cudaGraphExec_t* out)
{
    // grids first: nothing but stream work happens inside the capture
    std::vector<int> bl(b->n), bm(b->n);
    for (int i = 0; i < b->n; ++i) {
        int rc;
        if ((rc = region_blocks(b->ctx[i], 1, &bl[i])) || (rc = region_blocks(b->ctx[i], 0, &bm[i]))) return rc;
        if (blocks[i] > 0) {
            bl[i] = std::min(bl[i], blocks[i]);
            bm[i] = std::min(bm[i], blocks[i]);
        }
    }
    std::vector<cudaStream_t> saved(b->n);
    for (int i = 0; i < b->n; ++i) saved[i] = b->ctx[i]->stream;
    if (cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return SQ_ECUDA;
    }
    int rc = SQ_OK;
    if (cudaEventRecord(b->fork, b->own) != cudaSuccess) rc = SQ_ECUDA;
    for (int i = 0; i < b->n && rc == SQ_OK; ++i) {
        b->ctx[i]->stream = b->st[i];
        if (cudaStreamWaitEvent(b->st[i], b->fork, 0) != cudaSuccess) { rc = SQ_ECUDA; break; }
        rc = batch_enqueue_one(b, i, A, bl[i], bm[i]);
        if (rc) break;
        if (cudaEventRecord(b->join[i], b->st[i]) != cudaSuccess ||
            cudaStreamWaitEvent(b->own, b->join[i], 0) != cudaSuccess)
            rc = SQ_ECUDA;
    }
    for (int i = 0; i < b->n; ++i) b->ctx[i]->stream = saved[i];
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->own, &graph);
    if (rc == SQ_OK && e != cudaSuccess) rc = SQ_ECUDA;
    if (rc == SQ_OK && cudaGraphInstantiate(out, graph, 0) != cudaSuccess) rc = SQ_ECUDA;
    if (graph) cudaGraphDestroy(graph);
    if (rc) cudaGetLastError();
    return rc;
}

// Projector supports covering a point (atom density x support volume): the
// nonlocal share of a region point's arithmetic is about 8 flops per support
// against ~52 for the local stencil.
double proj_pairs(const sq_ctx* c)
{
    const double cell = (double)c->g.Nd * c->g.h * c->g.h * c->g.h;
    return (c->has_s || c->has_p) ? c->n_atoms * (4.0 / 3.0) * M_PI * c->rnl * c->rnl * c->rnl / cell : 0.0;
}

// Per-CTA scratch for at least `blocks` CTAs (a queue kernel's grid can be
// larger than the context's own, e.g. for a system with few nodes).
// cudaFree synchronises the device, so no kernel still uses the old slices.
int ensure_scratch(sq_ctx* c, int blocks)
{
    if (blocks <= c->grid_blocks) return SQ_OK;
    void* p = nullptr;
    int rc = dev_alloc(&p, c->scratch_bytes_per_cta * (size_t)blocks);
    if (rc) return rc;
    if (c->d_scratch) cudaFree(c->d_scratch);
    c->d_scratch = p;
    c->grid_blocks = blocks;
    return SQ_OK;
}

// The queue plan is open to batches whose contexts all use the single-CTA
// region kernels (the cluster kernels keep no per-CTA scratch).
bool queue_available(const sq_batch* b)
{
    for (const sq_ctx* c : b->ctx)
        if (c->cl_nc > 0 || !c->d_scratch) return false;
    return true;
}

int queue_config(int prec, int m, int which, size_t extra, int* bps, size_t* smem)
{
    return prec == SQ_FP32 ? queue_config_f32(m, which, extra, bps, smem) : queue_config_f64(m, which, extra, bps, smem);
}

constexpr long long VPAD_CHUNK = 32768;          // padded-potential elements per QI_VPAD item

// Groups (one region half-width and precision, at most QMAX systems each),
// their grids, and the item lists of their Lanczos and moments queues, with
// `npi` nodes per QI_NODES item.  Within a queue, the systems with the
// costlier nodes come first, so the last items taken are the cheaper ones.
int batch_build_queue(sq_batch* b, int npi)
{
    batch_free_graph(b);
    batch_free_queue(b);
    std::vector<sq_batch::Group> G;
    for (int i = 0; i < b->n; ++i) {
        const sq_ctx* c = b->ctx[i];
        sq_batch::Group* g = nullptr;
        for (auto& x : G)
            if (x.m == c->g.m && x.prec == c->precision && (int)x.sys.size() < QMAX) g = &x;
        if (!g) {
            G.emplace_back();
            g = &G.back();
            g->m = c->g.m;
            g->prec = c->precision;
        }
        g->sys.push_back(i);
    }
    std::vector<QItem> items;
    for (auto& g : G) {
        for (int i : g.sys) {
            g.xl = std::max(g.xl, region_extra(b->ctx[i], 1));
            g.xm = std::max(g.xm, region_extra(b->ctx[i], 0));
        }
        int bpl = 0, bpm = 0;
        size_t sm = 0;
        int rc;
        if ((rc = queue_config(g.prec, g.m, 1, g.xl, &bpl, &sm)) || (rc = queue_config(g.prec, g.m, 0, g.xm, &bpm, &sm)))
            return rc;
        const int sms = b->ctx[g.sys[0]]->sm_count;
        g.bl = bpl * sms;
        g.bm = bpm * sms;
        for (int i : g.sys)
            if ((rc = ensure_scratch(b->ctx[i], std::max(g.bl, g.bm)))) return rc;
        const int ns = (int)g.sys.size();
        g.need.assign(ns, 0);
        g.off_l = (int)items.size();
        for (int k = 0; k < ns; ++k) {
            const sq_ctx* c = b->ctx[g.sys[k]];
            const long long P = (long long)c->g.P1 * c->g.P2 * (c->g.n3 + 2 * c->g.m);
            for (long long e0 = 0; e0 < P; e0 += VPAD_CHUNK) {
                items.push_back({k, QI_VPAD, e0, std::min(P, e0 + VPAD_CHUNK)});
                ++g.need[k];
            }
        }
        for (int which = 1; which >= 0; --which) {
            if (which == 0) g.off_m = (int)items.size();
            std::vector<int> order(ns);
            for (int k = 0; k < ns; ++k) order[k] = k;
            auto cost = [&](int k) {                                 // per node, up to a common factor
                const sq_ctx* c = b->ctx[g.sys[k]];
                return (which == 1 ? 1.0 : (double)c->npl) * (1.0 + proj_pairs(c) * 8.0 / 52.0);
            };
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
            for (int k : order) {
                const long long Nd = b->ctx[g.sys[k]]->g.Nd;
                for (long long n0 = 0; n0 < Nd; n0 += npi) items.push_back({k, QI_NODES, n0, std::min(Nd, n0 + npi)});
            }
            if (which == 1) g.n_l = (int)items.size() - g.off_l;
            else g.n_m = (int)items.size() - g.off_m;
        }
    }
    int rc;
    if ((rc = dev_alloc(&b->d_items, sizeof(QItem) * items.size())) ||
        (rc = dev_alloc(&b->d_ctl, sizeof(unsigned) * (2 + QMAX) * G.size())))
        return rc;
    if (cudaMemcpy(b->d_items, items.data(), sizeof(QItem) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return SQ_ECUDA;
    }
    b->gfork.assign(G.size(), nullptr);
    for (auto& e : b->gfork)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return SQ_ECUDA;
        }
    b->groups = std::move(G);
    b->groups_npi = npi;
    return SQ_OK;
}

int queue_launch(int m, int which, const QueueArgs<float>& q, size_t extra, int blocks, cudaStream_t st)
{
    return queue_launch_f32(m, which, q, extra, blocks, st);
}
int queue_launch(int m, int which, const QueueArgs<double>& q, size_t extra, int blocks, cudaStream_t st)
{
    return queue_launch_f64(m, which, q, extra, blocks, st);
}

// Enqueue group gi of the queue plan on b->own: the Lanczos queue (QI_VPAD
// items, then the nodes), the tridiagonal extremes of its systems, the
// moments queue; then fork each system's Fermi search and density onto its
// own stream (joined at the end of the graph).
template <typename T>
int batch_enqueue_group(sq_batch* b, int gi, const BatchArgs& A)
{
    const sq_batch::Group& g = b->groups[gi];
    const int ns = (int)g.sys.size();
    unsigned* ctl = b->d_ctl + (size_t)gi * (2 + QMAX);
    QueueArgs<T> q;
    memset(&q, 0, sizeof(q));
    for (int k = 0; k < ns; ++k) {
        sq_ctx* c = b->ctx[g.sys[k]];
        RegionArgs<T> a = region_args<T>(c);
        a.n_lanczos = A.n_lanczos; a.nl_cap = c->nl_cap; a.alpha = c->d_alpha; a.beta = c->d_beta; a.klen = c->d_klen;
        q.sys[k] = a;
        q.V[k] = A.V[g.sys[k]];
        q.need[k] = g.need[k];
    }
    q.items = b->d_items + g.off_l;
    q.n_items = g.n_l;
    q.next = ctl;
    q.done = ctl + 2;
    q.budget = b->wait_budget;
    q.unset = b->wait_unset;
    int rc = queue_launch(g.m, 1, q, g.xl, g.bl, b->own);
    if (rc) return rc;
    for (int k = 0; k < ns; ++k) {
        sq_ctx* c = b->ctx[g.sys[k]];
        c->launches++;
        c->stream = b->own;
        if ((rc = launch_tridiag_bounds(c, A.margin, A.chi[g.sys[k]], A.zeta[g.sys[k]]))) return rc;
    }
    for (int k = 0; k < ns; ++k) {
        sq_ctx* c = b->ctx[g.sys[k]];
        RegionArgs<T> a = region_args<T>(c);
        const int i = g.sys[k];
        a.chi = A.chi[i]; a.zeta = A.zeta[i]; a.moments = A.moments[i];
        q.sys[k] = a;
    }
    q.items = b->d_items + g.off_m;
    q.n_items = g.n_m;
    q.next = ctl + 1;
    rc = queue_launch(g.m, 0, q, g.xm, g.bm, b->own);
    if (rc) return rc;
    if (cudaEventRecord(b->gfork[gi], b->own) != cudaSuccess) return SQ_ECUDA;
    for (int k = 0; k < ns; ++k) {
        const int i = g.sys[k];
        sq_ctx* c = b->ctx[i];
        c->launches++;
        c->stream = b->st[i];
        if (cudaStreamWaitEvent(b->st[i], b->gfork[gi], 0) != cudaSuccess) return SQ_ECUDA;
        if ((rc = launch_weights(c, A.moments[i]))) return rc;
        if ((rc = enqueue_fermi(c, A.chi[i], A.zeta[i], A.Ne[i], A.kT[i]))) return rc;
        if ((rc = enqueue_density(c, A.chi[i], A.zeta[i], 0.0, A.kT[i], A.rho[i], 1))) return rc;
        if (cudaEventRecord(b->join[i], b->st[i]) != cudaSuccess) return SQ_ECUDA;
    }
    return SQ_OK;
}

// Capture the queue plan: the counters cleared, the groups one after another
// on the batch's stream, every system's post-processing joined at the end.
int batch_capture_queue(sq_batch* b, const BatchArgs& A, cudaGraphExec_t* out)
{
    std::vector<cudaStream_t> saved(b->n);
    for (int i = 0; i < b->n; ++i) saved[i] = b->ctx[i]->stream;
    if (cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return SQ_ECUDA;
    }
    int rc = SQ_OK;
    if (cudaMemsetAsync(b->d_ctl, 0, sizeof(unsigned) * (2 + QMAX) * b->groups.size(), b->own) != cudaSuccess)
        rc = SQ_ECUDA;
    for (int gi = 0; gi < (int)b->groups.size() && rc == SQ_OK; ++gi)
        rc = b->groups[gi].prec == SQ_FP32 ? batch_enqueue_group<float>(b, gi, A) : batch_enqueue_group<double>(b, gi, A);
    for (int i = 0; i < b->n && rc == SQ_OK; ++i)
        if (cudaStreamWaitEvent(b->own, b->join[i], 0) != cudaSuccess) rc = SQ_ECUDA;
    for (int i = 0; i < b->n; ++i) b->ctx[i]->stream = saved[i];
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->own, &graph);
    if (rc == SQ_OK && e != cudaSuccess) rc = SQ_ECUDA;
    if (rc == SQ_OK && cudaGraphInstantiate(out, graph, 0) != cudaSuccess) rc = SQ_ECUDA;
    if (graph) cudaGraphDestroy(graph);
    if (rc) cudaGetLastError();
    return rc;
}

// Capture launch plan `kind` (SQ_BATCH_STREAMS / _STREAMS_SHARE with the
// per-system grids `blocks`, or SQ_BATCH_QUEUE with `npi` nodes per item).
int batch_capture(sq_batch* b, const BatchArgs& A, int kind, const std::vector<int>& blocks, int npi,
                  cudaGraphExec_t* out)
{
    if (kind != SQ_BATCH_QUEUE) return batch_capture_streams(b, A, blocks, out);
    if (b->groups_npi != npi) {
        const int rc = batch_build_queue(b, npi);
        if (rc) return rc;
    }
    return batch_capture_queue(b, A, out);
}

// Time one launch of an instantiated graph.
int batch_time(sq_batch* b, cudaGraphExec_t g, float* ms)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SQ_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return SQ_ECUDA; }
    int rc = SQ_OK;
    if (cudaEventRecord(e0, b->own) != cudaSuccess || cudaGraphLaunch(g, b->own) != cudaSuccess ||
        cudaEventRecord(e1, b->own) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
        rc = SQ_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

// Region-kernel grids cut to SM shares proportional to each system's work:
// nodes x region points x (n_lanczos + n_pl/2) x (1 + the projector share).
int share_blocks(sq_batch* b, const BatchArgs& A, std::vector<int>* share)
{
    const int n = b->n;
    std::vector<double> w(n, 0.0);
    double W = 0.0;
    for (int i = 0; i < n; ++i) {
        const sq_ctx* c = b->ctx[i];
        const double S = 2.0 * c->g.m + 1.0;
        w[i] = (double)c->g.Nd * S * S * S * (A.n_lanczos + c->npl / 2) * (1.0 + proj_pairs(c) * 8.0 / 52.0);
        W += w[i];
    }
    share->assign(n, 1);
    for (int i = 0; i < n; ++i) {
        int bm = 0;
        int rc = region_blocks(b->ctx[i], 0, &bm);
        if (rc) return rc;
        const int per_sm = std::max(1, bm / std::max(1, b->ctx[i]->sm_count));
        (*share)[i] = std::max(1, (int)std::floor(w[i] / W * b->ctx[i]->sm_count * per_sm));
    }
    return SQ_OK;
}

// The autotuner.  Candidate plans are timed as complete graphs on the first
// run and the fastest is kept:
//   SQ_BATCH_STREAMS        every system on its own stream, each region kernel
//                           on its full persistent grid (the systems' kernels
//                           queue for the SMs; small Fermi and density
//                           launches of a finished system overlap the next);
//   SQ_BATCH_STREAMS_SHARE  the same with grids cut to SM shares proportional
//                           to each system's work (systems side by side);
//   SQ_BATCH_QUEUE          persistent queue kernels per group of systems with
//                           one region size, with 1 or 4 nodes per item.
// A plan set with sq_batch_set_plan is used as given.  Thread-block clusters
// are not among the candidates: the cluster form of the region kernels is
// slower on every region size measured.
int batch_tune(sq_batch* b, const BatchArgs& A)
{
    const int n = b->n;
    std::vector<int> full(n, 0), share;
    int rc = share_blocks(b, A, &share);
    if (rc) return rc;
    struct Cand { int kind; int npi; };
    std::vector<Cand> cands;
    if (b->plan_req != SQ_BATCH_AUTO) {
        cands.push_back({b->plan_req, b->npi_req});
    } else {
        cands.push_back({SQ_BATCH_STREAMS, 1});
        cands.push_back({SQ_BATCH_STREAMS_SHARE, 1});
        if (queue_available(b)) {
            cands.push_back({SQ_BATCH_QUEUE, 1});
            cands.push_back({SQ_BATCH_QUEUE, 4});
        }
    }
    if (cands.size() == 1) {
        b->plan = cands[0].kind;
        b->npi = cands[0].npi;
        b->blocks = b->plan == SQ_BATCH_STREAMS_SHARE ? share : full;
        b->tuned = true;
        return SQ_OK;
    }
    float best = 0.f;
    int pick = 0;
    for (size_t k = 0; k < cands.size(); ++k) {
        cudaGraphExec_t g = nullptr;
        rc = batch_capture(b, A, cands[k].kind, cands[k].kind == SQ_BATCH_STREAMS_SHARE ? share : full, cands[k].npi, &g);
        float ms = 0.f;
        if (rc == SQ_OK) rc = batch_time(b, g, &ms);
        if (g) cudaGraphExecDestroy(g);
        if (rc == SQ_EUNSUPPORTED && cands[k].kind == SQ_BATCH_QUEUE) continue;   // a group's kernel does not fit
        if (rc) return rc;
        if (k == 0 || ms < best) {
            best = ms;
            pick = (int)k;
        }
    }
    b->plan = cands[pick].kind;
    b->npi = cands[pick].npi;
    b->blocks = b->plan == SQ_BATCH_STREAMS_SHARE ? share : full;
    b->tuned = true;
    return SQ_OK;
}

}  // namespace

extern "C" {

const char* sq_strerror(int s)
{
    switch (s) {
        case SQ_OK: return "ok";
        case SQ_EINVAL: return "invalid argument";
        case SQ_ECUDA: return "CUDA runtime error";
        case SQ_EBOUNDS: return "Chebyshev moment outside [-1,1]: spectrum not enclosed by [chi-zeta, chi+zeta]";
        case SQ_ENOCONV: return "Fermi-level bracket does not contain the electron count";
        case SQ_ETIMEOUT: return "device wait budget exceeded";
        case SQ_ENOMEM: return "device allocation failed";
        case SQ_ECAPACITY: return "per-node projector table capacity exceeded";
        case SQ_EUNSUPPORTED: return "request not supported by this build";
    }
    return "unknown status";
}

int sq_setup_grid(sq_ctx** out, int n1, int n2, int n3, double h, int fd_half_order, double r_cut, int npl,
                  int precision, int n_atoms, const double* atom_xyz_host, int n_proj_types,
                  const sq_proj_type* proj, void* cuda_stream)
{
    if (!out) return SQ_EINVAL;
    *out = nullptr;
    if (n1 < 1 || n2 < 1 || n3 < 1 || n1 > 4096 || n2 > 4096 || n3 > 4096) return SQ_EINVAL;
    if ((long long)n1 * n2 * n3 > (1LL << 31)) return SQ_EINVAL;
    if (!is_fin(h) || h <= 0.0 || !is_fin(r_cut) || r_cut < 0.0) return SQ_EINVAL;
    if (fd_half_order < 1 || fd_half_order > 16) return SQ_EINVAL;
    if (fd_half_order != FD_NO) return SQ_EUNSUPPORTED;
    if (npl < 4 || npl > MAX_NPL || npl % 4 != 0) return SQ_EINVAL;
    if (precision != SQ_FP64 && precision != SQ_FP32) return SQ_EINVAL;
    if (n_atoms < 0 || n_proj_types < 0 || n_proj_types > 2) return SQ_EINVAL;
    if (n_proj_types > 0 && !proj) return SQ_EINVAL;
    if (n_proj_types > 0 && n_atoms > 0 && !atom_xyz_host) return SQ_EINVAL;
    double rm = floor(r_cut / h + 1e-12);
    if (rm > MAX_M) return SQ_EUNSUPPORTED;
    int m = (int)rm;
    if (precision == SQ_FP64 && m > 12) return SQ_EUNSUPPORTED;
    int has_s = 0, has_p = 0;
    double gs = 0, gp = 0, rc = 0, rnl = 0;
    for (int t = 0; t < n_proj_types; ++t) {
        const sq_proj_type& p = proj[t];
        if ((p.l != 0 && p.l != 1) || !is_fin(p.gamma) || !is_fin(p.rc) || p.rc <= 0.0 || !is_fin(p.r_nl) ||
            p.r_nl <= 0.0)
            return SQ_EINVAL;
        if (p.l == 0) { if (has_s) return SQ_EUNSUPPORTED; has_s = 1; gs = p.gamma; }
        else { if (has_p) return SQ_EUNSUPPORTED; has_p = 1; gp = p.gamma; }
        if (t > 0 && (p.rc != rc || p.r_nl != rnl)) return SQ_EUNSUPPORTED;
        rc = p.rc;
        rnl = p.r_nl;
    }
    if (n_proj_types > 0 && 2.0 * rnl / h + 2.0 > NL_BOX) return SQ_EUNSUPPORTED;
    for (long long i = 0; n_proj_types > 0 && i < 3LL * n_atoms; ++i)
        if (!is_fin(atom_xyz_host[i])) return SQ_EINVAL;

    sq_ctx* c = new (std::nothrow) sq_ctx;
    if (!c) return SQ_ENOMEM;
    memset(c, 0, sizeof(*c));
    c->precision = precision;
    c->npl = npl;
    c->stream = (cudaStream_t)cuda_stream;
    c->g.n1 = n1; c->g.n2 = n2; c->g.n3 = n3;
    c->g.m = m;
    c->g.Nd = (long long)n1 * n2 * n3;
    c->g.P1 = n1 + 2 * m;
    c->g.P2 = n2 + 2 * m;
    c->g.h = h;
    fd_weights(FD_NO, h, c->g.w);
    c->n_atoms = (n_proj_types > 0) ? n_atoms : 0;
    c->has_s = has_s; c->has_p = has_p;
    c->gamma_s = gs; c->gamma_p = gp; c->rc = rc; c->rnl = rnl;

    int dev = 0, rcode;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        free_ctx(c);
        return SQ_ECUDA;
    }
    const size_t tsz = precision == SQ_FP32 ? sizeof(float) : sizeof(double);
    const long long P3 = n3 + 2 * m;
    if ((rcode = dev_alloc(&c->Vp, tsz * c->g.P1 * c->g.P2 * P3))) { free_ctx(c); return rcode; }
    if (c->n_atoms > 0) {
        if ((rcode = setup_projectors(c, atom_xyz_host))) { free_ctx(c); return rcode; }
    } else {
        c->ntile[0] = c->ntile[1] = c->ntile[2] = 1;
    }
    if ((rcode = select_cluster_kernels(c))) { free_ctx(c); return rcode; }
    // projector tables of the candidates in shared memory when they fit next
    // to the region vectors (both kernels must accept the size): all of them,
    // else the ones every step reads, else none.  SQ_NL_TABLES=global, hot or
    // all in the environment caps the choice (for comparisons).
    int bm = 0, bl = 0;
    c->nl_extra = 0;
    c->nl_mode = NL_GLOBAL;
    const char* env = getenv("SQ_NL_TABLES");
    const int cap_mode = !env ? NL_ALL : strcmp(env, "global") == 0 ? NL_GLOBAL : strcmp(env, "hot") == 0 ? NL_HOT : NL_ALL;
    for (int mode : {(int)NL_ALL, (int)NL_HOT}) {
        if (c->n_atoms == 0 || cap_mode == NL_GLOBAL) break;
        if (mode == NL_ALL && cap_mode == NL_HOT) continue;
        c->nl_mode = mode;
        c->nl_extra = nl_smem_bytes(mode, c->ccap, 2 * m + 1, c->lb, tsz);
        if (region_blocks(c, 0, &bm) == SQ_OK && region_blocks(c, 1, &bl) == SQ_OK) break;
        c->nl_mode = NL_GLOBAL;
        c->nl_extra = 0;
    }
    if ((rcode = region_blocks(c, 0, &bm)) || (rcode = region_blocks(c, 1, &bl))) { free_ctx(c); return rcode; }
    c->grid_blocks = std::max(bm, bl);
    c->scratch_bytes_per_cta = scratch_layout(m, tsz).total;
    if (c->cl_nc == 0 &&               // the cluster kernels keep everything in shared memory
        (rcode = dev_alloc(&c->d_scratch, c->scratch_bytes_per_cta * c->grid_blocks))) { free_ctx(c); return rcode; }
    c->red_blocks = c->sm_count * 4;
    if ((rcode = dev_alloc(&c->d_W, sizeof(double) * c->g.Nd * (npl + 1))) ||
        (rcode = dev_alloc(&c->d_red, sizeof(double) * 3 * c->red_blocks)) ||
        (rcode = dev_alloc(&c->d_fermi, sizeof(double) * 32)) ||
        (rcode = dev_alloc(&c->d_count, sizeof(unsigned) * 4)) || (rcode = dev_alloc(&c->d_err, sizeof(unsigned)))) {
        free_ctx(c);
        return rcode;
    }
    if (cudaMemsetAsync(c->d_count, 0, sizeof(unsigned) * 4, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        free_ctx(c);
        return SQ_ECUDA;
    }
    *out = c;
    return SQ_OK;
}

int sq_set_stream(sq_ctx* c, void* stream)
{
    if (!c) return SQ_EINVAL;
    c->stream = (cudaStream_t)stream;
    return SQ_OK;
}

int sq_spectral_bounds(sq_ctx* c, const double* V, double* chi, double* zeta, int n_lanczos, double margin)
{
    if (!c || n_lanczos < 1 || n_lanczos > 512 || !is_fin(margin) || margin < 0.0 || margin >= 1.0)
        return SQ_EINVAL;
    if (!is_device_ptr(V) || !is_device_ptr(chi) || !is_device_ptr(zeta)) return SQ_EINVAL;
    int rc = ensure_lanczos_buffers(c, n_lanczos);
    if (rc) return rc;
    if ((rc = launch_build_vpad(c, V))) return rc;
    int blocks = 0;
    if ((rc = region_blocks(c, 1, &blocks))) return rc;
    return enqueue_bounds(c, blocks, n_lanczos, margin, chi, zeta);
}

int sq_moments(sq_ctx* c, const double* V, const double* chi, const double* zeta, double* moments)
{
    if (!c) return SQ_EINVAL;
    if (!is_device_ptr(V) || !is_device_ptr(chi) || !is_device_ptr(zeta) || !is_device_ptr(moments))
        return SQ_EINVAL;
    int rc = launch_build_vpad(c, V);
    if (rc) return rc;
    int blocks = 0;
    if ((rc = region_blocks(c, 0, &blocks))) return rc;
    return enqueue_moments(c, blocks, chi, zeta, moments);
}

int sq_fermi_level(sq_ctx* c, const double* moments, const double* chi, const double* zeta, double n_electrons,
                   double kT, double* mu_host)
{
    if (!c || !mu_host || !is_fin(n_electrons) || !is_fin(kT) || kT <= 0.0) return SQ_EINVAL;
    if (n_electrons <= 0.0 || n_electrons >= 2.0 * (double)c->g.Nd) return SQ_EINVAL;
    if (!is_device_ptr(moments) || !is_device_ptr(chi) || !is_device_ptr(zeta)) return SQ_EINVAL;
    int rc = launch_weights(c, moments);
    if (rc) return rc;
    double mu = 0.0;
    rc = run_fermi(c, chi, zeta, n_electrons, kT, &mu);
    int e = take_device_error(c);
    if (e) return e;
    if (rc) return rc;
    *mu_host = mu;
    return SQ_OK;
}

int sq_density_energy(sq_ctx* c, const double* moments, const double* chi, const double* zeta, double mu, double kT,
                      double* rho, double* e_band_host, double* e_ent_host, double* n_elec_host)
{
    if (!c || !is_fin(mu) || !is_fin(kT) || kT <= 0.0) return SQ_EINVAL;
    if (!is_device_ptr(moments) || !is_device_ptr(chi) || !is_device_ptr(zeta) || !is_device_ptr(rho))
        return SQ_EINVAL;
    int rc = launch_weights(c, moments);
    if (rc) return rc;
    rc = run_density(c, chi, zeta, mu, kT, rho, e_band_host, e_ent_host, n_elec_host);
    int e = take_device_error(c);
    if (e) return e;
    return rc;
}

int sq_sync(sq_ctx* c)
{
    if (!c) return SQ_EINVAL;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SQ_ECUDA;
    return take_device_error(c);
}

long long sq_launch_count(const sq_ctx* c) { return c ? c->launches : -1; }

int sq_context_info(const sq_ctx* c, int* info, int n)
{
    if (!c || !info || n < 4) return SQ_EINVAL;
    info[0] = c->g.m;
    info[1] = c->ccap;
    info[2] = c->nl_mode;
    info[3] = c->grid_blocks;
    return SQ_OK;
}

void sq_destroy(sq_ctx* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
}

int sq_batch_create(sq_batch** out, int n, sq_ctx* const* ctxs, void* cuda_stream)
{
    if (!out) return SQ_EINVAL;
    *out = nullptr;
    if (n < 1 || n > 4096 || !ctxs) return SQ_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i]) return SQ_EINVAL;
    sq_batch* b = new (std::nothrow) sq_batch();
    if (!b) return SQ_ENOMEM;
    b->n = n;
    b->ctx.assign(ctxs, ctxs + n);
    b->stream = (cudaStream_t)cuda_stream;
    b->st.assign(n, nullptr);
    b->join.assign(n, nullptr);
    b->blocks.assign(n, 0);
    b->state.assign((size_t)n * FERMI_STATE, 0.0);
    int rc = SQ_OK;
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking) != cudaSuccess)
        rc = SQ_ECUDA;
    for (int i = 0; i < n && rc == SQ_OK; ++i)
        if (cudaStreamCreateWithFlags(&b->st[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) != cudaSuccess)
            rc = SQ_ECUDA;
    if (rc) {
        cudaGetLastError();
        sq_batch_destroy(b);
        return rc;
    }
    *out = b;
    return SQ_OK;
}

int sq_batch_run(sq_batch* b, const double* const* V, double* const* chi, double* const* zeta,
                 double* const* moments, double* const* rho, const double* n_electrons, const double* kT,
                 int n_lanczos, double margin)
{
    if (!b || !V || !chi || !zeta || !moments || !rho || !n_electrons || !kT) return SQ_EINVAL;
    if (n_lanczos < 1 || n_lanczos > 512 || !is_fin(margin) || margin < 0.0 || margin >= 1.0) return SQ_EINVAL;
    std::vector<const void*> key;
    std::vector<double> kv;
    for (int i = 0; i < b->n; ++i) {
        sq_ctx* c = b->ctx[i];
        if (!is_device_ptr(V[i]) || !is_device_ptr(chi[i]) || !is_device_ptr(zeta[i]) ||
            !is_device_ptr(moments[i]) || !is_device_ptr(rho[i]))
            return SQ_EINVAL;
        if (!is_fin(kT[i]) || kT[i] <= 0.0 || !is_fin(n_electrons[i]) || n_electrons[i] <= 0.0 ||
            n_electrons[i] >= 2.0 * (double)c->g.Nd)
            return SQ_EINVAL;
        int rc = ensure_lanczos_buffers(c, n_lanczos);
        if (rc) return rc;
        key.insert(key.end(), {V[i], chi[i], zeta[i], moments[i], rho[i]});
        kv.insert(kv.end(), {n_electrons[i], kT[i]});
    }
    BatchArgs A = {V, chi, zeta, moments, rho, n_electrons, kT, n_lanczos, margin};
    // the batch's stream follows the caller's (inputs written there are ready)
    if (cudaEventRecord(b->ev_in, b->stream) != cudaSuccess || cudaStreamWaitEvent(b->own, b->ev_in, 0) != cudaSuccess) {
        cudaGetLastError();
        return SQ_ECUDA;
    }
    const bool same = b->exec && key == b->key_ptr && kv == b->key_val && n_lanczos == b->key_nl &&
                      margin == b->key_margin;
    if (!same) {
        batch_free_graph(b);
        int rc = SQ_OK;
        if (!b->tuned) rc = batch_tune(b, A);
        if (rc == SQ_OK) rc = batch_capture(b, A, b->plan, b->blocks, b->npi, &b->exec);
        if (rc) {
            b->exec = nullptr;
            return rc;
        }
        b->key_ptr = key;
        b->key_val = kv;
        b->key_nl = n_lanczos;
        b->key_margin = margin;
    }
    if (cudaGraphLaunch(b->exec, b->own) != cudaSuccess || cudaEventRecord(b->ev_out, b->own) != cudaSuccess ||
        cudaStreamWaitEvent(b->stream, b->ev_out, 0) != cudaSuccess) {    // and the caller's follows the batch
        cudaGetLastError();
        return SQ_ECUDA;
    }
    for (sq_ctx* c : b->ctx) c->launches++;
    return SQ_OK;
}

int sq_batch_results(sq_batch* b, double* mu_host, double* e_band_host, double* e_ent_host, double* n_elec_host)
{
    if (!b) return SQ_EINVAL;
    for (int i = 0; i < b->n; ++i)
        if (cudaMemcpyAsync(b->state.data() + (size_t)i * FERMI_STATE, b->ctx[i]->d_fermi,
                            sizeof(double) * FERMI_STATE, cudaMemcpyDeviceToHost, b->own) != cudaSuccess) {
            cudaGetLastError();
            return SQ_ECUDA;
        }
    if (cudaStreamSynchronize(b->own) != cudaSuccess) {
        cudaGetLastError();
        return SQ_ECUDA;
    }
    int first = SQ_OK;
    for (int i = 0; i < b->n; ++i) {
        int e = take_device_error(b->ctx[i]);
        int r = fermi_result(b->state.data() + (size_t)i * FERMI_STATE, mu_host ? mu_host + i : nullptr,
                             e_band_host ? e_band_host + i : nullptr, e_ent_host ? e_ent_host + i : nullptr,
                             n_elec_host ? n_elec_host + i : nullptr);
        if (!first) first = e ? e : r;
    }
    return first;
}

int sq_batch_blocks(const sq_batch* b, int* blocks_host)
{
    if (!b || !blocks_host) return SQ_EINVAL;
    for (int i = 0; i < b->n; ++i) blocks_host[i] = b->blocks[i];
    return b->tuned ? SQ_OK : SQ_EINVAL;
}

int sq_batch_set_plan(sq_batch* b, int plan, int nodes_per_item)
{
    if (!b) return SQ_EINVAL;
    if (plan != SQ_BATCH_AUTO && plan != SQ_BATCH_STREAMS && plan != SQ_BATCH_STREAMS_SHARE && plan != SQ_BATCH_QUEUE)
        return SQ_EINVAL;
    if (plan == SQ_BATCH_QUEUE && (nodes_per_item < 1 || nodes_per_item > 4096)) return SQ_EINVAL;
    if (plan == SQ_BATCH_QUEUE && !queue_available(b)) return SQ_EUNSUPPORTED;
    batch_free_graph(b);
    b->plan_req = plan;
    b->npi_req = plan == SQ_BATCH_QUEUE ? nodes_per_item : 1;
    b->tuned = false;
    return SQ_OK;
}

int sq_batch_plan(const sq_batch* b, int* plan, int* nodes_per_item)
{
    if (!b || !plan || !nodes_per_item || !b->tuned) return SQ_EINVAL;
    *plan = b->plan;
    *nodes_per_item = b->plan == SQ_BATCH_QUEUE ? b->npi : 0;
    return SQ_OK;
}

int sq_batch_set_wait(sq_batch* b, long long budget_cycles, int wait_on_unset)
{
    if (!b || budget_cycles < 1 || budget_cycles > 1000000000000LL || (wait_on_unset != 0 && wait_on_unset != 1))
        return SQ_EINVAL;
    batch_free_graph(b);
    b->wait_budget = budget_cycles;
    b->wait_unset = wait_on_unset;
    return SQ_OK;
}

void sq_batch_destroy(sq_batch* b)
{
    if (!b) return;
    batch_free_graph(b);
    batch_free_queue(b);
    for (cudaStream_t s : b->st)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->own) cudaStreamDestroy(b->own);
    delete b;
}

}  // extern "C"
