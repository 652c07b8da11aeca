// sq_internal.cuh -- internal declarations shared by the libsq translation units.
//
// Data layout in HBM (all owned by sq_ctx):
//   Vp       potential copied into precision T with a periodic halo of m points
//            on every side: (n1+2m) x (n2+2m) x (n3+2m), x fastest.  The window
//            of node (i,j,k) is then the contiguous box starting at (i,j,k).
//   atom tables (one per atom, shared by all its periodic images):
//            box start lo[3] (atom-relative grid index), box length len[3],
//            separable Gaussian factors G[a][i] = exp(-(i h - R_a)^2/(2 rc^2))
//            and DG[a][i] = (i h - R_a) G[a][i] per axis a, and for every box
//            row (j,k) the x-interval of points with |r| < r_nl.
//   tile lists: for every tile of 8^3 nodes, the (atom, image box start) pairs
//            whose box meets some region of a node in the tile (CSR).
//   per-CTA scratch: the second recurrence vector (t^{i-1} / Lanczos v_old)
//            and the per-node projector candidate and row-entry lists.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "../../include/sq.h"

namespace sq {

constexpr int FD_NO = 6;             // n_o of Eq. (FD:Laplacian) this build supports
constexpr int MAX_M = 15;            // region side 2m+1 <= 31
constexpr int NL_BOX = 32;           // max projector box length per axis (points)
constexpr int TILE = 8;              // node tile edge for projector candidate lists
constexpr int MAX_CAND = 512;        // projector candidates per node
constexpr int ENTRIES_PER_ROW = 24;  // projector entries a region row may hold (FCC Al at h ~ 0.48: up to 14)
constexpr int MAX_NPL = 512;

// Error bits latched on the device (combined into one sq_status on the host).
constexpr unsigned ERR_BOUNDS = 1u;
constexpr unsigned ERR_CAPACITY = 2u;
constexpr unsigned ERR_NONFINITE = 4u;   // a potential value that is NaN or infinite
constexpr unsigned ERR_TIMEOUT = 8u;     // a bounded device wait ran out of its budget

struct AtomTab {                     // per-atom projector geometry (device)
    int lo[3];
    int len[3];
};

// Everything a kernel needs about the projectors.
template <typename T>
struct NLParams {
    int n_atoms;                     // 0 = local only
    const AtomTab* atoms;
    int lb;                          // table stride: longest projector box edge (points, <= NL_BOX)
    const T* G;                      // [atom][3][lb]
    const T* DG;                     // [atom][3][lb]
    const uint8_t* ivl;              // [atom][lb][lb][2]  (xlo, xhi) box-relative, empty: xlo > xhi
    const int* tile_start;           // [ntiles+1]
    const int4* tile_cand;           // (atom, box start x, y, z) unwrapped
    int ntile[3];
    int ccap;                        // most candidates any node has (exact, from the set-up)
    int smem;                        // placement of the per-candidate tables: NL_GLOBAL, NL_ALL or NL_HOT (shared memory after the region vectors)
    T cs;                            // h^3 gamma_s A_s^2   (0 if no s channel)
    T cp;                            // h^3 gamma_p A_p^2   (0 if no p channel)
};

// Projector entry record: one (candidate, region row) pair whose clipped
// support interval in x is non-empty, with the row's y/z Gaussian factors
//   f0 = G_y G_z,  f1 = DG_y G_z,  f2 = G_y DG_z.
// meta = key | xlo << 10 | xhi << 15 | (bx + 32) << 20, where key is the
// region row r = y + S z in candidate order and the candidate index c in row
// order, and bx (in [-31, 30]) the region column of the candidate's box start,
// so that the passes over the entries need no candidate table for it.  One
// 16-byte load in FP32.
template <typename T>
struct __align__(16) EntRec {
    uint32_t meta;
    T f0, f1, f2;
};
static_assert(sizeof(EntRec<float>) == 16 && sizeof(EntRec<double>) == 32, "record sizes assumed by the scratch layout");

// Per-CTA scratch (device, one slice per resident CTA).  The entries are kept
// twice, both built once per node and read every step:
//   by candidate (rows ascending within a candidate; candidate c owns
//     cent[cand_start[c] .. cand_start[c+1])), cut into chunks of 32 entries
//     (chunk_first[c] = first chunk of c) for the inner products;
//   by row, ENTRIES_PER_ROW slots per region row (candidates ascending), for
//     the update of the second vector.
// Everything but the entry lists moves to shared memory when it fits
// (NLParams::smem).
template <typename T>
struct CtaScratch {
    T* buf;                          // S^3 second vector (when not in shared memory)
    int4* cand;                      // candidates (atom, bx, by, bz): box start relative to the region
    int* clen;                       // candidate box lengths len_x | len_y << 8 | len_z << 16
    T* P;                            // 4 per candidate: projector inner products (S, X, Y, Z)
    T* TX;                           // 2*lb per candidate: (G_x, DG_x) at box column k (0 beyond the box)
    T* seg;                          // 4 per (candidate + warp): partial inner products of one warp
    EntRec<T>* cent;                 // candidate-ordered entries
    EntRec<T>* rec;                  // row-ordered entries, ENTRIES_PER_ROW per row
    int* cand_start;                 // ncand + 1
    int* chunk_first;                // ncand + 1
    uint8_t* row_n;                  // S^2: entries of each row
};

struct GridParams {
    int n1, n2, n3;
    int m;
    long long Nd;
    int P1, P2;                      // padded potential pitches (n1+2m, n2+2m)
    double h;
    double w[FD_NO + 1];             // FD weights of Eq. (FD:Laplacian)
};

// One element of the potential with its periodic halo (Section 3.1, the
// periodic index map): padded index t of (n1+2m) x (n2+2m) x (n3+2m), x fastest,
// takes V at ((i-m) mod n1, (j-m) mod n2, (k-m) mod n3).  A non-finite value
// latches ERR_NONFINITE.
template <typename T>
__device__ inline void vpad_elem(const double* __restrict__ V, T* __restrict__ Vp, int n1, int n2, int n3, int m,
                                 long long t, unsigned* err)
{
    const int P1 = n1 + 2 * m, P2 = n2 + 2 * m;
    const int i = (int)(t % P1);
    const int j = (int)((t / P1) % P2);
    const int k = (int)(t / ((long long)P1 * P2));
    const int a = ((i - m) % n1 + n1) % n1;
    const int b = ((j - m) % n2 + n2) % n2;
    const int c = ((k - m) % n3 + n3) % n3;
    const double v = V[a + (long long)n1 * (b + (long long)n2 * c)];
    if (!isfinite(v)) atomicOr(err, ERR_NONFINITE);
    Vp[t] = (T)v;
}

}  // namespace sq

struct sq_ctx {
    int precision;
    sq::GridParams g;
    int npl;
    cudaStream_t stream;
    int sm_count;
    long long launches;
    // potential copy with halo, in the recurrence precision
    void* Vp;
    // projectors
    int n_atoms;
    int has_s, has_p;
    double gamma_s, gamma_p, rc, rnl;
    sq::AtomTab* d_atoms;
    void* d_G;
    void* d_DG;
    uint8_t* d_ivl;
    int lb;
    int ccap;                        // most projector candidates of any node
    size_t nl_extra;                 // shared-memory bytes of the candidate tables (0: in global scratch)
    int nl_mode;                     // their placement: NL_GLOBAL, NL_ALL or NL_HOT (sq_region.cuh)
    int* d_tile_start;
    int4* d_tile_cand;
    int ntile[3];
    // FP32 cluster region kernels (sq_cluster.cuh): cluster size (0: the
    // single-CTA kernels), resident clusters and dynamic shared memory, per
    // kernel (0 moments, 1 Lanczos)
    int cl_nc;
    int cl_clusters[2];
    size_t cl_smem[2];
    // per-CTA scratch
    int grid_blocks;                 // resident CTAs used for the region kernels
    size_t scratch_bytes_per_cta;
    void* d_scratch;
    // Lanczos tridiagonals
    double* d_alpha;                 // [Nd][nl_max]
    double* d_beta;
    int* d_klen;
    int nl_cap;
    // quadrature weights and reductions
    double* d_W;                     // [Nd][npl+1]
    double* d_red;                   // block partials
    double* d_fermi;                 // bisection state
    unsigned* d_count;               // last-block counters
    unsigned* d_err;                 // latched device error bits
    int red_blocks;
};

// Launchers implemented in the kernel translation units.
namespace sq {
int launch_build_vpad(sq_ctx* ctx, const double* V);
int launch_lanczos(sq_ctx* ctx, int n_lanczos);
int launch_tridiag_bounds(sq_ctx* ctx, double margin, double* chi, double* zeta);
int launch_moments(sq_ctx* ctx, const double* chi, const double* zeta, double* moments);
int launch_weights(sq_ctx* ctx, const double* moments);
int run_fermi(sq_ctx* ctx, const double* chi, const double* zeta, double Ne, double kT, double* mu);
int run_density(sq_ctx* ctx, const double* chi, const double* zeta, double mu, double kT,
                double* rho, double* eb, double* es, double* ne);
// graph-capturable forms (no host wait): results stay in ctx->d_fermi
int enqueue_fermi(sq_ctx* ctx, const double* chi, const double* zeta, double Ne, double kT);
int enqueue_density(sq_ctx* ctx, const double* chi, const double* zeta, double mu, double kT, double* rho,
                    int mu_from_state);
constexpr int FERMI_STATE = 12;      // doubles of the device Fermi/energy state
int fermi_result(const double* st_host, double* mu, double* eb, double* es, double* ne);
int launch_proj_tables(sq_ctx* ctx, const double* d_R);
}  // namespace sq

#define SQ_CUDA_TRY(call)                                   \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return SQ_ECUDA;             \
    } while (0)
