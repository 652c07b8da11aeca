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
constexpr int ENTRIES_PER_ROW = 16;  // average row-entry capacity per region row (about 7-8 are used)
constexpr int MAX_NPL = 512;

// Error bits latched on the device (combined into one sq_status on the host).
constexpr unsigned ERR_BOUNDS = 1u;
constexpr unsigned ERR_CAPACITY = 2u;

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
    T cs;                            // h^3 gamma_s A_s^2   (0 if no s channel)
    T cp;                            // h^3 gamma_p A_p^2   (0 if no p channel)
};

// Per-CTA scratch layout (device, one slice per resident CTA).
// Projector entries are (candidate, region row) pairs with a non-empty clipped
// support interval; they are kept twice: by row (candidates ascending) for the
// update fused into the stencil sweep, and by candidate (rows ascending) for
// the inner products.
//   row-ordered meta:        c | xlo << 10 | xhi << 15
//   candidate-ordered meta:  r | xlo << 10 | xhi << 15      (r = y + S z)
//   factors f = (G_y G_z, DG_y G_z, G_y DG_z, 0) of the entry's row
template <typename T>
struct CtaScratch {
    T* buf;                          // S^3 second vector (when not in shared memory)
    int4* cand;                      // MAX_CAND candidates (atom, bx, by, bz) region-relative
    T* P;                            // MAX_CAND*4 projector inner products (S, X, Y, Z)
    T* TX;                           // MAX_CAND*S*2: (G_x, DG_x) of candidate c at region column x (0 outside box)
    uint32_t* ent_meta;              // cap, row-ordered
    T* ent_f;                        // cap*4, row-ordered
    uint32_t* cent_meta;             // cap, candidate-ordered
    T* cent_f;                       // cap*4, candidate-ordered
    int* row_start;                  // S^2 + 1
    int* row_fill;                   // S^2
    int* cand_start;                 // MAX_CAND + 1
};

struct GridParams {
    int n1, n2, n3;
    int m;
    long long Nd;
    int P1, P2;                      // padded potential pitches (n1+2m, n2+2m)
    double h;
    double w[FD_NO + 1];             // FD weights of Eq. (FD:Laplacian)
};

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
    int* d_tile_start;
    int4* d_tile_cand;
    int ntile[3];
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
int launch_proj_tables(sq_ctx* ctx, const double* d_R);
}  // namespace sq

#define SQ_CUDA_TRY(call)                                   \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return SQ_ECUDA;             \
    } while (0)
