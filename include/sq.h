/*
 * sq.h -- C ABI of libsq: the Clenshaw-Curtis Spectral Quadrature (SQ) hot
 * path of "SQDFT: Spectral Quadrature method for large-scale parallel O(N)
 * Kohn-Sham calculations at high temperature" (Suryanarayana, Pratapa,
 * Sharma, Pask; arXiv:1708.07913), on one NVIDIA GB300 GPU (sm_103a).
 *
 * Problem (Section 2, Eqs. DensityMatrix, rho; Section 3.2): given the
 * effective potential V on a periodic finite-difference grid of N_d nodes,
 * compute for every node q the Chebyshev moments of its nodal Hamiltonian
 * H_q (H restricted to the cube of side 2 R_cut about q with zero Dirichlet
 * boundary), the Fermi level mu that puts N_e electrons in the cell, and the
 * nodal electron density, band-structure energy and electronic entropy.
 *
 * Entry points, by group
 *   - the path: sq_setup_grid, sq_spectral_bounds, sq_moments,
 *     sq_fermi_level, sq_density_energy (+ sq_density_energy_noalloc);
 *   - forces: sq_nl_forces, sq_nl_forces_nodes (Section 3.4);
 *   - batched systems: sq_batch_* (one CUDA graph per step);
 *   - SCF loop: sq_poisson, sq_effective_potential, sq_kerker, sq_mixer_*;
 *   - learned SCF warm start: sq_cnn_*;
 *   - housekeeping: sq_set_stream, sq_sync, sq_launch_count, sq_context_info, sq_destroy,
 *     sq_strerror.
 *
 * Conventions
 *   - Hartree atomic units (Ha, bohr).
 *   - Grid: n1 x n2 x n3 nodes, spacing h, node (i,j,k) at (i h, j h, k h);
 *     every per-node array is x-fastest: index q = i + n1*(j + n2*k).
 *   - Unless stated otherwise, array arguments are DEVICE pointers owned by
 *     the caller (any allocator, e.g. PyTorch), FP64, densely packed.
 *   - Every call is enqueued on the context's CUDA stream.  sq_spectral_bounds
 *     and sq_moments are asynchronous; sq_fermi_level, sq_density_energy and
 *     sq_sync synchronise the stream because they return host scalars.
 *   - Errors: every call returns an sq_status.  Argument errors are detected
 *     on the host before anything is enqueued.  Device-side errors (a moment
 *     with |rho^j| > 1 + tol, a capacity overflow, a wait budget exceeded) are
 *     latched in the context and returned by the next synchronising call.
 *     No C++ exception crosses this interface.
 *   - Thread safety: a context may be used by one host thread at a time.
 */
#ifndef SQ_H
#define SQ_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SQ_OK = 0,
    SQ_EINVAL = 1,      /* invalid argument (checked on the host; a non-finite       */
                        /* potential value is detected on the device and latched)    */
    SQ_ECUDA = 2,       /* a CUDA runtime call or kernel launch failed               */
    SQ_EBOUNDS = 3,     /* spectrum outside [chi-zeta, chi+zeta]: |rho^j| > 1 + tol   */
    SQ_ENOCONV = 4,     /* Fermi-level bracket does not contain N_e                  */
    SQ_ETIMEOUT = 5,    /* a device wait exceeded its budget                          */
    SQ_ENOMEM = 6,      /* device allocation failed                                   */
    SQ_ECAPACITY = 7,   /* a per-node table (projector candidates/rows) overflowed    */
    SQ_EUNSUPPORTED = 8 /* valid request that this build does not implement           */
} sq_status;

typedef enum {
    SQ_FP64 = 0,        /* recurrence, Lanczos and all sums in FP64                   */
    SQ_FP32 = 1         /* recurrence and Lanczos vectors in FP32; moments, Lanczos   */
                        /* coefficients, weights, Fermi level and energies in FP64    */
} sq_precision;

/* One Kleinman-Bylander projector channel (Section 2, Eq. Hamiltonian: V_nl;
 * Section 3.1: restriction to the region of influence).  The paper uses
 * Troullier-Martins projectors; this library implements Gaussian channels
 *   l = 0:  chi(r)   = A_s exp(-r^2/(2 rc^2)),       A_s = (pi rc^2)^(-3/4)
 *   l = 1:  chi_a(r) = A_p r_a exp(-r^2/(2 rc^2)),   A_p = (sqrt 2/rc) A_s
 * supported on |r| < r_nl, entering H as gamma h^3 chi chi^T per projector.
 * At most one l = 0 and one l = 1 channel, sharing rc and r_nl. */
typedef struct {
    int l;              /* 0 (s) or 1 (p)                     */
    double gamma;       /* KB energy, Ha                      */
    double rc;          /* Gaussian width, bohr               */
    double r_nl;        /* support radius, bohr               */
} sq_proj_type;

typedef struct sq_ctx sq_ctx;

/* Create a context for one grid/geometry (Section 3.1: grid, FD order,
 * region of influence; Section 3.2: quadrature order).
 *   n1,n2,n3       grid nodes per axis (>= 1)
 *   h              mesh spacing, bohr (> 0)
 *   fd_half_order  n_o of Eq. (FD:Laplacian); this build supports 6
 *   r_cut          R_cut, bohr; region half-width m = floor(r_cut/h) points,
 *                  region side 2m+1 <= 31
 *   npl            quadrature degree n_pl (multiple of 4, 4 <= npl <= 512)
 *   precision      sq_precision
 *   n_atoms, atom_xyz_host   HOST array n_atoms*3 (bohr); may be NULL iff
 *                  n_atoms == 0 or n_proj_types == 0
 *   n_proj_types, proj       HOST array of channels; NULL / 0 = local only
 *   cuda_stream    cudaStream_t to enqueue on (NULL = legacy default stream)
 * Allocates device memory for projector tables and per-CTA scratch.
 * On error *out is set to NULL. */
int sq_setup_grid(sq_ctx **out, int n1, int n2, int n3, double h,
                  int fd_half_order, double r_cut, int npl, int precision,
                  int n_atoms, const double *atom_xyz_host,
                  int n_proj_types, const sq_proj_type *proj,
                  void *cuda_stream);

/* Change the stream later calls enqueue on. */
int sq_set_stream(sq_ctx *ctx, void *cuda_stream);

/* Spectral bounds of every nodal Hamiltonian by the Lanczos method
 * (Section 3.2, text after Eq. rhoqj: lambda_min, lambda_max of H_q, then
 * chi_q = (max+min)/2, zeta_q = (max-min)/2).  Start vector uniform on the
 * region; exactly n_lanczos steps (fewer only on breakdown, beta <= 1e-10 *
 * scale); extreme Ritz values by Sturm bisection in FP64; both ends widened
 * by margin * max(theta_max - theta_min, 1 Ha).
 *   V     device, N_d FP64 effective potential; a NaN or infinite value
 *         (here or in sq_moments) latches SQ_EINVAL, returned by the next
 *         synchronising call
 *   chi   device, N_d FP64 output
 *   zeta  device, N_d FP64 output
 *   1 <= n_lanczos <= 512, 0 <= margin < 1. */
int sq_spectral_bounds(sq_ctx *ctx, const double *V, double *chi, double *zeta,
                       int n_lanczos, double margin);

/* Chebyshev moments rho_q^j, j = 0..npl (Section 3.2, Eqs. Rec:FD, rhoqj):
 * t^0 = e_q, t^1 = Hhat t^0, t^{i+1} = 2 Hhat t^i - t^{i-1}, Hhat = (H_q -
 * chi_q)/zeta_q, run to i = npl/2; rho^j = t^j at the node for j <= npl/2,
 * and from the product property 2T_aT_b = T_{a+b} + T_{|a-b|}:
 * rho^{2a} = 2 t^a.t^a - rho^0, rho^{2a+1} = 2 t^{a+1}.t^a - rho^1.
 *   V         device, N_d FP64
 *   chi,zeta  device, N_d FP64 (zeta > 0)
 *   moments   device, N_d*(npl+1) FP64 output, node-major
 * A moment with |rho^j| > 1 + tol (tol 1e-6 FP64, 1e-4 FP32) latches
 * SQ_EBOUNDS. */
int sq_moments(sq_ctx *ctx, const double *V, const double *chi, const double *zeta,
               double *moments);

/* Fermi level (Section 3.2): solve 2 sum_q sum_j c_q^j(mu) rho_q^j = N_e with
 * c_q^j the Chebyshev coefficients of the Fermi-Dirac function (Eq. cqj) by
 * discrete orthogonality at the npl+1 zeros of T_{npl+1}.  Bisection on
 * [min(chi-zeta) - 10 kT, max(chi+zeta) + 10 kT] until the midpoint equals an
 * end point in FP64 (at most 200 steps).  Also stores the quadrature weights
 * W_qk in the context for sq_density_energy.
 *   moments, chi, zeta   device, as produced above
 *   n_electrons          0 < N_e < 2 N_d
 *   kT                   smearing sigma > 0, Ha
 *   mu_host              HOST output
 * Synchronises the stream.  SQ_ENOCONV if N(lo) > N_e or N(hi) < N_e. */
int sq_fermi_level(sq_ctx *ctx, const double *moments, const double *chi,
                   const double *zeta, double n_electrons, double kT, double *mu_host);

/* Nodal density, band energy and entropy energy at Fermi level mu
 * (Eq. ElectronDensity; Eqs. Eband, d_q; Eqs. Entropy, e_q):
 *   rho_q  = (2/h^3) sum_k W_qk g_qk
 *   E_band = 2 sum_q sum_k W_qk (chi_q + zeta_q x_k) g_qk
 *   E_ent  = 2 kT sum_q sum_k W_qk [g ln g + (1-g) ln(1-g)]   (0 ln 0 = 0)
 *   N      = h^3 sum_q rho_q
 * with g_qk = 1/(1 + exp((chi_q + zeta_q x_k - mu)/kT)).  Recomputes W from
 * the moments.
 *   rho                   device, N_d FP64 output
 *   e_band_host, e_ent_host, n_elec_host   HOST outputs (each may be NULL)
 * Synchronises the stream. */
int sq_density_energy(sq_ctx *ctx, const double *moments, const double *chi,
                      const double *zeta, double mu, double kT, double *rho,
                      double *e_band_host, double *e_ent_host, double *n_elec_host);

/* Density, band energy and entropy like sq_density_energy, for callers that
 * must not allocate device memory (no context, no cudaMalloc, no allocating
 * library call).  The paper has no counterpart: this exists for host programs
 * that reserve all device memory for their own allocator, or fix their memory
 * budget at start-up, and so cannot let a library allocate.
 *   n1,n2,n3, h, npl      grid and degree as in sq_setup_grid (npl % 4 == 0,
 *                         4 <= npl <= 512, n1*n2*n3 <= 2^31); larger sizes
 *                         are rejected with SQ_EINVAL
 *   moments, chi, zeta    device inputs as for sq_fermi_level
 *   mu, kT                Fermi level and smearing (kT > 0)
 *   rho                   device output, N_d FP64
 *   e_band_host, e_ent_host, n_elec_host   HOST outputs (each may be NULL)
 *   cuda_stream           stream to run on (NULL = legacy default stream)
 * The quadrature weights are recomputed per node instead of stored.  The
 * reduction's scratch is one fixed library-wide device array of 49,184 bytes
 * (partials for at most 2048 blocks), present on every device that loads the
 * library until the process exits.  The first call on a device looks up that
 * array's device address (with the device current); later calls reuse it.
 * Every call shares the array: each call clears its counter before use, and
 * calls that overlap on the GPU (other streams or host threads) race on it.
 * Synchronises the stream. */
int sq_density_energy_noalloc(int n1, int n2, int n3, double h, int npl,
                              const double *moments, const double *chi, const double *zeta,
                              double mu, double kT, double *rho,
                              double *e_band_host, double *e_ent_host, double *n_elec_host,
                              void *cuda_stream);

/* Nonlocal component of the atomic forces (Section 3.4, Eq. Discrete:NLforce,
 * with the recurrence of Eq. Rec:FD1 run to n_pl):
 *   f_I = -4 sum_q sum_{p of atom I} gamma_p h^3 chi_p(q) chi_p^T grad_h D_q,
 *   D_q = sum_{j=0}^{npl} c_q^j t^j   (t^j as for sq_moments, run to npl),
 * c_q^j the Chebyshev coefficients of the Fermi-Dirac function at mu, kT on
 * [chi_q - zeta_q, chi_q + zeta_q] (discrete orthogonality at the npl+1
 * zeros of T_{npl+1}, c^0 halved), grad_h the central finite-difference
 * gradient of Eq. FD:Gradient (order n_o) inside the node's region, zero
 * outside it.  Every periodic image of every projector whose support meets
 * the region enters, as in H_q; only nodes inside some projector's support
 * contribute.
 *   V          device, N_d FP64 (the potential the bounds were computed for)
 *   chi, zeta  device, N_d FP64 (from sq_spectral_bounds)
 *   mu, kT     Fermi level (e.g. from sq_fermi_level) and smearing > 0, Ha
 *   forces     device, n_atoms*3 FP64 output (Ha/bohr, atom-major x,y,z),
 *              overwritten; may be NULL when the context has no projectors
 * The recurrence vectors, D and the projector inner products are in the
 * context's precision (FP32 or FP64); the coefficients c^j and the final
 * contraction are FP64.  The recurrence runs on the machinery of the region
 * kernels (one CTA per node, vectors in shared memory); in FP32 its
 * projector update adds with shared-memory atomics, so repeated calls agree
 * to FP32 rounding, and FP64 results repeat bit for bit.  Where that form
 * does not fit the context (or with SQ_FORCE_KERNEL=legacy in the
 * environment) a first form with every vector in global scratch runs, which
 * repeats bit for bit in both precisions.  Allocates, on first use, about
 * (resident CTAs) x (s (2m+1)^3 + 12 KB + 24 n_atoms) bytes of workspace in
 * the context (s = 4 or 8 bytes; the first form: 2 x SMs x (4 s (2m+1)^3 +
 * (384 + 128 s) (2m+1)^2 + (24 + 4 s) ccap + 24 n_atoms)).
 * Synchronises the stream; a projector-table overflow (more candidates or
 * row entries than the tables hold) returns SQ_ECAPACITY. */
int sq_nl_forces(sq_ctx *ctx, const double *V, const double *chi, const double *zeta,
                 double mu, double kT, double *forces);

/* The same sum restricted to the nodes listed in `nodes` (device array of
 * n_nodes int64 node indices q, 1 <= n_nodes <= N_d; a node listed twice
 * contributes twice): the force contributions of a sample of nodes, each of
 * which the sum over all nodes adds once.  The list is copied to the host
 * and checked (every index in [0, N_d)) before anything is enqueued;
 * SQ_EINVAL otherwise. */
int sq_nl_forces_nodes(sq_ctx *ctx, const double *V, const double *chi, const double *zeta,
                       double mu, double kT, const long long *nodes, long long n_nodes,
                       double *forces);

/* ---------------------------------------------------------------------------
 * Batch of independent systems.  The paper treats one system at a time (its
 * parallelism is over the nodes of one grid, Section 3.2); it has no
 * counterpart for this.  A batch runs the whole step of the path -- spectral
 * bounds, moments, Fermi level and density/energies, as the single-system
 * calls above define them -- for every context in it as ONE CUDA graph
 * launch, so that systems of uneven size, region and temperature share the
 * GPU and the launch-bound Fermi-level bisections of the systems overlap.
 * The contexts of a batch must be distinct.
 *
 * sq_batch_create(out, n, ctxs, cuda_stream)
 *   ctxs: HOST array of n >= 1 contexts, not owned (they must outlive the
 *   batch and must not be used elsewhere while a batch run is in flight).
 *   cuda_stream: the caller's stream (NULL = legacy default stream); batch
 *   runs start after work already enqueued on it, and work enqueued on it
 *   afterwards starts after the batch.  Creates one stream per system.
 * sq_batch_run(b, V, chi, zeta, moments, rho, n_electrons, kT, n_lanczos,
 *              margin)
 *   V, chi, zeta, moments, rho: HOST arrays of n DEVICE pointers, each with
 *   the layout of the single-system calls; n_electrons, kT: HOST arrays of n.
 *   Enqueues the step of every system and returns without waiting.  Unless
 *   sq_batch_set_plan fixed a plan, the first call tunes the launch (and so
 *   takes about four extra batch steps): the plans below are timed as whole
 *   graphs and the fastest is kept.  A call whose pointers or parameters
 *   differ from the previous call's re-captures the graph (same plan).
 *   Argument errors are SQ_EINVAL (checked on the host before anything is
 *   enqueued).
 *
 * Launch plans:
 *   SQ_BATCH_STREAMS        each system on its own stream, every region
 *                           kernel on its full persistent grid;
 *   SQ_BATCH_STREAMS_SHARE  the same with grids cut to SM shares
 *                           proportional to each system's work (nodes x
 *                           region points x steps);
 *   SQ_BATCH_QUEUE          systems grouped by region half-width and
 *                           precision (at most 8 per group); per group one
 *                           persistent Lanczos kernel and one persistent
 *                           moments kernel take work items from a device
 *                           queue (one atomic add per item): slabs of each
 *                           system's padded potential, then runs of
 *                           nodes_per_item nodes.  A Lanczos item waits until
 *                           its system's potential slabs are done: a bounded
 *                           spin of at most the wait budget (SM clock cycles,
 *                           default 2e9, about a second); when it runs out the
 *                           item is skipped and the run's result is
 *                           SQ_ETIMEOUT (from sq_batch_results).  Not
 *                           available when a context uses the cluster form
 *                           of the region kernels (SQ_EUNSUPPORTED).
 * sq_batch_set_plan(b, plan, nodes_per_item)
 *   SQ_BATCH_AUTO (the default: tune on the next run) or one of the plans
 *   above, used as given; nodes_per_item in [1, 4096] for SQ_BATCH_QUEUE
 *   (ignored otherwise).  Drops the captured graph.
 * sq_batch_plan(b, plan, nodes_per_item): HOST ints receive the plan in use
 *   (nodes_per_item 0 unless SQ_BATCH_QUEUE); SQ_EINVAL before the first run.
 * sq_batch_set_wait(b, budget_cycles, wait_on_unset)
 *   budget_cycles in [1, 1e12]: the queue plan's wait budget.
 *   wait_on_unset = 1 makes every wait target one more potential slab than
 *   exists, so every wait runs out (a test of the time-out path: the run
 *   completes with SQ_ETIMEOUT and undefined results, and the batch and its
 *   contexts stay usable); 0 restores normal waits.  Drops the captured
 *   graph.
 * sq_batch_results(b, mu, e_band, e_ent, n_elec)
 *   Waits for the last run; HOST arrays of n (each may be NULL) receive each
 *   system's Fermi level, band energy, entropy energy and electron count
 *   (rho etc. are in the device arrays given to sq_batch_run).  Returns the
 *   first error of any system (SQ_ENOCONV, a latched device error, ...).
 * sq_batch_blocks(b, blocks): HOST array of n: the region-kernel grid chosen
 *   per system (0 = the full persistent grid, and always 0 for the queue
 *   plan); SQ_EINVAL before the first run.
 * sq_batch_destroy(b): releases the batch's streams and graph (NULL: no-op).
 * ------------------------------------------------------------------------- */
typedef struct sq_batch sq_batch;
int sq_batch_create(sq_batch **out, int n, sq_ctx *const *ctxs, void *cuda_stream);
int sq_batch_run(sq_batch *b, const double *const *V, double *const *chi, double *const *zeta,
                 double *const *moments, double *const *rho, const double *n_electrons,
                 const double *kT, int n_lanczos, double margin);
int sq_batch_results(sq_batch *b, double *mu_host, double *e_band_host, double *e_ent_host,
                     double *n_elec_host);
int sq_batch_blocks(const sq_batch *b, int *blocks_host);
enum {
    SQ_BATCH_AUTO = -1,
    SQ_BATCH_STREAMS = 0,
    SQ_BATCH_STREAMS_SHARE = 1,
    SQ_BATCH_QUEUE = 2
};
int sq_batch_set_plan(sq_batch *b, int plan, int nodes_per_item);
int sq_batch_plan(const sq_batch *b, int *plan, int *nodes_per_item);
int sq_batch_set_wait(sq_batch *b, long long budget_cycles, int wait_on_unset);
void sq_batch_destroy(sq_batch *b);

/* ---------------------------------------------------------------------------
 * Self-consistent field (SCF) loop around the path.  The paper iterates on
 * the effective potential V_eff = V_xc + phi (Section 3, footnote on the SCF
 * method), with phi from the Poisson problem of Eq. PoissonEqn solved by AAR
 * and Periodic Pulay mixing; these calls provide the conjugate-gradient,
 * Slater X-alpha and Anderson-mixing counterparts, on the device.
 *
 * sq_poisson(ctx, rho, phi, tol, max_iter, iters_host, rel_resid_host)
 *   phi solves -(1/4 pi) lap_h phi = rho - mean(rho) on the context's
 *   periodic grid (Eq. PoissonEqn with the pseudocharges replaced by the
 *   uniform neutralising background; lap_h the Laplacian of
 *   Eq. FD:Laplacian with the context's order), phi with zero mean.
 *   Conjugate gradients from phi = 0 until ||b - A phi|| <= tol ||b||,
 *   b = 4 pi (rho - mean(rho)); a neutral rho (b below 1e-13 of 4 pi ||rho||)
 *   gives phi = 0.  rho, phi: device, N_d FP64.  0 < tol < 1, max_iter >= 0.
 *   iters_host, rel_resid_host: HOST outputs (may be NULL).  SQ_ENOCONV if
 *   max_iter is reached first.  Allocates 4 N_d doubles of workspace in the
 *   context on first use.  Synchronises the stream.
 * sq_widen_bounds(ctx, V, V_ref, chi_ref, zeta_ref, chi, zeta, w_host)
 *   Spectral bounds of the nodal Hamiltonians of V from bounds computed for
 *   V_ref, without a Lanczos run.  H_q(V) = H_q(V_ref) + diag(V - V_ref) on
 *   the region, so (Weyl's inequality) every eigenvalue of H_q moves by at
 *   most w = max_t |V(t) - V_ref(t)|: chi = chi_ref, zeta = zeta_ref + w
 *   enclose the spectrum of H_q(V) wherever chi_ref +- zeta_ref enclose that
 *   of H_q(V_ref) (Section 3.2 needs only an enclosing interval; a wider one
 *   costs accuracy at a given n_pl, not correctness).  For an SCF loop whose
 *   potential changes little between iterations.
 *   V, V_ref, chi_ref, zeta_ref: device N_d FP64; chi, zeta: device N_d FP64
 *   outputs (may be chi_ref, zeta_ref themselves); w_host: HOST output (may
 *   be NULL).  Synchronises the stream; SQ_EINVAL if w is not finite.
 * sq_effective_potential(ctx, V_loc, phi, rho, alpha, V_out)
 *   V_out = V_loc + phi + v_x(rho), v_x = -(3 alpha / 2)(3 rho / pi)^(1/3)
 *   (Slater X-alpha; alpha = 2/3 is uniform-gas exchange; 0 where rho <= 0).
 *   All device, N_d FP64; 0 < alpha < 10.  Asynchronous.
 * sq_kerker(ctx, v_in, v_out, k0, amin, tol, max_iter, v_pre, rel_resid_host,
 *           iters_host)
 *   Preconditioned SCF residual for the mixer: with f = v_out - v_in,
 *   v_pre = v_in + P f,  P = (-lap_h + amin k0^2)(-lap_h + k0^2)^{-1}
 *   (Kerker-type; Fourier symbol (S + amin k0^2)/(S + k0^2), S the symbol
 *   of -lap_h: long wavelengths scaled by amin, the mean exactly, short
 *   ones passed).  (-lap_h + k0^2) u = f by conjugate gradients from 0
 *   until ||f - A u|| <= tol ||f||, then v_pre = v_in + f - (1 - amin) k0^2 u.
 *   Giving (v_in, v_pre) to sq_mixer_step mixes P f in place of f.
 *   rel_resid_host (HOST, may be NULL) = ||f|| / ||v_out||, the
 *   unpreconditioned residual; iters_host (may be NULL) the CG iterations.
 *   All device, N_d FP64; v_pre must not alias v_in or v_out; k0 > 0,
 *   0 < amin <= 1, 0 < tol < 1, max_iter >= 0.  Uses the context's Poisson
 *   workspace.  SQ_ENOCONV if max_iter is reached.  Synchronises the stream.
 * sq_mixer_create(out, n, history, beta, cuda_stream)
 *   An Anderson mixer for vectors of n doubles keeping the last `history`
 *   (0..16) differences, mixing parameter 0 < beta <= 1, on cuda_stream
 *   (NULL = legacy).  Allocates 2 (history + 1) n doubles.
 * sq_mixer_step(mx, v_in, v_out, v_next, rel_resid_host)
 *   For the fixed-point map v_in -> v_out (residual f = v_out - v_in):
 *   records (v_in, f), returns ||f|| / ||v_out|| in rel_resid_host (HOST,
 *   may be NULL) and writes v_next = v_in + beta f - (dX + beta dF) gamma,
 *   gamma minimising ||f - dF gamma|| over the stored differences (if their
 *   normal equations are numerically singular the history is not used).
 *   Device vectors of n doubles.  Synchronises the mixer's stream.
 * sq_mixer_set_period(mx, period, steps_done): Periodic Pulay mixing (the
 *   paper's scheme, Section 3): the extrapolation above on steps period-1,
 *   2 period-1, ... (counting steps from 0) and simple mixing v_in + beta f
 *   on the others, the history recorded on every step; steps_done sets the
 *   step count (0 for a new loop, the steps already taken when resuming).
 *   1 <= period <= 1000 (1, the default, extrapolates on every step).
 * sq_mixer_history(mx, count_host): pairs currently stored (0..history+1).
 * sq_mixer_export(mx, X_host, F_host): copy the stored iterates and residuals,
 *   oldest first, into HOST arrays of count x n doubles each (for a
 *   checkpoint).  sq_mixer_import(mx, count, X_host, F_host): replace the
 *   history by count <= history + 1 such pairs (resuming from a checkpoint).
 * sq_mixer_reset(mx): forget the history and the step count.
 * sq_mixer_destroy(mx): release.
 * ------------------------------------------------------------------------- */
int sq_poisson(sq_ctx *ctx, const double *rho, double *phi, double tol, int max_iter,
               int *iters_host, double *rel_resid_host);
int sq_widen_bounds(sq_ctx *ctx, const double *V, const double *V_ref, const double *chi_ref,
                    const double *zeta_ref, double *chi, double *zeta, double *w_host);
int sq_effective_potential(sq_ctx *ctx, const double *V_loc, const double *phi, const double *rho,
                           double alpha, double *V_out);
int sq_kerker(sq_ctx *ctx, const double *v_in, const double *v_out, double k0, double amin, double tol,
              int max_iter, double *v_pre, double *rel_resid_host, int *iters_host);
typedef struct sq_mixer sq_mixer;
int sq_mixer_create(sq_mixer **out, long long n, int history, double beta, void *cuda_stream);
int sq_mixer_step(sq_mixer *mx, const double *v_in, const double *v_out, double *v_next,
                  double *rel_resid_host);
int sq_mixer_set_period(sq_mixer *mx, int period, long long steps_done);
int sq_mixer_history(const sq_mixer *mx, int *count_host);
int sq_mixer_export(sq_mixer *mx, double *X_host, double *F_host);
int sq_mixer_import(sq_mixer *mx, int count, const double *X_host, const double *F_host);
int sq_mixer_reset(sq_mixer *mx);
void sq_mixer_destroy(sq_mixer *mx);

/* ---------------------------------------------------------------------------
 * Learned SCF warm start.  The paper has no counterpart.  A small 3-D
 * convolutional network, trained on densities the SQ path itself produces,
 * maps the 9^3 patch of the effective potential around each node to the
 * node's density, so that an SCF can start from a predicted density
 * instead of the bare local potential.  On the periodic n1 x n2 x n3 grid:
 *   x0  = (V - v_shift) / v_scale
 *   a1  = silu(conv5(x0; W1) + b1)     1 -> 32 channels, 5^3 kernel
 *   a2  = silu(conv3(a1; W2) + b2)     32 -> 32 channels, 3^3 kernel
 *   y   = conv3(a2; W3) + b3           32 -> 1 channel, 3^3 kernel
 *   rho = rho_scale * softplus(y)
 * with conv_k(x; W)[o](p) = sum_i sum_{d in [-r,r]^3} W[o,i,d] x[i](p + d)
 * (periodic cross-correlation, r = (k-1)/2), silu(z) = z/(1 + e^-z),
 * softplus(y) = log(1 + e^y); loss = mean((rho - rho_ref)^2) / rho_scale^2.
 * Weights and activations are stored in bfloat16 (bf16 = 1) or FP32
 * (bf16 = 0), every sum accumulates in FP32, and the master weights,
 * biases, gradients and Adam moments are FP32.  Results repeat bit for bit.
 *
 * Parameters travel as one HOST array of FP64 in the network's natural
 * order: W1 (32,1,5,5,5), b1 (32), W2 (32,32,3,3,3), b2 (32), W3 (1,32,3,3,3),
 * b3 (1), each C-ordered with the kernel axes (dz, dy, dx) -- 32,577 values
 * (sq_cnn_param_count(32)).
 *
 * sq_cnn_create(out, channels, bf16, cuda_stream): channels must be 32
 *   (SQ_EUNSUPPORTED otherwise).  Allocates the weights; activation buffers
 *   grow on first use with a grid (about 4 N (3 C s + 4 C + 5) bytes for N
 *   nodes, s = 2 or 4 bytes of storage, plus the weight-gradient partials).
 * sq_cnn_set_params(net, params_host, v_shift, v_scale, rho_scale): load
 *   weights (rounded to FP32), input shift/scale (v_scale != 0) and output
 *   scale (> 0); resets the Adam state.  sq_cnn_get_params: read them back.
 * sq_cnn_forward(net, n1, n2, n3, V, rho): V, rho device N FP64.
 * sq_cnn_set_shift(net, shift): an extra constant subtracted from V before
 *   the input scaling, x0 = (V - v_shift - shift)/v_scale, in every later
 *   forward and backward call (0 after sq_cnn_set_params).  With shift =
 *   the Fermi level the network maps V - mu to rho.
 * sq_cnn_forward_sum(net, n1, n2, n3, V, rho, sum_host): the forward pass
 *   and sum_q rho_q (HOST output; fixed-order reduction; synchronises).
 * sq_cnn_backward(net, n1, n2, n3, V, rho_ref, rho, accumulate, loss_host):
 *   forward into rho, the loss against rho_ref (all device N FP64) into
 *   loss_host (HOST, may be NULL; synchronises when given), and the
 *   gradient of the loss with respect to every parameter, stored in the net
 *   (accumulate = 1 adds it to the stored gradient, e.g. over a batch of
 *   systems).  sq_cnn_get_grads(net, grads_host): read it (natural order).
 * sq_cnn_adam_step(net, lr, beta1, beta2, eps, grad_scale): one Adam step
 *   (Kingma and Ba) on the stored gradient times grad_scale:
 *   m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 *   w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 * sq_cnn_destroy(net): release (NULL: no-op).
 * Grids up to 2^28 nodes, each edge 1..4096; argument errors SQ_EINVAL.
 * ------------------------------------------------------------------------- */
typedef struct sq_cnn sq_cnn;
long long sq_cnn_param_count(int channels);
int sq_cnn_create(sq_cnn **out, int channels, int bf16, void *cuda_stream);
int sq_cnn_set_params(sq_cnn *net, const double *params_host, double v_shift, double v_scale,
                      double rho_scale);
int sq_cnn_get_params(sq_cnn *net, double *params_host);
int sq_cnn_forward(sq_cnn *net, int n1, int n2, int n3, const double *V, double *rho);
int sq_cnn_set_shift(sq_cnn *net, double shift);
int sq_cnn_forward_sum(sq_cnn *net, int n1, int n2, int n3, const double *V, double *rho,
                       double *sum_host);
int sq_cnn_backward(sq_cnn *net, int n1, int n2, int n3, const double *V, const double *rho_ref,
                    double *rho, int accumulate, double *loss_host);
int sq_cnn_get_grads(sq_cnn *net, double *grads_host);
int sq_cnn_adam_step(sq_cnn *net, double lr, double beta1, double beta2, double eps, double grad_scale);
void sq_cnn_destroy(sq_cnn *net);

/* Wait for the context's stream and return any latched device error. */
int sq_sync(sq_ctx *ctx);

/* Number of kernel launches this context has enqueued since creation. */
long long sq_launch_count(const sq_ctx *ctx);

/* Launch configuration the context chose (host only, no synchronisation).
 * info_host: HOST array of n >= 4 ints receiving
 *   [0] m, the region half-width in grid points (region side 2m+1);
 *   [1] the largest number of projector candidates of any node;
 *   [2] where the per-candidate projector tables live during the region
 *       kernels: 0 global scratch, 1 all in shared memory, 2 the tables every
 *       step reads in shared memory and the rest in global scratch;
 *   [3] resident CTAs of the region kernels (per-CTA scratch slices).
 * SQ_EINVAL for a NULL context or n < 4. */
int sq_context_info(const sq_ctx *ctx, int *info_host, int n);

/* Release all device memory of the context (NULL is a no-op). */
void sq_destroy(sq_ctx *ctx);

/* Static description of a status code. */
const char *sq_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* SQ_H */
