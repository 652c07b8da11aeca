/*
 * sq_oracle.c -- plain, serial, FP64 CPU oracle for the Clenshaw-Curtis
 * Spectral Quadrature (SQ) hot path of Suryanarayana et al., "SQDFT: Spectral
 * Quadrature method for large-scale parallel O(N) Kohn-Sham calculations at
 * high temperature" (arXiv:1708.07913).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that the
 * CUDA path is compared against.  Only tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or constant with the CUDA library, and the CUDA library never calls it.
 *
 * Everything is written the slow, obvious way: one node at a time, the nodal
 * Hamiltonian applied matrix-free with explicit loops, sums in natural order.
 *
 * Parity status: every function below is pinned by tests under tests/
 * (closed forms, textbook finite-difference coefficients, dense
 * diagonalisation, invariants); none is "parity unpinned".
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_NO 16

/* ------------------------------------------------------------------------ */
/* System description (mirrors the ctypes Structure in oracle/__init__.py).  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n1, n2, n3;          /* grid points per axis (periodic cell)          */
    double h;                /* mesh spacing, bohr                             */
    int no;                  /* FD half order n_o (Section 3.1)                */
    int m;                   /* region half-width in points, floor(R_cut/h)    */
    int periodic;            /* 0: infinite-cell cube (zero Dirichlet outside) */
                             /* 1: region = whole periodic cell                */
    const double *V;         /* n1*n2*n3 effective potential, x fastest        */
    int n_atoms;
    const double *R;         /* n_atoms*3 positions, bohr                      */
    int n_ptypes;            /* projector channels per atom                    */
    const int *pl;           /* angular momentum of each channel (0 or 1)      */
    const double *pgamma;    /* KB energy of each channel, Ha                  */
    const double *prc;       /* Gaussian width of each channel, bohr           */
    const double *prnl;      /* support radius of each channel, bohr           */
} or_sys;

/* ------------------------------------------------------------------------ */
/* Section 3.1, Eq. (FD:Laplacian): central finite-difference weights.       */
/*   w_0 = -(1/h^2) sum_{q=1}^{n_o} 1/q^2                                    */
/*   w_d = 2(-1)^{d+1} (n_o!)^2 / (h^2 d^2 (n_o-d)! (n_o+d)!),  d = 1..n_o   */
/* The d = 0 term of the 3-D sum appears once per +-axis term, i.e. 6 times. */
/* ------------------------------------------------------------------------ */
static double factorial(int k) { double f = 1.0; for (int i = 2; i <= k; ++i) f *= i; return f; }

int or_fd_weights(int no, double h, double *w)
{
    if (no < 1 || no > OR_MAX_NO || !(h > 0.0)) return 1;
    double s = 0.0;
    for (int q = 1; q <= no; ++q) s += 1.0 / ((double)q * q);
    w[0] = -s / (h * h);
    for (int d = 1; d <= no; ++d) {
        double sign = (d % 2 == 1) ? 1.0 : -1.0;   /* (-1)^{d+1} */
        w[d] = 2.0 * sign / (h * h * d * d) * factorial(no) * factorial(no)
               / (factorial(no - d) * factorial(no + d));
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Nodal Hamiltonian H_q (Section 3.1, region of influence; Eq. Hamiltonian) */
/*   H_q = -1/2 Lap_h + V_eff + V_nl restricted to the cube of side 2m+1     */
/* centred at node q.  Stencil neighbours outside the cube are dropped (zero  */
/* Dirichlet); V is looked up through the periodic index map of Section 3.1. */
/* In periodic mode the region is the whole cell and the stencil wraps.      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int npts;                /* support points inside the region */
    int *idx;                /* region point indices             */
    double *val;             /* projector values chi(x)          */
    double gamma;            /* KB energy                        */
    int atom;                /* atom the projector belongs to    */
} or_proj;

typedef struct {
    int S1, S2, S3;          /* region dims                                  */
    long Ns;                 /* S1*S2*S3                                     */
    int periodic;
    int no;
    double w[OR_MAX_NO + 1];
    double h;
    double *vloc;            /* V at region points                           */
    long centre;             /* index of node q inside the region            */
    int nproj;
    or_proj *proj;
} or_op;

static long wrap(long i, long n) { long r = i % n; return r < 0 ? r + n : r; }
static long floor_div(long a, long b) { long q = a / b; if ((a % b != 0) && ((a < 0) != (b < 0))) --q; return q; }
static long ceil_div(long a, long b) { return -floor_div(-a, b); }

/* Gaussian KB projectors (form fixed by the synthetic workload; the paper    */
/* uses Troullier-Martins projectors, Section 4):                             */
/*   s: A_s exp(-r^2/(2 rc^2)),        A_s = (pi rc^2)^(-3/4)                */
/*   p: A_p r_a exp(-r^2/(2 rc^2)),    A_p = (sqrt(2)/rc) (pi rc^2)^(-3/4)   */
/* with support |r| < r_nl.  Displacements are formed as I*h - R_a where I is */
/* the grid index relative to the atom's own image (integer shift exact).    */
static double proj_value(int l, int comp, double rc, double dx, double dy, double dz)
{
    double r2 = dx * dx + dy * dy + dz * dz;
    double g = exp(-r2 / (2.0 * rc * rc));
    double As = pow(M_PI * rc * rc, -0.75);
    if (l == 0) return As * g;
    double Ap = sqrt(2.0) / rc * As;
    double ra = (comp == 0) ? dx : (comp == 1) ? dy : dz;
    return Ap * ra * g;
}

static void op_add_proj(or_op *op, int npts, const int *idx, const double *val, double gamma, int atom)
{
    op->proj = (or_proj *)realloc(op->proj, sizeof(or_proj) * (op->nproj + 1));
    or_proj *p = &op->proj[op->nproj++];
    p->npts = npts;
    p->idx = (int *)malloc(sizeof(int) * (npts > 0 ? npts : 1));
    p->val = (double *)malloc(sizeof(double) * (npts > 0 ? npts : 1));
    memcpy(p->idx, idx, sizeof(int) * npts);
    memcpy(p->val, val, sizeof(double) * npts);
    p->gamma = gamma;
    p->atom = atom;
}

static void op_free(or_op *op)
{
    if (!op) return;
    for (int i = 0; i < op->nproj; ++i) { free(op->proj[i].idx); free(op->proj[i].val); }
    free(op->proj);
    free(op->vloc);
    free(op);
}

/* Build H_q for node q (flat index, x fastest). */
static or_op *op_build(const or_sys *s, long q)
{
    or_op *op = (or_op *)calloc(1, sizeof(or_op));
    long n1 = s->n1, n2 = s->n2, n3 = s->n3;
    long qi = q % n1, qj = (q / n1) % n2, qk = q / (n1 * n2);
    op->periodic = s->periodic;
    op->no = s->no;
    op->h = s->h;
    or_fd_weights(s->no, s->h, op->w);
    if (s->periodic) { op->S1 = (int)n1; op->S2 = (int)n2; op->S3 = (int)n3; }
    else { op->S1 = op->S2 = op->S3 = 2 * s->m + 1; }
    op->Ns = (long)op->S1 * op->S2 * op->S3;
    op->vloc = (double *)malloc(sizeof(double) * op->Ns);
    /* unwrapped grid index of region point (a, b, c) = origin + (a, b, c) */
    long o1 = s->periodic ? 0 : qi - s->m;
    long o2 = s->periodic ? 0 : qj - s->m;
    long o3 = s->periodic ? 0 : qk - s->m;
    for (long c = 0; c < op->S3; ++c)
        for (long b = 0; b < op->S2; ++b)
            for (long a = 0; a < op->S1; ++a)
                op->vloc[a + op->S1 * (b + op->S2 * c)] =
                    s->V[wrap(o1 + a, n1) + n1 * (wrap(o2 + b, n2) + n2 * wrap(o3 + c, n3))];
    op->centre = s->periodic ? q : (long)s->m + op->S1 * ((long)s->m + op->S2 * (long)s->m);

    /* projectors: every atom image whose support sphere meets the region */
    int *tidx = (int *)malloc(sizeof(int) * op->Ns);
    double *tval = (double *)malloc(sizeof(double) * op->Ns);
    double *dense = s->periodic ? (double *)malloc(sizeof(double) * op->Ns) : NULL;
    for (int t = 0; t < s->n_ptypes; ++t) {
        int l = s->pl[t];
        double rc = s->prc[t], rnl = s->prnl[t], gam = s->pgamma[t];
        int ncomp = (l == 0) ? 1 : 3;
        for (int I = 0; I < s->n_atoms; ++I) {
            const double *R = &s->R[3 * I];
            /* atom-relative grid index range of the support */
            long lo1 = (long)ceil((R[0] - rnl) / s->h), hi1 = (long)floor((R[0] + rnl) / s->h);
            long lo2 = (long)ceil((R[1] - rnl) / s->h), hi2 = (long)floor((R[1] + rnl) / s->h);
            long lo3 = (long)ceil((R[2] - rnl) / s->h), hi3 = (long)floor((R[2] + rnl) / s->h);
            for (int comp = 0; comp < ncomp; ++comp) {
                if (s->periodic) {
                    /* periodised projector: sum over all images, folded into the cell */
                    for (long p = 0; p < op->Ns; ++p) dense[p] = 0.0;
                    int any = 0;
                    for (long K = lo3; K <= hi3; ++K)
                        for (long J = lo2; J <= hi2; ++J)
                            for (long Ii = lo1; Ii <= hi1; ++Ii) {
                                double dx = Ii * s->h - R[0], dy = J * s->h - R[1], dz = K * s->h - R[2];
                                if (dx * dx + dy * dy + dz * dz >= rnl * rnl) continue;
                                long p = wrap(Ii, n1) + n1 * (wrap(J, n2) + n2 * wrap(K, n3));
                                dense[p] += proj_value(l, comp, rc, dx, dy, dz);
                                any = 1;
                            }
                    if (!any) continue;
                    int np = 0;
                    for (long p = 0; p < op->Ns; ++p)
                        if (dense[p] != 0.0) { tidx[np] = (int)p; tval[np] = dense[p]; ++np; }
                    op_add_proj(op, np, tidx, tval, gam, I);
                } else {
                    /* image shifts e for which the support box [lo+e n, hi+e n] meets */
                    /* the region [o, o+S-1] along every axis                          */
                    long S = op->S1;
                    long e1lo = ceil_div(o1 - hi1, n1), e1hi = floor_div(o1 + S - 1 - lo1, n1);
                    long e2lo = ceil_div(o2 - hi2, n2), e2hi = floor_div(o2 + S - 1 - lo2, n2);
                    long e3lo = ceil_div(o3 - hi3, n3), e3hi = floor_div(o3 + S - 1 - lo3, n3);
                    for (long e3 = e3lo; e3 <= e3hi; ++e3)
                        for (long e2 = e2lo; e2 <= e2hi; ++e2)
                            for (long e1 = e1lo; e1 <= e1hi; ++e1) {
                                int np = 0;
                                for (long c = 0; c < S; ++c) {
                                    long K = o3 + c - e3 * n3;      /* index relative to this image */
                                    if (K < lo3 || K > hi3) continue;
                                    for (long b = 0; b < S; ++b) {
                                        long J = o2 + b - e2 * n2;
                                        if (J < lo2 || J > hi2) continue;
                                        long alo = lo1 + e1 * n1 - o1, ahi = hi1 + e1 * n1 - o1;
                                        if (alo < 0) alo = 0;
                                        if (ahi > S - 1) ahi = S - 1;
                                        for (long a = alo; a <= ahi; ++a) {
                                            long Ii = o1 + a - e1 * n1;
                                            double dx = Ii * s->h - R[0], dy = J * s->h - R[1], dz = K * s->h - R[2];
                                            if (dx * dx + dy * dy + dz * dz >= rnl * rnl) continue;
                                            tidx[np] = (int)(a + S * (b + S * c));
                                            tval[np] = proj_value(l, comp, rc, dx, dy, dz);
                                            ++np;
                                        }
                                    }
                                }
                                if (np > 0) op_add_proj(op, np, tidx, tval, gam, I);
                            }
                }
            }
        }
    }
    free(tidx); free(tval); free(dense);
    return op;
}

/* y = H_q x.  Kinetic part: -1/2 sum_{d=0}^{n_o} w_d (six neighbours at     */
/* distance d), the d = 0 term giving -3 w_0 on the diagonal.                */
/* Nonlocal part: sum_p gamma_p chi_p h^3 <chi_p, x> (trapezoidal rule,      */
/* Eq. IntApprox).                                                           */
static void op_apply(const or_op *op, const double *x, double *y)
{
    int S1 = op->S1, S2 = op->S2, S3 = op->S3;
    for (int c = 0; c < S3; ++c)
        for (int b = 0; b < S2; ++b)
            for (int a = 0; a < S1; ++a) {
                long p = a + (long)S1 * (b + (long)S2 * c);
                double acc = (-3.0 * op->w[0] + op->vloc[p]) * x[p];
                for (int d = 1; d <= op->no; ++d) {
                    double nb = 0.0;
                    int ap = a + d, am = a - d, bp = b + d, bm = b - d, cp = c + d, cm = c - d;
                    if (op->periodic) {
                        ap = (int)wrap(ap, S1); am = (int)wrap(am, S1);
                        bp = (int)wrap(bp, S2); bm = (int)wrap(bm, S2);
                        cp = (int)wrap(cp, S3); cm = (int)wrap(cm, S3);
                    }
                    if (ap < S1) nb += x[ap + (long)S1 * (b + (long)S2 * c)];
                    if (am >= 0) nb += x[am + (long)S1 * (b + (long)S2 * c)];
                    if (bp < S2) nb += x[a + (long)S1 * (bp + (long)S2 * c)];
                    if (bm >= 0) nb += x[a + (long)S1 * (bm + (long)S2 * c)];
                    if (cp < S3) nb += x[a + (long)S1 * (b + (long)S2 * cp)];
                    if (cm >= 0) nb += x[a + (long)S1 * (b + (long)S2 * cm)];
                    acc += -0.5 * op->w[d] * nb;
                }
                y[p] = acc;
            }
    double h3 = op->h * op->h * op->h;
    for (int i = 0; i < op->nproj; ++i) {
        const or_proj *pj = &op->proj[i];
        double dot = 0.0;
        for (int k = 0; k < pj->npts; ++k) dot += pj->val[k] * x[pj->idx[k]];
        double coef = pj->gamma * h3 * dot;
        for (int k = 0; k < pj->npts; ++k) y[pj->idx[k]] += coef * pj->val[k];
    }
}

/* ------------------------------------------------------------------------ */
/* Public helpers for tests: region size, matrix-free apply, dense H_q.      */
/* ------------------------------------------------------------------------ */
long or_region_size(const or_sys *s)
{
    if (s->periodic) return (long)s->n1 * s->n2 * s->n3;
    long S = 2L * s->m + 1;
    return S * S * S;
}

int or_apply_H(const or_sys *s, long q, const double *x, double *y)
{
    or_op *op = op_build(s, q);
    op_apply(op, x, y);
    op_free(op);
    return 0;
}

/* H (Ns x Ns, row-major) built column by column from the matrix-free apply. */
int or_dense_H(const or_sys *s, long q, double *H)
{
    or_op *op = op_build(s, q);
    long N = op->Ns;
    double *e = (double *)calloc(N, sizeof(double));
    double *col = (double *)malloc(sizeof(double) * N);
    for (long j = 0; j < N; ++j) {
        e[j] = 1.0;
        op_apply(op, e, col);
        for (long i = 0; i < N; ++i) H[i * N + j] = col[i];
        e[j] = 0.0;
    }
    free(e); free(col); op_free(op);
    return 0;
}

/* Number of projector vectors that H_q carries (atom images x components). */
int or_num_projectors(const or_sys *s, long q)
{
    or_op *op = op_build(s, q);
    int n = op->nproj;
    op_free(op);
    return n;
}

/* ------------------------------------------------------------------------ */
/* Section 3.2 (text after Eq. rhoqj): lambda_min and lambda_max of H_q by   */
/* the Lanczos method.  Start vector uniform 1/sqrt(Ns); a fixed number of   */
/* steps without re-orthogonalisation; stop early only on breakdown          */
/* (beta <= 1e-10 * scale).  The extreme Ritz values are the extreme         */
/* eigenvalues of the tridiagonal T_k, found by Sturm-sequence bisection.    */
/* ------------------------------------------------------------------------ */

/* number of eigenvalues of T (diag a[0..k-1], offdiag b[0..k-2]) below x */
static int sturm_count(int k, const double *a, const double *b, double x)
{
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < k; ++i) {
        double bb = (i > 0) ? b[i - 1] * b[i - 1] : 0.0;
        d = (a[i] - x) - (i > 0 ? bb / d : 0.0);
        if (d == 0.0) d = -1e-300;          /* x is an eigenvalue of a leading block: count it */
        if (d < 0.0) ++cnt;
    }
    return cnt;
}

int or_tridiag_extremes(int k, const double *a, const double *b, double *lmin, double *lmax)
{
    if (k < 1) return 1;
    double glo = INFINITY, ghi = -INFINITY;      /* Gershgorin enclosure */
    for (int i = 0; i < k; ++i) {
        double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < k - 1 ? fabs(b[i]) : 0.0);
        if (a[i] - r < glo) glo = a[i] - r;
        if (a[i] + r > ghi) ghi = a[i] + r;
    }
    double pad = 1e-12 * (fabs(glo) + fabs(ghi)) + 1e-300;
    glo -= pad; ghi += pad;
    /* lambda_min: smallest x with count(x) >= 1 */
    double lo = glo, hi = ghi;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (sturm_count(k, a, b, mid) >= 1) hi = mid; else lo = mid;
    }
    *lmin = 0.5 * (lo + hi);
    /* lambda_max: largest x with count(x) <= k-1 */
    lo = glo; hi = ghi;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (sturm_count(k, a, b, mid) >= k) hi = mid; else lo = mid;
    }
    *lmax = 0.5 * (lo + hi);
    return 0;
}

/* Lanczos recurrence on H_q; returns the number of steps k actually taken  */
/* and fills alpha[0..k-1], beta[0..k-2].                                    */
static int lanczos_op(const or_op *op, int nsteps, double *alpha, double *beta)
{
    long N = op->Ns;
    double *v = (double *)malloc(sizeof(double) * N);
    double *vold = (double *)calloc(N, sizeof(double));
    double *w = (double *)malloc(sizeof(double) * N);
    double inv = 1.0 / sqrt((double)N);
    for (long i = 0; i < N; ++i) v[i] = inv;
    double bprev = 0.0, scale = 0.0;
    int k = 0;
    for (int it = 0; it < nsteps; ++it) {
        op_apply(op, v, w);
        for (long i = 0; i < N; ++i) w[i] -= bprev * vold[i];
        double a = 0.0;
        for (long i = 0; i < N; ++i) a += w[i] * v[i];
        for (long i = 0; i < N; ++i) w[i] -= a * v[i];
        double b2 = 0.0;
        for (long i = 0; i < N; ++i) b2 += w[i] * w[i];
        double b = sqrt(b2);
        alpha[it] = a;
        k = it + 1;
        if (it == nsteps - 1) break;
        if (fabs(a) + bprev > scale) scale = fabs(a) + bprev;
        if (b <= 1e-10 * scale) break;              /* invariant subspace reached */
        beta[it] = b;
        for (long i = 0; i < N; ++i) { vold[i] = v[i]; v[i] = w[i] / b; }
        bprev = b;
    }
    free(v); free(vold); free(w);
    return k;
}

int or_lanczos_tridiag(const or_sys *s, long q, int nsteps, double *alpha, double *beta, int *k_out)
{
    or_op *op = op_build(s, q);
    *k_out = lanczos_op(op, nsteps, alpha, beta);
    op_free(op);
    return 0;
}

/* chi_q = (lmax+lmin)/2, zeta_q = (lmax-lmin)/2 (Section 3.2) after widening */
/* both ends by margin * max(theta_max - theta_min, 1 Ha).                    */
int or_bounds(const or_sys *s, long nq, const long *nodes, int n_lanczos, double margin,
              double *chi, double *zeta)
{
    if (n_lanczos < 1) return 1;
    double *a = (double *)malloc(sizeof(double) * n_lanczos);
    double *b = (double *)malloc(sizeof(double) * n_lanczos);
    for (long t = 0; t < nq; ++t) {
        or_op *op = op_build(s, nodes[t]);
        int k = lanczos_op(op, n_lanczos, a, b);
        op_free(op);
        double tmin, tmax;
        or_tridiag_extremes(k, a, b, &tmin, &tmax);
        double width = tmax - tmin;
        if (width < 1.0) width = 1.0;
        double lo = tmin - margin * width, hi = tmax + margin * width;
        chi[t] = 0.5 * (hi + lo);
        zeta[t] = 0.5 * (hi - lo);
    }
    free(a); free(b);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Section 3.2, Eq. (Rec:FD) and Eq. (rhoqj): Chebyshev moments.             */
/*   Hhat_q = (H_q - chi_q I)/zeta_q                                         */
/*   t^0 = w_q (unit vector at the node), t^1 = Hhat t^0,                    */
/*   t^{i+1} = 2 Hhat t^i - t^{i-1}                                          */
/* product_rule = 0: the plain definition rho^j = w_q^T t^j for j = 0..npl.  */
/* product_rule = 1: recurrence only to npl/2; higher moments from the       */
/*   product property 2 T_a T_b = T_{a+b} + T_{|a-b|}:                       */
/*     rho^{2a}   = 2 t^a . t^a     - rho^0                                  */
/*     rho^{2a+1} = 2 t^{a+1} . t^a - rho^1                                  */
/*   (the printed Eq. rhoqj has the two terms' signs swapped; the identity   */
/*   in the footnote of Section 3.2 fixes them as written here).             */
/* ------------------------------------------------------------------------ */
static void hhat_apply(const or_op *op, double chi, double zeta, const double *x, double *y)
{
    op_apply(op, x, y);
    for (long i = 0; i < op->Ns; ++i) y[i] = (y[i] - chi * x[i]) / zeta;
}

int or_moments(const or_sys *s, long nq, const long *nodes, const double *chi, const double *zeta,
               int npl, int product_rule, double *mom)
{
    if (npl < 2 || (product_rule && npl % 2 != 0)) return 1;
    for (long t = 0; t < nq; ++t) {
        or_op *op = op_build(s, nodes[t]);
        long N = op->Ns, c = op->centre;
        int last = product_rule ? npl / 2 : npl;
        double **tv = (double **)malloc(sizeof(double *) * (last + 1));
        for (int i = 0; i <= last; ++i) tv[i] = (double *)calloc(N, sizeof(double));
        tv[0][c] = 1.0;
        hhat_apply(op, chi[t], zeta[t], tv[0], tv[1]);
        for (int i = 1; i < last; ++i) {
            hhat_apply(op, chi[t], zeta[t], tv[i], tv[i + 1]);
            for (long p = 0; p < N; ++p) tv[i + 1][p] = 2.0 * tv[i + 1][p] - tv[i - 1][p];
        }
        double *out = &mom[t * (npl + 1)];
        for (int j = 0; j <= last; ++j) out[j] = tv[j][c];
        if (product_rule) {
            for (int j = last + 1; j <= npl; ++j) {
                int a = j / 2;
                double dot = 0.0;
                if (j % 2 == 0) {
                    for (long p = 0; p < N; ++p) dot += tv[a][p] * tv[a][p];
                    out[j] = 2.0 * dot - out[0];
                } else {
                    for (long p = 0; p < N; ++p) dot += tv[a + 1][p] * tv[a][p];
                    out[j] = 2.0 * dot - out[1];
                }
            }
        }
        for (int i = 0; i <= last; ++i) free(tv[i]);
        free(tv);
        op_free(op);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Section 3.2, Eq. (cqj), evaluated by discrete orthogonality at the        */
/* npl+1 zeros x_k = cos(pi (k+1/2)/(npl+1)) of T_{npl+1}.  The coefficients */
/* c^j are folded into per-node quadrature weights                           */
/*   W_k = (2/(npl+1)) sum'_{j=0}^{npl} rho^j T_j(x_k)  (j = 0 term halved)   */
/* so that sum_j c^j rho^j = sum_k W_k f(x_k) for the interpolant of f.      */
/* ------------------------------------------------------------------------ */
double or_cheb_node(int npl, int k) { return cos(M_PI * (k + 0.5) / (npl + 1)); }

int or_cc_weights(long nq, int npl, const double *mom, double *W)
{
    int K = npl + 1;
    for (long t = 0; t < nq; ++t) {
        const double *r = &mom[t * K];
        for (int k = 0; k < K; ++k) {
            double x = or_cheb_node(npl, k);
            double Tm1 = 1.0, T = x;                    /* T_0, T_1 */
            double s = 0.5 * r[0];
            for (int j = 1; j < K; ++j) {
                s += r[j] * T;
                double Tn = 2.0 * x * T - Tm1;
                Tm1 = T; T = Tn;
            }
            W[t * K + k] = 2.0 / K * s;
        }
    }
    return 0;
}

/* Fermi-Dirac function of Eq. (DensityMatrix): g(E) = 1/(1+exp((E-mu)/sigma)) */
static double fermi(double E, double mu, double kT) { return 1.0 / (1.0 + exp((E - mu) / kT)); }

/* Electron count 2 sum_q sum_j c_q^j rho_q^j = 2 sum_q sum_k W_qk g(chi_q + zeta_q x_k) */
double or_electron_count(long nq, int npl, const double *W, const double *chi, const double *zeta,
                         double mu, double kT)
{
    int K = npl + 1;
    double N = 0.0;
    for (long t = 0; t < nq; ++t)
        for (int k = 0; k < K; ++k)
            N += 2.0 * W[t * K + k] * fermi(chi[t] + zeta[t] * or_cheb_node(npl, k), mu, kT);
    return N;
}

/* Section 3.2: the Fermi level solves 2 sum sum c rho = N_e.  Bisection on  */
/* [min(chi-zeta) - 10 kT, max(chi+zeta) + 10 kT]; stop when the midpoint    */
/* equals an end point in FP64, or after 200 steps.  Returns 4 if the        */
/* bracket does not straddle N_e.                                            */
int or_fermi_level(long nq, int npl, const double *W, const double *chi, const double *zeta,
                   double Ne, double kT, double *mu_out, int *iters_out)
{
    double lo = INFINITY, hi = -INFINITY;
    for (long t = 0; t < nq; ++t) {
        if (chi[t] - zeta[t] < lo) lo = chi[t] - zeta[t];
        if (chi[t] + zeta[t] > hi) hi = chi[t] + zeta[t];
    }
    lo -= 10.0 * kT; hi += 10.0 * kT;
    double Nlo = or_electron_count(nq, npl, W, chi, zeta, lo, kT);
    double Nhi = or_electron_count(nq, npl, W, chi, zeta, hi, kT);
    if (!(Nlo <= Ne && Nhi >= Ne)) { *mu_out = NAN; *iters_out = 0; return 4; }
    int it;
    for (it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (or_electron_count(nq, npl, W, chi, zeta, mid, kT) < Ne) lo = mid; else hi = mid;
    }
    *mu_out = 0.5 * (lo + hi);
    *iters_out = it;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. (ElectronDensity), Eq. (Eband)/(d_q), Eq. (Entropy)/(e_q):            */
/*   rho_q  = (2/h^3) sum_k W_qk g_qk                                        */
/*   E_band = 2 sum_q sum_k W_qk (chi_q + zeta_q x_k) g_qk                    */
/*   E_ent  = 2 sigma sum_q sum_k W_qk [g ln g + (1-g) ln(1-g)],  0 ln 0 = 0  */
/*   N      = h^3 sum_q rho_q                                                */
/* with the d and e coefficients taken as the interpolants of r g(r) and of  */
/* the entropy function at the same nodes (discrete orthogonality).          */
/* ------------------------------------------------------------------------ */
int or_density_energy(long nq, int npl, const double *W, const double *chi, const double *zeta,
                      double mu, double kT, double h, double *rho,
                      double *e_band, double *e_ent, double *n_elec)
{
    int K = npl + 1;
    double h3 = h * h * h;
    double eb = 0.0, es = 0.0, ne = 0.0;
    for (long t = 0; t < nq; ++t) {
        double r = 0.0;
        for (int k = 0; k < K; ++k) {
            double E = chi[t] + zeta[t] * or_cheb_node(npl, k);
            double x = (E - mu) / kT;
            double g = 1.0 / (1.0 + exp(x));
            double gm = 1.0 / (1.0 + exp(-x));            /* 1 - g */
            double wk = W[t * K + k];
            r += wk * g;
            eb += 2.0 * wk * E * g;
            double sfun = 0.0;
            if (g > 0.0) sfun += g * log(g);
            if (gm > 0.0) sfun += gm * log(gm);
            es += 2.0 * kT * wk * sfun;
        }
        rho[t] = 2.0 / h3 * r;
        ne += h3 * rho[t];
    }
    *e_band = eb; *e_ent = es; *n_elec = ne;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Nonlocal component of the atomic force (Section 3.4, Eq. Discrete:NLforce */
/* with the recurrence of Eq. Rec:FD1 run to n_pl):                           */
/*   f_I^nl = -4 sum_q sum_{p of atom I} gamma_p h^3 chi_p(q) chi_p^T grad_h D_q */
/* D_q = sum_{j=0}^{npl} c^j t^j (t^0 = e_q, t^1 = Hhat e_q, t^{j+1} = 2 Hhat  */
/* t^j - t^{j-1}), the node's column of the density matrix in its region;     */
/* c^j the Chebyshev interpolation coefficients of the Fermi-Dirac function   */
/* g((chi_q + zeta_q x - mu)/kT) at the npl+1 zeros x_k (c^0 halved, the      */
/* discrete orthogonality of the density calculation); grad_h the central     */
/* finite-difference gradient of Eq. FD:Gradient inside the region (zero      */
/* outside it; wrapped in periodic mode).  V_nl^{I'} = gamma h^3 chi chi^T    */
/* per projector, every image of the atom included.  Adds into F[3*I+a].      */
/* ------------------------------------------------------------------------ */
static void grad_apply(const or_op *op, const double *wt, int axis, const double *x, double *y)
{
    int S1 = op->S1, S2 = op->S2, S3 = op->S3;
    for (int c = 0; c < S3; ++c)
        for (int b = 0; b < S2; ++b)
            for (int a = 0; a < S1; ++a) {
                double acc = 0.0;
                for (int d = 1; d <= op->no; ++d) {
                    int pa = a, pb = b, pc = c, ma = a, mb = b, mc = c;
                    if (axis == 0) { pa += d; ma -= d; }
                    else if (axis == 1) { pb += d; mb -= d; }
                    else { pc += d; mc -= d; }
                    double xp = 0.0, xm = 0.0;
                    if (op->periodic) {
                        xp = x[wrap(pa, S1) + S1 * (wrap(pb, S2) + S2 * wrap(pc, S3))];
                        xm = x[wrap(ma, S1) + S1 * (wrap(mb, S2) + S2 * wrap(mc, S3))];
                    } else {
                        if (pa < S1 && pb < S2 && pc < S3) xp = x[pa + S1 * (pb + S2 * pc)];
                        if (ma >= 0 && mb >= 0 && mc >= 0) xm = x[ma + S1 * (mb + S2 * mc)];
                    }
                    acc += wt[d] * (xp - xm);
                }
                y[a + S1 * (b + S2 * c)] = acc;
            }
}

/* Eq. (FD:Gradient): central first-derivative weights
 *   wt_d = (-1)^{d+1} (n_o!)^2 / (h d (n_o-d)! (n_o+d)!),  d = 1..n_o,
 * so that f'(x) ~ sum_d wt_d (f(x + d h) - f(x - d h)); wt[0] = 0. */
int or_grad_weights(int no, double h, double *wt)
{
    if (no < 1 || no > OR_MAX_NO || !(h > 0.0)) return 1;
    wt[0] = 0.0;
    for (int d = 1; d <= no; ++d) {
        double sign = (d % 2 == 1) ? 1.0 : -1.0;             /* (-1)^{d+1} */
        wt[d] = sign / (h * d) * factorial(no) * factorial(no) / (factorial(no - d) * factorial(no + d));
    }
    return 0;
}

int or_nl_force(const or_sys *s, long nq, const long *nodes, const double *chi, const double *zeta, int npl,
                double mu, double kT, double *F)
{
    if (npl < 1 || !(kT > 0.0)) return 1;
    const int no = s->no;
    double wt[OR_MAX_NO + 1];
    if (or_grad_weights(no, s->h, wt)) return 1;
    const double h3 = s->h * s->h * s->h;
    double *c = (double *)malloc(sizeof(double) * (npl + 1));
    for (long iq = 0; iq < nq; ++iq) {
        or_op *op = op_build(s, nodes[iq]);
        const long N = op->Ns, ctr = op->centre;
        /* projectors that are non-zero at the node */
        int any = 0;
        for (int p = 0; p < op->nproj; ++p)
            for (int k = 0; k < op->proj[p].npts; ++k)
                if (op->proj[p].idx[k] == ctr) any = 1;
        if (!any) { op_free(op); continue; }
        /* c^j by discrete orthogonality at the zeros of T_{npl+1} */
        for (int j = 0; j <= npl; ++j) {
            double acc = 0.0;
            for (int k = 0; k <= npl; ++k) {
                double x = or_cheb_node(npl, k);
                acc += fermi(chi[iq] + zeta[iq] * x, mu, kT) * cos(j * acos(x));
            }
            c[j] = 2.0 / (npl + 1) * acc;
        }
        c[0] *= 0.5;
        double *tm = (double *)calloc(N, sizeof(double)), *t = (double *)calloc(N, sizeof(double));
        double *tn = (double *)malloc(sizeof(double) * N), *D = (double *)calloc(N, sizeof(double));
        double *g = (double *)malloc(sizeof(double) * N);
        tm[ctr] = 1.0;                                        /* t^0 = e_q */
        hhat_apply(op, chi[iq], zeta[iq], tm, t);             /* t^1       */
        for (long i = 0; i < N; ++i) D[i] = c[0] * tm[i] + (npl >= 1 ? c[1] * t[i] : 0.0);
        for (int j = 2; j <= npl; ++j) {
            hhat_apply(op, chi[iq], zeta[iq], t, tn);
            for (long i = 0; i < N; ++i) {
                tn[i] = 2.0 * tn[i] - tm[i];
                D[i] += c[j] * tn[i];
            }
            double *tmp = tm; tm = t; t = tn; tn = tmp;
        }
        for (int axis = 0; axis < 3; ++axis) {
            grad_apply(op, wt, axis, D, g);
            for (int p = 0; p < op->nproj; ++p) {
                const or_proj *pr = &op->proj[p];
                double chi_q = 0.0, proj = 0.0;
                for (int k = 0; k < pr->npts; ++k) {
                    if (pr->idx[k] == ctr) chi_q = pr->val[k];
                    proj += pr->val[k] * g[pr->idx[k]];
                }
                F[3 * pr->atom + axis] -= 4.0 * pr->gamma * h3 * chi_q * proj;
            }
        }
        free(tm); free(t); free(tn); free(D); free(g);
        op_free(op);
    }
    free(c);
    return 0;
}
