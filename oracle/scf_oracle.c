/*
 * scf_oracle.c -- plain, serial, FP64 CPU oracle for the pieces of the
 * self-consistent field (SCF) loop around the Spectral Quadrature path:
 * the periodic finite-difference Poisson solve for the electrostatic
 * potential (Eq. PoissonEqn, solved by conjugate gradients in place of the
 * paper's AAR, Section 3), Slater X-alpha exchange in place of the paper's
 * LDA (Section 3.3, energy), and Anderson mixing of the effective potential
 * in place of the paper's Periodic Pulay mixing (Section 3).
 *
 * TEST INFRASTRUCTURE ONLY, like sq_oracle.c: tests, the package's smoke
 * check and the benchmark's CPU leg are the only callers; it shares no code
 * with the CUDA library.
 *
 * Parity status: or_laplacian_periodic, or_poisson_cg, or_xalpha,
 * or_anderson_step and or_kerker are pinned by tests/test_oracle_scf.py
 * (discrete Fourier symbol of the operator, exact spectral solve, derivative
 * of the exchange energy, finite termination of Anderson mixing on linear
 * maps, the preconditioner's Fourier symbol); the SCF loop built from them
 * is pinned against dense diagonalisation, with and without the
 * preconditioner.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

int or_fd_weights(int no, double h, double *w);   /* sq_oracle.c, Eq. (FD:Laplacian) */

/* y = -lap_h x on the periodic n1 x n2 x n3 grid (x fastest), with the
 * central finite-difference weights of Eq. (FD:Laplacian): the d = 0 term of
 * its sum appears in all six +-axis terms, so
 *   lap_h x(p) = 6 w_0 x(p) + sum_axes sum_{d=1..no} w_d (x(p + d e) + x(p - d e)). */
int or_laplacian_periodic(int n1, int n2, int n3, double h, int no, const double *x, double *y)
{
    double w[17];
    if (no < 1 || no > 16 || or_fd_weights(no, h, w)) return 1;
    for (long k = 0; k < n3; ++k)
        for (long j = 0; j < n2; ++j)
            for (long i = 0; i < n1; ++i) {
                const long p = i + n1 * (j + n2 * k);
                double lap = 6.0 * w[0] * x[p];
                for (int d = 1; d <= no; ++d) {
                    lap += w[d] * (x[((i + d) % n1 + n1) % n1 + n1 * (j + n2 * k)] +
                                   x[((i - d) % n1 + n1) % n1 + n1 * (j + n2 * k)]);
                    lap += w[d] * (x[i + n1 * ((((j + d) % n2) + n2) % n2 + n2 * k)] +
                                   x[i + n1 * ((((j - d) % n2) + n2) % n2 + n2 * k)]);
                    lap += w[d] * (x[i + n1 * (j + n2 * ((((k + d) % n3) + n3) % n3))] +
                                   x[i + n1 * (j + n2 * ((((k - d) % n3) + n3) % n3))]);
                }
                y[p] = -lap;
            }
    return 0;
}

static double dot(long n, const double *a, const double *b)
{
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static void remove_mean(long n, double *x)
{
    double m = 0.0;
    for (long i = 0; i < n; ++i) m += x[i];
    m /= (double)n;
    for (long i = 0; i < n; ++i) x[i] -= m;
}

/* Electrostatic potential of the electron density on the periodic cell
 * (Eq. PoissonEqn): -(1/4 pi) lap_h phi = rho - rho_bar, the pseudocharges
 * replaced by the uniform neutralising background rho_bar = mean(rho); phi
 * has zero mean.  Conjugate gradients on A = -lap_h (symmetric, positive on
 * zero-mean grid functions, singular on constants) with b = 4 pi (rho -
 * rho_bar), from phi = 0, until ||b - A phi|| <= tol ||b|| or max_iter
 * iterations.  The constants are kept out: b and every search direction are
 * made mean-free, and b below 1e-13 of 4 pi ||rho|| (a neutral density up to
 * rounding) gives phi = 0.  Returns 0 on convergence, 2 if max_iter was
 * reached. */
int or_poisson_cg(int n1, int n2, int n3, double h, int no, const double *rho, double *phi, double tol,
                  int max_iter, int *iters, double *rel_resid)
{
    const long n = (long)n1 * n2 * n3;
    double *b = malloc(sizeof(double) * n), *r = malloc(sizeof(double) * n);
    double *p = malloc(sizeof(double) * n), *Ap = malloc(sizeof(double) * n);
    if (!b || !r || !p || !Ap) { free(b); free(r); free(p); free(Ap); return 1; }
    double mean = 0.0;
    for (long i = 0; i < n; ++i) mean += rho[i];
    mean /= (double)n;
    for (long i = 0; i < n; ++i) {
        b[i] = 4.0 * M_PI * (rho[i] - mean);
        phi[i] = 0.0;
    }
    remove_mean(n, b);
    for (long i = 0; i < n; ++i) {
        r[i] = b[i];
        p[i] = b[i];
    }
    double bnorm = sqrt(dot(n, b, b));
    if (bnorm <= 1e-13 * 4.0 * M_PI * sqrt(dot(n, rho, rho))) bnorm = 0.0;
    double rr = dot(n, r, r);
    int it = 0, status = 0;
    if (bnorm > 0.0) {
        while (sqrt(rr) > tol * bnorm) {
            if (it >= max_iter) { status = 2; break; }
            or_laplacian_periodic(n1, n2, n3, h, no, p, Ap);
            const double alpha = rr / dot(n, p, Ap);
            for (long i = 0; i < n; ++i) {
                phi[i] += alpha * p[i];
                r[i] -= alpha * Ap[i];
            }
            const double rr_new = dot(n, r, r);
            const double beta = rr_new / rr;
            for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
            remove_mean(n, p);
            rr = rr_new;
            ++it;
        }
        remove_mean(n, phi);
    } else {
        rr = 0.0;
    }
    *iters = it;
    *rel_resid = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
    free(b); free(r); free(p); free(Ap);
    return status;
}

/* Slater X-alpha exchange potential of the (spin-unpolarised) density:
 *   v_x(rho) = -(3 alpha / 2) (3 rho / pi)^(1/3),
 * the derivative of E_x = -(9 alpha / 8) (3/pi)^(1/3) int rho^(4/3); alpha =
 * 2/3 is the exchange of the uniform electron gas.  rho <= 0 gives 0. */
void or_xalpha(long n, const double *rho, double alpha, double *vx)
{
    for (long i = 0; i < n; ++i)
        vx[i] = rho[i] > 0.0 ? -1.5 * alpha * cbrt(3.0 * rho[i] / M_PI) : 0.0;
}

/* One Anderson mixing step for the fixed-point problem x = g(x) with
 * residual f = g(x) - x.  Xs and Fs hold the last mh + 1 iterates and
 * residuals (row-major (mh + 1) x n, oldest first, the current ones last).
 * With dX_i = x_{i+1} - x_i and dF_i = f_{i+1} - f_i, gamma minimises
 * || f - dF gamma ||_2 (normal equations, Gaussian elimination with partial
 * pivoting; a pivot below 1e-14 of the largest diagonal entry drops the
 * history, i.e. gamma = 0), and
 *   x_next = x + beta f - (dX + beta dF) gamma.
 * mh = 0 is simple mixing x + beta f.  Returns 1 if the history was dropped. */
int or_anderson_step(long n, int mh, const double *Xs, const double *Fs, double beta, double *x_next)
{
    const double *x = Xs + (long)mh * n, *f = Fs + (long)mh * n;
    double gamma[32] = {0};
    int dropped = 0;
    if (mh > 0) {
        if (mh > 32) return 2;
        double G[32][33];
        double *dFi = malloc(sizeof(double) * n), *dFj = malloc(sizeof(double) * n);
        if (!dFi || !dFj) { free(dFi); free(dFj); return 3; }
        for (int i = 0; i < mh; ++i) {
            for (long t = 0; t < n; ++t) dFi[t] = Fs[(long)(i + 1) * n + t] - Fs[(long)i * n + t];
            G[i][mh] = dot(n, dFi, f);
            for (int j = 0; j <= i; ++j) {
                for (long t = 0; t < n; ++t) dFj[t] = Fs[(long)(j + 1) * n + t] - Fs[(long)j * n + t];
                G[i][j] = G[j][i] = dot(n, dFi, dFj);
            }
        }
        free(dFi); free(dFj);
        double dmax = 0.0;
        for (int i = 0; i < mh; ++i) dmax = fmax(dmax, G[i][i]);
        for (int c = 0; c < mh && !dropped; ++c) {
            int piv = c;
            for (int r = c + 1; r < mh; ++r)
                if (fabs(G[r][c]) > fabs(G[piv][c])) piv = r;
            if (!(fabs(G[piv][c]) > 1e-14 * dmax)) { dropped = 1; break; }
            if (piv != c)
                for (int k = 0; k <= mh; ++k) { double t = G[c][k]; G[c][k] = G[piv][k]; G[piv][k] = t; }
            for (int r = c + 1; r < mh; ++r) {
                const double fct = G[r][c] / G[c][c];
                for (int k = c; k <= mh; ++k) G[r][k] -= fct * G[c][k];
            }
        }
        if (!dropped)
            for (int c = mh - 1; c >= 0; --c) {
                double s = G[c][mh];
                for (int k = c + 1; k < mh; ++k) s -= G[c][k] * gamma[k];
                gamma[c] = s / G[c][c];
            }
        else
            memset(gamma, 0, sizeof(gamma));
    }
    for (long t = 0; t < n; ++t) {
        double v = x[t] + beta * f[t];
        for (int i = 0; i < mh; ++i) {
            const double dX = Xs[(long)(i + 1) * n + t] - Xs[(long)i * n + t];
            const double dF = Fs[(long)(i + 1) * n + t] - Fs[(long)i * n + t];
            v -= (dX + beta * dF) * gamma[i];
        }
        x_next[t] = v;
    }
    return dropped;
}

/* Kerker-type preconditioner of an SCF residual f (a reading: the paper's
 * Periodic Pulay mixing is used with such a preconditioner in its SPARC
 * lineage, but the paper does not state one):
 *   y = (-lap_h + a k0^2) (-lap_h + k0^2)^{-1} f = f - (1 - a) k0^2 u,
 *   (-lap_h + k0^2) u = f,
 * i.e. the Fourier symbol (S + a k0^2)/(S + k0^2) with S >= 0 the symbol of
 * -lap_h: wavelengths long against 2 pi/k0 are scaled by a (0 < a <= 1; the
 * mean by exactly a), short ones pass.  u by conjugate gradients from 0
 * until ||f - A u|| <= tol ||f|| or max_iter iterations.  Returns 0, 1 on
 * bad arguments, 2 if max_iter was reached. */
int or_kerker(int n1, int n2, int n3, double h, int no, double k0, double amin, const double *f, double *y,
              double tol, int max_iter, int *iters)
{
    if (!(k0 > 0.0) || !(amin > 0.0) || !(amin <= 1.0)) return 1;
    const long n = (long)n1 * n2 * n3;
    const double s = k0 * k0;
    double *u = calloc(n, sizeof(double)), *r = malloc(sizeof(double) * n);
    double *p = malloc(sizeof(double) * n), *Ap = malloc(sizeof(double) * n);
    if (!u || !r || !p || !Ap) { free(u); free(r); free(p); free(Ap); return 1; }
    for (long i = 0; i < n; ++i) { r[i] = f[i]; p[i] = f[i]; }
    const double fnorm = sqrt(dot(n, f, f));
    double rr = dot(n, r, r);
    int it = 0, status = 0;
    while (fnorm > 0.0 && sqrt(rr) > tol * fnorm) {
        if (it >= max_iter) { status = 2; break; }
        or_laplacian_periodic(n1, n2, n3, h, no, p, Ap);
        for (long i = 0; i < n; ++i) Ap[i] += s * p[i];
        const double alpha = rr / dot(n, p, Ap);
        for (long i = 0; i < n; ++i) {
            u[i] += alpha * p[i];
            r[i] -= alpha * Ap[i];
        }
        const double rr_new = dot(n, r, r);
        for (long i = 0; i < n; ++i) p[i] = r[i] + (rr_new / rr) * p[i];
        rr = rr_new;
        ++it;
    }
    for (long i = 0; i < n; ++i) y[i] = f[i] - (1.0 - amin) * s * u[i];
    if (iters) *iters = it;
    free(u); free(r); free(p); free(Ap);
    return status;
}
