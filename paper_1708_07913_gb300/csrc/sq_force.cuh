// sq_force.cuh -- the nonlocal component of the atomic forces (Section 3.4,
// Eq. Discrete:NLforce), with the recurrence of Eq. Rec:FD1 run to n_pl:
//
//   f_I^nl = -4 sum_q sum_{p of atom I} gamma_p h^3 chi_p(q) chi_p^T grad_h D_q,
//   D_q = sum_{j=0}^{n_pl} c^j t^j,   t^0 = e_q, t^1 = Hhat t^0,
//   t^{j+1} = 2 Hhat t^j - t^{j-1},  Hhat = (H_q - chi_q)/zeta_q,
//
// where D_q is node q's column of the density matrix inside its region, c^j
// the Chebyshev interpolation coefficients of the Fermi-Dirac function on
// [chi_q - zeta_q, chi_q + zeta_q] (discrete orthogonality at the n_pl + 1
// zeros of T_{n_pl+1}, c^0 halved), and grad_h the central finite-difference
// gradient of Eq. FD:Gradient inside the region (zero outside it).  Only
// nodes inside the support of some projector contribute.
//
// One CTA per node (persistent grid).  The current recurrence vector lives
// in shared memory (or, in the form kept for comparisons, in global scratch
// with the others); t^{j-1}, the local part of H t and D are in per-CTA
// global scratch.  Per node, every region row (y, z) gets
// the list of candidate images whose support crosses it (x-interval and
// box-relative row), and every candidate the list of its row entries in row
// order.  Every step is three block-wide phases:
//   (a) the local part of H (stencil + V) at every region point, and, one
//       thread per row, the partial inner products <chi_c, t> of each of the
//       row's entries;
//   (a2) one thread per candidate: its inner products, the partials of its
//       entries added in row order;
//   (b) the projector update (a point visits its row's entries only), the
//       shift/scale to Hhat, the three-term step and D += c^j t^{j+1}.
// The contribution of each (node, candidate image) pair is added to a
// per-CTA force array in candidate order by one thread, and a second kernel
// adds the CTA arrays in block order: the result repeats bit for bit for a
// given grid.  T is the context's recurrence precision: the three vectors,
// D, the projector inner products and the potential/projector tables are in
// T; the interpolation coefficients and the final contraction (the gradient
// sums and the force) are in FP64.
//
// The code uses block barriers and plain loads/stores only (no warp
// intrinsics), every loop has a fixed trip count, and every table index is
// clipped to the region or the projector box.
#pragma once
#include "sq_internal.cuh"

namespace sq {

constexpr int FORCE_NT = 256;        // threads per CTA of the force kernel
constexpr int FORCE_EPR = 32;        // projector entries a region row may hold

template <typename T>
struct ForceArgs {
    GridParams g;
    T lap[FD_NO + 1];                // lap[0] = -3 w_0 (diagonal), lap[d] = -w_d/2 (d >= 1)
    double grad[FD_NO + 1];          // gradient weights of Eq. FD:Gradient, d = 1..n_o
    const T* Vp;                     // potential with a periodic halo of m points
    NLParams<T> nl;
    const double* chi;
    const double* zeta;
    double mu;
    double kT;
    int npl;
    const long long* nodes;          // nodes to visit (device; validated on the host), or nullptr: all
    long long nq;                    // their number (N_d when nodes is nullptr)
    // per-CTA scratch (slices of the sizes given)
    T* vec;                          // 4 S^3 per CTA: t^{j-1}, t^j, t^{j+1}, D
    int4* cand;                      // ccap per CTA: (atom, box start relative to the region)
    int* clen;                       // ccap per CTA: box lengths len_x | len_y << 8 | len_z << 16
    T* P;                            // 4 ccap per CTA: <chi_s, t>, <chi_px, t>, <chi_py, t>, <chi_pz, t>
    int2* rowent;                    // S^2 FORCE_EPR per CTA: (c | xlo << 10 | xhi << 15, jj | kk << 8)
    int* rown;                       // S^2 per CTA: entries of each row
    int* cent;                       // S^2 FORCE_EPR per CTA: entry indices r FORCE_EPR + e of each candidate
    int* cstart;                     // ccap + 1 per CTA: candidate c owns cent[cstart[c] .. cstart[c+1])
    T* part;                         // 4 S^2 FORCE_EPR per CTA: partial inner products of each entry
    double* Fcta;                    // 3 n_atoms per CTA
    unsigned* err;
};

__device__ inline int fmin_i(int a, int b) { return a < b ? a : b; }
__device__ inline int fmax_i(int a, int b) { return a > b ? a : b; }

// Region row (y, z) of candidate cr: its support x-interval [xlo, xhi] in
// region columns and the box-relative row (jj, kk); false if the row misses
// the box or the support.
template <typename T>
__device__ inline bool force_row(const NLParams<T>& nl, int4 cr, int ln, int S, int y, int z, int& xlo,
                                 int& xhi, int& jj, int& kk)
{
    jj = y - cr.z;
    kk = z - cr.w;
    if (jj < 0 || jj >= ((ln >> 8) & 255) || kk < 0 || kk >= ((ln >> 16) & 255)) return false;
    const uint8_t* iv = nl.ivl + (((size_t)cr.x * nl.lb + jj) * nl.lb + kk) * 2;
    const int lo = iv[0], hi = iv[1];
    if (lo > hi) return false;
    xlo = fmax_i(lo + cr.y, 0);
    xhi = fmin_i(hi + cr.y, fmin_i(cr.y + (ln & 255), S) - 1);
    return xlo <= xhi;
}

// Per-CTA views of the row and candidate entry lists.
template <typename T>
struct ForceLists {
    const int4* cand;
    const int* clen;
    int ncand;
    const int2* rowent;
    const int* rown;
    const int* cent;
    const int* cstart;
    T* part;
    T* P;
};

// One step t' = Hhat x (first) or t' = 2 Hhat x - xm, then D += cj t'.
//   INPLACE = false: x, xm, y in global scratch; y receives t'.
//   INPLACE = true:  x in shared memory and overwritten by t' point by point
//                    in phase (b) (each thread reads and writes only its own
//                    points there); the old x goes to xm, which becomes the
//                    next step's t^{j-1}; y holds the local part only.
// Both forms evaluate the same expressions in the same order.
template <typename T, bool INPLACE>
__device__ inline void force_hhat(const ForceArgs<T>& a, int qi, int qj, int qk, int S, T chq, T zq,
                                  const ForceLists<T>& L, T* x, T* xm, bool first, T* y, T* D, T cj)
{
    const int tid = threadIdx.x;
    const long long S2 = (long long)S * S, S3 = S2 * S;
    const NLParams<T>& nl = a.nl;
    const int lb = nl.lb;
    // (a) local part, and the partial inner products of every row entry
    for (long long p = tid; p < S3; p += FORCE_NT) {
        const int px = (int)(p % S), py = (int)((p / S) % S), pz = (int)(p / S2);
        const T v = a.Vp[(long long)(qi + px) +
                         (long long)a.g.P1 * ((long long)(qj + py) + (long long)a.g.P2 * (qk + pz))];
        T acc = (a.lap[0] + v) * x[p];
        for (int d = 1; d <= FD_NO; ++d) {
            T nb = 0;
            if (px + d < S) nb += x[p + d];
            if (px - d >= 0) nb += x[p - d];
            if (py + d < S) nb += x[p + (long long)d * S];
            if (py - d >= 0) nb += x[p - (long long)d * S];
            if (pz + d < S) nb += x[p + (long long)d * S2];
            if (pz - d >= 0) nb += x[p - (long long)d * S2];
            acc += a.lap[d] * nb;
        }
        y[p] = acc;
    }
    for (int r = tid; r < S * S; r += FORCE_NT) {
        const int n = L.rown[r];
        const T* xr = x + (long long)r * S;
        for (int e = 0; e < n; ++e) {
            const int2 en = L.rowent[r * FORCE_EPR + e];
            const int c = en.x & 1023, xlo = (en.x >> 10) & 31, xhi = (en.x >> 15) & 31;
            const int jj = en.y & 255, kk = (en.y >> 8) & 255;
            const int4 cr = L.cand[c];
            const T* Gt = nl.G + (size_t)cr.x * 3 * lb;
            const T* Dt = nl.DG + (size_t)cr.x * 3 * lb;
            T sg = 0, sd = 0;
            for (int xx = xlo; xx <= xhi; ++xx) {
                const T v = xr[xx];
                sg += Gt[xx - cr.y] * v;
                sd += Dt[xx - cr.y] * v;
            }
            const T gy = Gt[lb + jj], dgy = Dt[lb + jj], gz = Gt[2 * lb + kk], dgz = Dt[2 * lb + kk];
            T* o = L.part + 4 * ((size_t)r * FORCE_EPR + e);
            o[0] = gy * gz * sg;
            o[1] = gy * gz * sd;
            o[2] = dgy * gz * sg;
            o[3] = gy * dgz * sg;
        }
    }
    __syncthreads();
    // (a2) per candidate, its entries' partials in row order
    for (int c = tid; c < L.ncand; c += FORCE_NT) {
        T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
        for (int k = L.cstart[c]; k < L.cstart[c + 1]; ++k) {
            const T* o = L.part + 4 * (size_t)L.cent[k];
            s0 += o[0];
            s1 += o[1];
            s2 += o[2];
            s3 += o[3];
        }
        L.P[4 * c + 0] = s0;
        L.P[4 * c + 1] = s1;
        L.P[4 * c + 2] = s2;
        L.P[4 * c + 3] = s3;
    }
    __syncthreads();
    // (b) projector update from the point's row entries, Hhat, three-term step, D
    const T cs = nl.cs, cp = nl.cp;
    for (long long p = tid; p < S3; p += FORCE_NT) {
        const int px = (int)(p % S);
        const int r = (int)(p / S);
        T acc = y[p];
        const int n = L.rown[r];
        for (int e = 0; e < n; ++e) {
            const int2 en = L.rowent[r * FORCE_EPR + e];
            const int xlo = (en.x >> 10) & 31, xhi = (en.x >> 15) & 31;
            if (px < xlo || px > xhi) continue;
            const int c = en.x & 1023, jj = en.y & 255, kk = (en.y >> 8) & 255;
            const int4 cr = L.cand[c];
            const int ii = px - cr.y;
            const T* Gt = nl.G + (size_t)cr.x * 3 * lb;
            const T* Dt = nl.DG + (size_t)cr.x * 3 * lb;
            const T gx = Gt[ii], dgx = Dt[ii], gy = Gt[lb + jj], dgy = Dt[lb + jj];
            const T gz = Gt[2 * lb + kk], dgz = Dt[2 * lb + kk];
            const T* Pc = L.P + 4 * c;
            acc += cs * Pc[0] * (gx * gy * gz) +
                   cp * (Pc[1] * (dgx * gy * gz) + Pc[2] * (gx * dgy * gz) + Pc[3] * (gx * gy * dgz));
        }
        const T xv = x[p];
        T v = (acc - chq * xv) / zq;
        if (!first) v = (T)2 * v - xm[p];
        if (INPLACE) {
            xm[p] = xv;
            x[p] = v;
        } else {
            y[p] = v;
        }
        D[p] += cj * v;
    }
    __syncthreads();
}

// Dynamic shared memory of the force kernel (the current recurrence vector
// in the in-place form).  A host build of this header supplies the buffer.
#ifdef __CUDACC__
__device__ inline unsigned char* force_dyn_smem()
{
    extern __shared__ __align__(16) unsigned char sq_force_dyn[];
    return sq_force_dyn;
}
#else
unsigned char* force_dyn_smem();
#endif

template <typename T, bool INPLACE>
__global__ void __launch_bounds__(FORCE_NT) nl_force_kernel(ForceArgs<T> a)
{
    __shared__ double s_fk[MAX_NPL + 1];     // Fermi function at the Chebyshev zeros
    __shared__ double s_th[MAX_NPL + 1];     // their angles
    __shared__ double s_c[MAX_NPL + 1];      // interpolation coefficients c^j
    __shared__ double s_f[3 * MAX_CAND];     // force contribution of each candidate
    __shared__ int4 s_rec[FORCE_NT];
    __shared__ int s_len[FORCE_NT];
    __shared__ int s_keep[FORCE_NT];
    __shared__ int s_n;
    __shared__ int s_touch;

    const int tid = threadIdx.x;
    const int M = a.g.m, S = 2 * M + 1;
    const long long S3 = (long long)S * S * S;
    const NLParams<T>& nl = a.nl;
    const int cap = nl.ccap;
    const int npl = a.npl;
    T* tm = a.vec + (size_t)blockIdx.x * 4 * S3;
    T* t = tm + S3;
    T* tn = t + S3;
    T* D = tn + S3;
    int4* cand = a.cand + (size_t)blockIdx.x * cap;
    int* clen = a.clen + (size_t)blockIdx.x * cap;
    T* P = a.P + (size_t)blockIdx.x * 4 * cap;
    const int S2i = S * S;
    int2* rowent = a.rowent + (size_t)blockIdx.x * S2i * FORCE_EPR;
    int* rown = a.rown + (size_t)blockIdx.x * S2i;
    int* cent = a.cent + (size_t)blockIdx.x * S2i * FORCE_EPR;
    int* cstart = a.cstart + (size_t)blockIdx.x * (cap + 1);
    T* part = a.part + (size_t)blockIdx.x * 4 * S2i * FORCE_EPR;
    double* Fc = a.Fcta + (size_t)blockIdx.x * 3 * nl.n_atoms;
    for (int i = tid; i < 3 * nl.n_atoms; i += FORCE_NT) Fc[i] = 0.0;
    const long long ctr = (long long)M + (long long)S * (M + (long long)S * M);

    for (long long iq = blockIdx.x; iq < a.nq; iq += gridDim.x) {
        const long long q = a.nodes ? a.nodes[iq] : iq;
        const int qi = (int)(q % a.g.n1), qj = (int)((q / a.g.n1) % a.g.n2);
        const int qk = (int)(q / ((long long)a.g.n1 * a.g.n2));
        // (1) the node's projector candidates: the boxes of its tile's list
        // that meet its region, in list order
        const int tile = qi / TILE + nl.ntile[0] * (qj / TILE + nl.ntile[1] * (qk / TILE));
        const int beg = nl.tile_start[tile], end = nl.tile_start[tile + 1];
        if (tid == 0) s_n = 0;
        for (int c0 = beg; c0 < end; c0 += FORCE_NT) {
            __syncthreads();
            const int c = c0 + tid;
            int keep = 0;
            if (c < end) {
                const int4 tc = nl.tile_cand[c];
                const AtomTab at = nl.atoms[tc.x];
                const int bx = tc.y - (qi - M), by = tc.z - (qj - M), bz = tc.w - (qk - M);
                keep = bx < S && bx + at.len[0] > 0 && by < S && by + at.len[1] > 0 && bz < S && bz + at.len[2] > 0;
                s_rec[tid] = make_int4(tc.x, bx, by, bz);
                s_len[tid] = at.len[0] | (at.len[1] << 8) | (at.len[2] << 16);
            }
            s_keep[tid] = keep;
            __syncthreads();
            if (tid == 0) {
                int n = s_n;
                const int cnt = fmin_i(FORCE_NT, end - c0);
                for (int i = 0; i < cnt; ++i) {
                    if (!s_keep[i]) continue;
                    if (n < cap) {
                        cand[n] = s_rec[i];
                        clen[n] = s_len[i];
                        ++n;
                    } else {
                        atomicOr(a.err, ERR_CAPACITY);
                    }
                }
                s_n = n;
            }
        }
        __syncthreads();
        const int ncand = s_n;
        // (2) is the node inside some projector's support?
        if (tid == 0) {
            int touch = 0;
            for (int c = 0; c < ncand && !touch; ++c) {
                int xlo, xhi, jj, kk;
                if (force_row(nl, cand[c], clen[c], S, M, M, xlo, xhi, jj, kk) && xlo <= M && M <= xhi) touch = 1;
            }
            s_touch = touch;
        }
        __syncthreads();
        if (!s_touch) continue;
        // (2b) row entries (each row scans the candidates in order), then each
        // candidate's entries in row order (counted, offsets, filled)
        for (int r = tid; r < S2i; r += FORCE_NT) {
            const int y = r % S, z = r / S;
            int n = 0;
            for (int c = 0; c < ncand; ++c) {
                int xlo, xhi, jj, kk;
                if (!force_row(nl, cand[c], clen[c], S, y, z, xlo, xhi, jj, kk)) continue;
                if (n < FORCE_EPR) {
                    rowent[r * FORCE_EPR + n] = make_int2(c | (xlo << 10) | (xhi << 15), jj | (kk << 8));
                    ++n;
                } else {
                    atomicOr(a.err, ERR_CAPACITY);
                }
            }
            rown[r] = n;
        }
        __syncthreads();
        for (int c = tid; c < ncand; c += FORCE_NT) {
            const int4 cr = cand[c];
            const int ln = clen[c];
            const int z0 = fmax_i(cr.w, 0), z1 = fmin_i(cr.w + ((ln >> 16) & 255), S);
            const int y0 = fmax_i(cr.z, 0), y1 = fmin_i(cr.z + ((ln >> 8) & 255), S);
            int cnt = 0;
            for (int z = z0; z < z1; ++z)
                for (int y = y0; y < y1; ++y) {
                    const int r = y + S * z;
                    for (int e = 0; e < rown[r]; ++e) cnt += (rowent[r * FORCE_EPR + e].x & 1023) == c;
                }
            cstart[c + 1] = cnt;
        }
        __syncthreads();
        if (tid == 0) {
            cstart[0] = 0;
            for (int c = 0; c < ncand; ++c) cstart[c + 1] += cstart[c];
        }
        __syncthreads();
        for (int c = tid; c < ncand; c += FORCE_NT) {
            const int4 cr = cand[c];
            const int ln = clen[c];
            const int z0 = fmax_i(cr.w, 0), z1 = fmin_i(cr.w + ((ln >> 16) & 255), S);
            const int y0 = fmax_i(cr.z, 0), y1 = fmin_i(cr.z + ((ln >> 8) & 255), S);
            int k = cstart[c];
            for (int z = z0; z < z1; ++z)
                for (int y = y0; y < y1; ++y) {
                    const int r = y + S * z;
                    for (int e = 0; e < rown[r]; ++e)
                        if ((rowent[r * FORCE_EPR + e].x & 1023) == c) cent[k++] = r * FORCE_EPR + e;
                }
        }
        const ForceLists<T> lists{cand, clen, ncand, rowent, rown, cent, cstart, part, P};
        // (3) c^j = (2/(n_pl+1)) sum_k g(chi + zeta x_k) T_j(x_k), c^0 halved
        const double chq = a.chi[q], zq = a.zeta[q];
        for (int k = tid; k <= npl; k += FORCE_NT) {
            const double xk = cos(M_PI * (k + 0.5) / (npl + 1));
            s_th[k] = acos(xk);
            s_fk[k] = 1.0 / (1.0 + exp((chq + zq * xk - a.mu) / a.kT));
        }
        __syncthreads();
        for (int j = tid; j <= npl; j += FORCE_NT) {
            double acc = 0.0;
            for (int k = 0; k <= npl; ++k) acc += s_fk[k] * cos(j * s_th[k]);
            s_c[j] = (j == 0 ? 1.0 : 2.0) / (npl + 1) * acc;
        }
        __syncthreads();
        // (4) t^0 = e_q, D = c^0 t^0; the recurrence to n_pl accumulating D
        const T chT = (T)chq, zT = (T)zq;
        if (INPLACE) {
            T* xs = reinterpret_cast<T*>(force_dyn_smem());
            for (long long p = tid; p < S3; p += FORCE_NT) {
                xs[p] = p == ctr ? (T)1 : (T)0;
                D[p] = p == ctr ? (T)s_c[0] : (T)0;
            }
            __syncthreads();
            for (int j = 1; j <= npl; ++j)
                force_hhat<T, true>(a, qi, qj, qk, S, chT, zT, lists, xs, tm, j == 1, t, D, (T)s_c[j]);
        } else {
            for (long long p = tid; p < S3; p += FORCE_NT) {
                tm[p] = p == ctr ? (T)1 : (T)0;
                D[p] = p == ctr ? (T)s_c[0] : (T)0;
            }
            __syncthreads();
            force_hhat<T, false>(a, qi, qj, qk, S, chT, zT, lists, tm, nullptr, true, t, D, (T)s_c[1]);
            for (int j = 2; j <= npl; ++j) {
                force_hhat<T, false>(a, qi, qj, qk, S, chT, zT, lists, t, tm, false, tn, D, (T)s_c[j]);
                T* r = tm;
                tm = t;
                t = tn;
                tn = r;
            }
        }
        // (5) per (candidate, axis): -4 sum_comp coef chi'(q) <chi', grad_axis D>
        const long long sa[3] = {1, S, (long long)S * S};
        for (int task = tid; task < 3 * ncand; task += FORCE_NT) {
            const int c = task / 3, ax = task % 3;
            const int4 cr = cand[c];
            const int ln = clen[c];
            double val = 0.0;
            int xlo, xhi, jj, kk;
            if (force_row(nl, cr, ln, S, M, M, xlo, xhi, jj, kk) && xlo <= M && M <= xhi) {
                const T* Gt = nl.G + (size_t)cr.x * 3 * nl.lb;
                const T* Dt = nl.DG + (size_t)cr.x * 3 * nl.lb;
                const int lb = nl.lb;
                const int i0 = M - cr.y;
                const double g0x = Gt[i0], g0y = Gt[lb + jj], g0z = Gt[2 * lb + kk];
                const double s0 = g0x * g0y * g0z;
                const double x0 = (double)Dt[i0] * g0y * g0z;
                const double y0v = g0x * (double)Dt[lb + jj] * g0z;
                const double z0v = g0x * g0y * (double)Dt[2 * lb + kk];
                double ss = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
                const int z0 = fmax_i(cr.w, 0), z1 = fmin_i(cr.w + ((ln >> 16) & 255), S);
                const int y0 = fmax_i(cr.z, 0), y1 = fmin_i(cr.z + ((ln >> 8) & 255), S);
                for (int z = z0; z < z1; ++z)
                    for (int yy = y0; yy < y1; ++yy) {
                        int rlo, rhi, rj, rk;
                        if (!force_row(nl, cr, ln, S, yy, z, rlo, rhi, rj, rk)) continue;
                        const double gy = Gt[lb + rj], dgy = Dt[lb + rj], gz = Gt[2 * lb + rk], dgz = Dt[2 * lb + rk];
                        for (int xx = rlo; xx <= rhi; ++xx) {
                            const int pc[3] = {xx, yy, z};
                            const long long p = (long long)xx + (long long)S * (yy + (long long)S * z);
                            double gd = 0.0;
                            for (int d = 1; d <= FD_NO; ++d) {
                                const double dp = pc[ax] + d < S ? (double)D[p + d * sa[ax]] : 0.0;
                                const double dm = pc[ax] - d >= 0 ? (double)D[p - d * sa[ax]] : 0.0;
                                gd += a.grad[d] * (dp - dm);
                            }
                            const int ii = xx - cr.y;
                            const double gx = Gt[ii], dgx = Dt[ii];
                            ss += gx * gy * gz * gd;
                            sx += dgx * gy * gz * gd;
                            sy += gx * dgy * gz * gd;
                            sz += gx * gy * dgz * gd;
                        }
                    }
                val = -4.0 * ((double)nl.cs * s0 * ss + (double)nl.cp * (x0 * sx + y0v * sy + z0v * sz));
            }
            s_f[task] = val;
        }
        __syncthreads();
        if (tid == 0)
            for (int c = 0; c < ncand; ++c)
                for (int ax = 0; ax < 3; ++ax) Fc[3 * cand[c].x + ax] += s_f[3 * c + ax];
        __syncthreads();
    }
}

// F[i] = sum over CTAs b (in order) of Fcta[b][i].
__global__ void force_sum_kernel(const double* __restrict__ Fcta, int nblk, int n3, double* __restrict__ F)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += Fcta[(size_t)b * n3 + i];
    F[i] = s;
}

}  // namespace sq
