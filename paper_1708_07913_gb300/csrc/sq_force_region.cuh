// sq_force_region.cuh -- the nonlocal atomic forces (Section 3.4, Eq.
// Discrete:NLforce) on the machinery of the region kernels:
//
//   f_I^nl = -4 sum_q sum_{p of atom I} gamma_p h^3 chi_p(q) chi_p^T grad_h D_q,
//   D_q = sum_{j=0}^{n_pl} c^j t^j,   t^0 = e_q, t^1 = Hhat t^0,
//   t^{j+1} = 2 Hhat t^j - t^{j-1},   Hhat = (H_q - chi_q)/zeta_q,
//
// with c^j the Chebyshev interpolation coefficients of the Fermi-Dirac
// function on [chi_q - zeta_q, chi_q + zeta_q] (discrete orthogonality at the
// n_pl + 1 zeros of T_{n_pl+1}, c^0 halved) and grad_h the central
// finite-difference gradient of Eq. FD:Gradient inside the region (zero
// outside it).  Only nodes inside the support of some projector contribute.
//
// One CTA per node, as in moments_node: the same projector set-up, inner
// products, update and stencil sweep (t in shared memory, the compact layout
// at 27^3 and 29^3), run to n_pl instead of n_pl/2, with D += c^{j} t^{j}
// folded into the sweep (D in per-CTA global scratch, touched only by the
// thread that owns the point).  Then one warp per (projector candidate,
// axis) contracts chi_p with the gradient of D over the candidate's support,
// lanes over the points of each support row, FP64 sums reduced in a fixed
// tree; thread 0 adds the node's contributions to a per-CTA force array in
// candidate order, and force_sum_kernel adds the CTA arrays in block order.
// The FP64 result repeats bit for bit; in FP32 the projector update adds
// with shared-memory atomics (as in the moments kernel), so repeated runs
// differ at the rounding level.
#pragma once
#include "sq_region.cuh"

namespace sq {

template <typename T>
struct ForceRegionArgs {
    RegionArgs<T> r;                 // region arguments (chi, zeta, npl; projector tables; scratch)
    double grad[FD_NO + 1];          // gradient weights of Eq. FD:Gradient, d = 1..n_o
    double mu, kT;
    const long long* nodes;          // nodes to visit (device, validated on the host), or nullptr: all
    long long nq;                    // their number
    T* D;                            // per CTA: S^3, x fastest
    double* fpart;                   // per CTA: 3 MAX_CAND, one node's (candidate, axis) contributions
    double* Fcta;                    // per CTA: 3 n_atoms
};

// Dynamic shared memory beyond the region vectors: the Fermi function at the
// Chebyshev zeros and the coefficients (n_pl + 1 each), then the projector
// tables.
__host__ __device__ inline size_t force_coef_bytes(int npl) { return 16 + (size_t)2 * (npl + 1) * sizeof(double); }

template <typename T, int M, bool DB>
__device__ void force_node(const ForceRegionArgs<T>& f, unsigned char* smem_raw, long long node, double* Fc)
{
    using G = Geo<M>;
    static_assert(!G::CY || DB, "compact regions must keep both vectors in shared memory");
    const RegionArgs<T>& a = f.r;
    T* bufA = reinterpret_cast<T*>(smem_raw);
    __shared__ int red_i[33];
    __shared__ int s_touch;
    __shared__ double s_dummy;
    double* s_fk = reinterpret_cast<double*>(smem_raw + align16(region_smem<T, M>()));
    double* s_c = s_fk + (a.npl + 1);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    CtaScratch<T> sc = cta_scratch(a, M);
    if (a.nl.smem) nl_tables_in_smem(sc, s_c + (a.npl + 1), a.nl.smem, a.nl.ccap, G::S, a.nl.lb);
    T* bufB = DB ? bufA + G::ELEMS : sc.buf;
    T* D = f.D + (size_t)blockIdx.x * G::NS;
    double* fpart = f.fpart + (size_t)blockIdx.x * 3 * MAX_CAND;
    const int npl = a.npl;

    const int qi = (int)(node % a.g.n1);
    const int qj = (int)((node / a.g.n1) % a.g.n2);
    const int qk = (int)(node / ((long long)a.g.n1 * a.g.n2));
    const T* vwin = a.Vp + ((size_t)qk * a.g.P2 + qj) * a.g.P1 + qi;

    const int ncand = nl_setup<T, M>(a, sc, qi, qj, qk, red_i);
    __syncthreads();
    // is the node inside some candidate's support?  (the entries of its own row)
    if (warp == 0) {
        const int r0 = M + G::S * M;
        const int n0 = sc.row_n[r0];
        bool in = false;
        for (int e = lane; e < n0; e += 32) {
            const uint32_t meta = sc.rec[(size_t)r0 * ENTRIES_PER_ROW + e].meta;
            in |= (int)((meta >> 10) & 31u) <= M && M <= (int)((meta >> 15) & 31u);
        }
        const unsigned any = __ballot_sync(0xffffffffu, in);
        if (lane == 0) s_touch = any != 0u;
    }
    __syncthreads();
    if (!s_touch) return;

    // c^j = (2/(n_pl+1)) sum_k g(chi + zeta x_k) T_j(x_k), c^0 halved
    const double chq = a.chi[node], zq = a.zeta[node];
    for (int k = tid; k <= npl; k += G::NT) {
        const double xk = cos(M_PI * (k + 0.5) / (npl + 1));
        s_fk[k] = 1.0 / (1.0 + exp((chq + zq * xk - f.mu) / f.kT));
    }
    __syncthreads();
    for (int j = tid; j <= npl; j += G::NT) {
        double acc = 0.0;
        for (int k = 0; k <= npl; ++k) acc += s_fk[k] * cos(j * (M_PI * (k + 0.5) / (npl + 1)));
        s_c[j] = (j == 0 ? 1.0 : 2.0) / (npl + 1) * acc;
    }
    // t^0 = e_q, t^{-1} = 0, D = c^0 t^0
    for (int i = tid; i < G::ELEMS; i += G::NT) bufA[i] = 0;
    if (DB) for (int i = tid; i < G::ELEMS; i += G::NT) bufB[i] = 0;
    else for (int i = tid; i < G::NS; i += G::NT) bufB[i] = 0;
    __syncthreads();
    const int ctr = M + G::S * (M + G::S * M);
    for (int i = tid; i < G::NS; i += G::NT) D[i] = i == ctr ? (T)s_c[0] : T(0);
    if (tid == 0) bufA[G::LEAD + M * G::PLANE + M * G::PX + M] = 1;
    __syncthreads();

    const T dshift = (T)(-3.0 * a.g.w[0] - chq);
    const T s1 = (T)(1.0 / zq), s2 = (T)(2.0 / zq);
    T* cur = bufA;
    T* sec = bufB;
    for (int i = 0; i < npl; ++i) {
        const T s = (i == 0) ? s1 : s2;
        nl_dots<T, M>(a, sc, cur, ncand);
        __syncthreads();
        nl_collect<T, M>(sc, ncand);
        __syncthreads();
        if constexpr (sizeof(T) == 4) nl_update_red<T, M, DB>(a, sc, sec, ncand, s);
        else nl_update<T, M, DB>(a, sc, sec, s);
        __syncthreads();
        const T cd = (T)s_c[i + 1];
        T u0, u1, u2;
        if (G::CY && (warp < FD_NO || warp >= G::S - FD_NO))   // warp-uniform
            stencil_sweep<T, M, true, DB, true, true>(a, cur, sec, vwin, s, dshift, u0, u1, u2, &s_dummy, D, cd);
        else
            stencil_sweep<T, M, true, DB, false, true>(a, cur, sec, vwin, s, dshift, u0, u1, u2, &s_dummy, D, cd);
        __syncthreads();
        if (DB) { T* t = cur; cur = sec; sec = t; }
    }

    // one warp per (candidate, axis): -4 sum_comp coef chi'(q) <chi', grad_axis D>
    const NLParams<T>& nl = a.nl;
    const int lb = nl.lb;
    const int sa[3] = {1, G::S, G::S * G::S};
    for (int task = warp; task < 3 * ncand; task += G::NW) {
        const int c = task / 3, ax = task % 3;
        const int4 cr = sc.cand[c];
        const int ln = sc.clen[c];
        const int lx = ln & 255, ly = (ln >> 8) & 255, lz = (ln >> 16) & 255;
        double val = 0.0;
        const int i0 = M - cr.y, j0 = M - cr.z, k0 = M - cr.w;
        int xlo0 = 0, xhi0 = -1;
        const bool inside = i0 >= 0 && i0 < lx && j0 >= 0 && j0 < ly && k0 >= 0 && k0 < lz &&
                            nl_row_interval<T, M>(nl, cr.x, cr.y, j0, k0, xlo0, xhi0) && xlo0 <= M && M <= xhi0;
        if (inside) {                                 // warp-uniform
            const T* Gt = nl.G + (size_t)cr.x * 3 * lb;
            const T* Dt = nl.DG + (size_t)cr.x * 3 * lb;
            const double g0x = Gt[i0], g0y = Gt[lb + j0], g0z = Gt[2 * lb + k0];
            const double s0 = g0x * g0y * g0z;
            const double x0 = (double)Dt[i0] * g0y * g0z;
            const double y0v = g0x * (double)Dt[lb + j0] * g0z;
            const double z0v = g0x * g0y * (double)Dt[2 * lb + k0];
            double ss = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
            const int zb = max(cr.w, 0), ze = min(cr.w + lz, G::S);
            const int yb = max(cr.z, 0), ye = min(cr.z + ly, G::S);
            for (int z = zb; z < ze; ++z)
                for (int yy = yb; yy < ye; ++yy) {
                    int rlo, rhi;
                    if (!nl_row_interval<T, M>(nl, cr.x, cr.y, yy - cr.z, z - cr.w, rlo, rhi)) continue;
                    const double gy = Gt[lb + yy - cr.z], dgy = Dt[lb + yy - cr.z];
                    const double gz = Gt[2 * lb + z - cr.w], dgz = Dt[2 * lb + z - cr.w];
                    const int xx = rlo + lane;
                    if (xx > rhi) continue;
                    const int pc[3] = {xx, yy, z};
                    const int p = xx + G::S * (yy + G::S * z);
                    double gd = 0.0;
#pragma unroll
                    for (int d = 1; d <= FD_NO; ++d) {
                        const double dp = pc[ax] + d < G::S ? (double)D[p + d * sa[ax]] : 0.0;
                        const double dm = pc[ax] - d >= 0 ? (double)D[p - d * sa[ax]] : 0.0;
                        gd += f.grad[d] * (dp - dm);
                    }
                    const double gx = Gt[xx - cr.y], dgx = Dt[xx - cr.y];
                    ss += gx * gy * gz * gd;
                    sx += dgx * gy * gz * gd;
                    sy += gx * dgy * gz * gd;
                    sz += gx * gy * dgz * gd;
                }
            ss = warp_sum(ss);
            sx = warp_sum(sx);
            sy = warp_sum(sy);
            sz = warp_sum(sz);
            val = -4.0 * ((double)nl.cs * s0 * ss + (double)nl.cp * (x0 * sx + y0v * sy + z0v * sz));
        }
        if (lane == 0) fpart[task] = val;
    }
    __syncthreads();
    if (tid == 0)
        for (int c = 0; c < ncand; ++c)
            for (int ax = 0; ax < 3; ++ax) Fc[3 * sc.cand[c].x + ax] += fpart[3 * c + ax];
    __syncthreads();
}

template <typename T, int M, bool DB>
__global__ void __launch_bounds__(Geo<M>::NT, (region_min_blocks<T, M>()))
force_region_kernel(ForceRegionArgs<T> f)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* Fc = f.Fcta + (size_t)blockIdx.x * 3 * f.r.nl.n_atoms;
    for (int i = threadIdx.x; i < 3 * f.r.nl.n_atoms; i += Geo<M>::NT) Fc[i] = 0.0;
    __syncthreads();
    for (long long iq = blockIdx.x; iq < f.nq; iq += gridDim.x)
        force_node<T, M, DB>(f, smem_raw, f.nodes ? f.nodes[iq] : iq, Fc);
}

}  // namespace sq
