// sq_region.cuh -- per-node region kernels: Lanczos spectral bounds and the
// Chebyshev recurrence with moments (Section 3.2, Eqs. Rec:FD and rhoqj).
//
// One CTA owns one node at a time (persistent grid, nodes strided by
// gridDim.x so that CTAs running together work on neighbouring nodes and
// share potential windows and projector tables in L2).  The current vector
// of the recurrence lives in shared memory in a padded layout with shared
// zero halos: rows of pitch S+6 and planes of S+6 rows, so the 6 zero columns
// after row y serve as the x-halo of row y+1 and the 6 zero rows after plane z
// serve as the y-halo of plane z+1.  Every x/y neighbour of the 37-point
// stencil is then a compile-time offset with no bounds test (zero Dirichlet
// boundary of Section 3.1 for free).  Thread (x, y) owns the column through
// the region and marches in z, keeping the 13 z-values it needs in a register
// queue.  The second vector (t^{i-1} / Lanczos v_old) is touched only
// pointwise by the thread that owns its column: it sits in shared memory next
// to the first when both fit (FP32 regions up to 25^3, FP64 up to 19^3), and
// in per-CTA global scratch otherwise.
#pragma once
#include "sq_internal.cuh"

namespace sq {

template <int M>
struct Geo {
    static constexpr int S = 2 * M + 1;
    static constexpr int PX = S + 6;
    static constexpr int PY = S + 6;
    static constexpr int PLANE = PX * PY;
    static constexpr int LEAD = 6 * PX + 6;
    static constexpr int ELEMS = LEAD + S * PLANE;
    static constexpr int NS = S * S * S;
    static constexpr int NT = ((S * S + 31) / 32) * 32;
    static constexpr int NW = NT / 32;
};

// The second vector of the recurrence (t^{i-1}, later t^{i+1}) or of Lanczos
// (v_old, then w): in shared memory with the same padded layout as the first
// when two vectors fit (DB = true), otherwise unpadded in per-CTA global
// scratch.  Only the thread that owns a column (or a row, in the projector
// pre-pass) touches it, so its layout needs no halo.
template <int M, bool DB>
struct Sec {
    using G = Geo<M>;
    static constexpr int ZS = DB ? G::PLANE : G::S * G::S;
    template <typename T>
    __device__ static T* col(T* base, int x, int y) { return DB ? base + G::LEAD + y * G::PX + x : base + y * G::S + x; }
    template <typename T>
    __device__ static T* row(T* base, int y, int z)
    {
        return DB ? base + G::LEAD + z * G::PLANE + y * G::PX : base + ((size_t)z * G::S + y) * G::S;
    }
};

// Both region vectors in shared memory?  (227 KB per CTA, minus ~8 KB static.)
template <typename T, int M>
constexpr bool fits_double_buffer() { return 2 * (size_t)Geo<M>::ELEMS * sizeof(T) + 8192 <= 232448; }

// Per-CTA scratch carving (identical on host and device).
struct ScratchLayout {
    size_t buf, cand, P, row_start, entries, total;
};
__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
__host__ __device__ inline ScratchLayout scratch_layout(int m, size_t tsize)
{
    int S = 2 * m + 1;
    ScratchLayout L;
    size_t off = 0;
    L.buf = off;       off = align256(off + (size_t)S * S * S * tsize);
    L.cand = off;      off = align256(off + (size_t)MAX_CAND * sizeof(int4));
    L.P = off;         off = align256(off + (size_t)MAX_CAND * 4 * tsize);
    L.row_start = off; off = align256(off + (size_t)(S * S + 1) * sizeof(int));
    L.entries = off;   off = align256(off + (size_t)S * S * ENTRIES_PER_ROW * sizeof(uint32_t));
    L.total = off;
    return L;
}

template <typename T>
struct RegionArgs {
    GridParams g;
    const T* Vp;
    NLParams<T> nl;
    char* scratch;
    size_t scratch_stride;
    unsigned* err;
    // Chebyshev moments
    const double* chi;
    const double* zeta;
    double* moments;
    int npl;
    double mom_tol;
    // Lanczos
    int n_lanczos;
    int nl_cap;
    double* alpha;
    double* beta;
    int* klen;
};

template <typename T>
__device__ inline CtaScratch<T> cta_scratch(const RegionArgs<T>& a, int m)
{
    ScratchLayout L = scratch_layout(m, sizeof(T));
    char* base = a.scratch + (size_t)blockIdx.x * a.scratch_stride;
    CtaScratch<T> s;
    s.buf = reinterpret_cast<T*>(base + L.buf);
    s.cand = reinterpret_cast<int4*>(base + L.cand);
    s.P = reinterpret_cast<T*>(base + L.P);
    s.row_start = reinterpret_cast<int*>(base + L.row_start);
    s.entries = reinterpret_cast<uint32_t*>(base + L.entries);
    return s;
}

__device__ inline double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ inline float warp_sumf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T> __device__ inline T warp_sumT(T v);
template <> __device__ inline float warp_sumT<float>(float v) { return warp_sumf(v); }
template <> __device__ inline double warp_sumT<double>(double v) { return warp_sum(v); }

// Sum of one double over the block; every thread returns the same value
// (fixed summation order: warp tree, then warps in index order).
template <int NW>
__device__ inline double block_sum(double v, double* red)
{
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) t += red[w];
    __syncthreads();
    return t;
}

template <int NW>
__device__ inline void block_sum2(double& a, double& b, double* red)
{
    a = warp_sum(a);
    b = warp_sum(b);
    if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = a; red[32 + (threadIdx.x >> 5)] = b; }
    __syncthreads();
    double ta = 0.0, tb = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) { ta += red[w]; tb += red[32 + w]; }
    __syncthreads();
    a = ta; b = tb;
}

// Exclusive prefix of an int over the block (every thread gets its offset and
// the total).  Uses red_i[0..NW].
template <int NW>
__device__ inline int block_excl_scan(int v, int* red_i, int& total)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int n = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += n;
    }
    if (lane == 31) red_i[w] = incl;
    __syncthreads();
    int off = 0;
    total = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        int c = red_i[k];
        if (k < w) off += c;
        total += c;
    }
    __syncthreads();
    return off + incl - v;
}

// ------------------------------------------------------------------------
// Projector bookkeeping for one node (Section 3.1: V_nl restricted to the
// region).  Candidates: atom images of the node's tile whose box meets the
// region, kept in tile-list order.  Row entries: for every region row (y,z),
// the candidates whose support crosses it with their clipped x-interval, in
// candidate order (so every sum below has a fixed order).
// ------------------------------------------------------------------------
template <typename T, int M>
__device__ int nl_setup(const RegionArgs<T>& a, const CtaScratch<T>& sc, int qi, int qj, int qk,
                        int* red_i)
{
    using G = Geo<M>;
    const NLParams<T>& nl = a.nl;
    const int tid = threadIdx.x;
    int tile = (qi / TILE) + nl.ntile[0] * ((qj / TILE) + nl.ntile[1] * (qk / TILE));
    int beg = nl.tile_start[tile], end = nl.tile_start[tile + 1];
    int ncand = 0;
    for (int c0 = beg; c0 < end; c0 += G::NT) {
        int c = c0 + tid;
        int keep = 0;
        int4 rec = make_int4(0, 0, 0, 0);
        if (c < end) {
            int4 tc = nl.tile_cand[c];
            AtomTab at = nl.atoms[tc.x];
            int bx = tc.y - (qi - M), by = tc.z - (qj - M), bz = tc.w - (qk - M);
            keep = (bx < G::S && bx + at.len[0] > 0 && by < G::S && by + at.len[1] > 0 &&
                    bz < G::S && bz + at.len[2] > 0);
            rec = make_int4(tc.x, bx, by, bz);
        }
        int tot;
        int pos = block_excl_scan<G::NW>(keep, red_i, tot);
        if (keep) {
            if (ncand + pos < MAX_CAND) sc.cand[ncand + pos] = rec;
            else atomicOr(a.err, ERR_CAPACITY);
        }
        ncand += tot;
    }
    if (ncand > MAX_CAND) ncand = MAX_CAND;
    __syncthreads();

    // row entries, two passes (count, scan, fill) for a deterministic order
    const int nrow = G::S * G::S;
    int y = tid % G::S, z = tid / G::S;
    int cnt = 0;
    if (tid < nrow) {
        for (int c = 0; c < ncand; ++c) {
            int4 rec = sc.cand[c];
            AtomTab at = nl.atoms[rec.x];
            int jj = y - rec.z, kk = z - rec.w;
            if (jj < 0 || jj >= at.len[1] || kk < 0 || kk >= at.len[2]) continue;
            const uint8_t* iv = nl.ivl + (((size_t)rec.x * NL_BOX + jj) * NL_BOX + kk) * 2;
            int xlo = iv[0], xhi = iv[1];
            if (xlo > xhi) continue;
            xlo = max(xlo + rec.y, 0);
            xhi = min(xhi + rec.y, G::S - 1);
            if (xlo <= xhi) ++cnt;
        }
    }
    int total;
    int off = block_excl_scan<G::NW>(cnt, red_i, total);
    const int cap = nrow * ENTRIES_PER_ROW;
    if (total > cap && tid == 0) atomicOr(a.err, ERR_CAPACITY);
    if (tid < nrow) {
        sc.row_start[tid] = min(off, cap);
        if (tid == nrow - 1) sc.row_start[nrow] = min(off + cnt, cap);
        int e = off;
        for (int c = 0; c < ncand && e < cap; ++c) {
            int4 rec = sc.cand[c];
            AtomTab at = nl.atoms[rec.x];
            int jj = y - rec.z, kk = z - rec.w;
            if (jj < 0 || jj >= at.len[1] || kk < 0 || kk >= at.len[2]) continue;
            const uint8_t* iv = nl.ivl + (((size_t)rec.x * NL_BOX + jj) * NL_BOX + kk) * 2;
            int xlo = iv[0], xhi = iv[1];
            if (xlo > xhi) continue;
            xlo = max(xlo + rec.y, 0);
            xhi = min(xhi + rec.y, G::S - 1);
            if (xlo <= xhi) {
                sc.entries[e] = (uint32_t)c | ((uint32_t)xlo << 16) | ((uint32_t)xhi << 24);
                ++e;
            }
        }
    }
    __syncthreads();
    return ncand;
}

// Projector inner products of the shared-memory vector (trapezoidal rule,
// Eq. IntApprox, without the h^3 which sits in cs/cp):
//   S_c = sum G t, X_c = sum D_x G t, Y_c = sum D_y G t, Z_c = sum D_z G t
// over the support of candidate c inside the region.  The Gaussian factorises
// per axis, so each region row is reduced along x first.  One warp per
// candidate, lanes over rows, warp tree at the end: fixed order.
template <typename T, int M>
__device__ void nl_dots(const RegionArgs<T>& a, const CtaScratch<T>& sc, const T* sm, int ncand)
{
    using G = Geo<M>;
    const NLParams<T>& nl = a.nl;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = warp; c < ncand; c += G::NW) {
        int4 rec = sc.cand[c];
        AtomTab at = nl.atoms[rec.x];
        const T* Gt = nl.G + (size_t)rec.x * 3 * NL_BOX;
        const T* Dt = nl.DG + (size_t)rec.x * 3 * NL_BOX;
        int j0 = max(0, -rec.z), j1 = min(at.len[1], G::S - rec.z);
        int k0 = max(0, -rec.w), k1 = min(at.len[2], G::S - rec.w);
        int nj = j1 - j0;
        int nrows = (nj > 0 && k1 > k0) ? nj * (k1 - k0) : 0;
        T aS = 0, aX = 0, aY = 0, aZ = 0;
        for (int r = lane; r < nrows; r += 32) {
            int jj = j0 + r % nj, kk = k0 + r / nj;
            const uint8_t* iv = nl.ivl + (((size_t)rec.x * NL_BOX + jj) * NL_BOX + kk) * 2;
            int xlo = iv[0], xhi = iv[1];
            if (xlo > xhi) continue;
            xlo = max(xlo + rec.y, 0);
            xhi = min(xhi + rec.y, G::S - 1);
            if (xlo > xhi) continue;
            int y = rec.z + jj, z = rec.w + kk;
            const T* row = sm + G::LEAD + z * G::PLANE + y * G::PX;
            const T* gx = Gt - rec.y;
            const T* dx = Dt - rec.y;
            T u = 0, u2 = 0;
            for (int x = xlo; x <= xhi; ++x) {
                T tv = row[x];
                u += gx[x] * tv;
                u2 += dx[x] * tv;
            }
            T gy = Gt[NL_BOX + jj], dgy = Dt[NL_BOX + jj];
            T gz = Gt[2 * NL_BOX + kk], dgz = Dt[2 * NL_BOX + kk];
            T gyz = gy * gz;
            aS += gyz * u;
            aX += gyz * u2;
            aY += dgy * gz * u;
            aZ += gy * dgz * u;
        }
        aS = warp_sumT<T>(aS);
        aX = warp_sumT<T>(aX);
        aY = warp_sumT<T>(aY);
        aZ = warp_sumT<T>(aZ);
        if (lane == 0) {
            sc.P[4 * c + 0] = aS;
            sc.P[4 * c + 1] = aX;
            sc.P[4 * c + 2] = aY;
            sc.P[4 * c + 3] = aZ;
        }
    }
}

// buf <- a * buf - coef * V_nl t   (one thread per region row, fixed order)
//   V_nl t (x) = sum_c h^3 G(x) [gamma_s A_s^2 S_c + gamma_p A_p^2 (D_x X_c + D_y Y_c + D_z Z_c)]
template <typename T, int M, bool DB>
__device__ void nl_prepass(const RegionArgs<T>& a, const CtaScratch<T>& sc, T* sec, T scale_old, bool zero_old,
                           T coef)
{
    using G = Geo<M>;
    const NLParams<T>& nl = a.nl;
    const int tid = threadIdx.x;
    if (tid >= G::S * G::S) return;
    int y = tid % G::S, z = tid / G::S;
    T* brow = Sec<M, DB>::row(sec, y, z);
    if (zero_old) {
        for (int x = 0; x < G::S; ++x) brow[x] = 0;
    } else if (scale_old != T(1)) {
        for (int x = 0; x < G::S; ++x) brow[x] *= scale_old;
    }
    int e0 = sc.row_start[tid], e1 = sc.row_start[tid + 1];
    const T cs = nl.cs * coef, cp = nl.cp * coef;
    for (int e = e0; e < e1; ++e) {
        uint32_t ent = sc.entries[e];
        int c = ent & 0xffff, xlo = (ent >> 16) & 0xff, xhi = ent >> 24;
        int4 rec = sc.cand[c];
        const T* Gt = nl.G + (size_t)rec.x * 3 * NL_BOX;
        const T* Dt = nl.DG + (size_t)rec.x * 3 * NL_BOX;
        int jj = y - rec.z, kk = z - rec.w;
        T gy = Gt[NL_BOX + jj], dgy = Dt[NL_BOX + jj];
        T gz = Gt[2 * NL_BOX + kk], dgz = Dt[2 * NL_BOX + kk];
        T pS = sc.P[4 * c + 0], pX = sc.P[4 * c + 1], pY = sc.P[4 * c + 2], pZ = sc.P[4 * c + 3];
        T gyz = gy * gz;
        T b0 = cs * gyz * pS + cp * (dgy * gz * pY + gy * dgz * pZ);
        T b1 = cp * gyz * pX;
        const T* gx = Gt - rec.y;
        const T* dx = Dt - rec.y;
        for (int x = xlo; x <= xhi; ++x) brow[x] -= gx[x] * b0 + dx[x] * b1;
    }
}

// Column-wise FP32/FP64 accumulation type for dot products: each thread sums
// its own column in T, the block then sums columns in FP64.
template <typename T>
struct ColAcc { T v; };

// ------------------------------------------------------------------------
// Stencil sweep of H (local part, Eq. FD:Laplacian + V):
//   out(p) = s * [ (-3 w_0 + V(p) - shift) t(p) - 1/2 sum_d w_d (6 nbrs at d) ] - sec(p)
// RECUR = true (Chebyshev step): out = t^{i+1} and sec holds t^{i-1}.
//   DB:  out replaces t^{i-1} in sec (pointwise, no barrier); the caller
//        swaps the two buffers after the sweep.
//   !DB: out replaces t^i in shared memory plane by plane (one barrier per
//        plane keeps the neighbours of the next plane intact) and t^i goes
//        to sec, which becomes t^{i-1}.
//   The thread accumulates out.out and out.t^i over its column.
// RECUR = false (Lanczos): out = w goes to sec; t is left in place; the
//   thread accumulates out.t.
// ------------------------------------------------------------------------
template <typename T, int M, bool RECUR, bool DB>
__device__ void stencil_sweep(const RegionArgs<T>& a, T* cur, T* sec, const T* vwin, T s, T dshift,
                              const T (&wd)[FD_NO + 1], T& acc_a, T& acc_b, T* centre_out)
{
    using G = Geo<M>;
    using SV = Sec<M, DB>;
    const int tid = threadIdx.x;
    const bool active = tid < G::S * G::S;
    const int x = tid % G::S, y = tid / G::S;
    T* col = cur + G::LEAD + y * G::PX + x;
    T* bcol = SV::col(sec, x, y);
    const size_t vplane = (size_t)a.g.P1 * a.g.P2;
    const T* vcol = vwin + (size_t)y * a.g.P1 + x;
    T q[13];
#pragma unroll
    for (int d = 0; d < 6; ++d) q[d] = 0;
#pragma unroll
    for (int d = 0; d < 7; ++d) q[6 + d] = (active && d < G::S) ? col[d * G::PLANE] : T(0);
    T aa = 0, ab = 0;
#pragma unroll
    for (int z = 0; z < G::S; ++z) {
        T out = 0;
        const T c = q[6];
        if (active) {
            const T* p = col + z * G::PLANE;
            T lap = 0;
#pragma unroll
            for (int d = 1; d <= FD_NO; ++d) {
                T nb = (p[d] + p[-d]) + (p[d * G::PX] + p[-d * G::PX]) + (q[6 + d] + q[6 - d]);
                lap += wd[d] * nb;
            }
            T vz = vcol[z * vplane];
            T hv = (vz + dshift) * c + lap;
            out = s * hv - bcol[z * SV::ZS];
        }
        if (RECUR && !DB) __syncthreads();
        if (active) {
            if (RECUR) {
                if (!DB) col[z * G::PLANE] = out;
                bcol[z * SV::ZS] = DB ? out : c;
                aa += out * out;
                ab += out * c;
                if (x == M && y == M && z == M) *centre_out = out;
            } else {
                bcol[z * SV::ZS] = out;
                ab += out * c;
            }
        }
#pragma unroll
        for (int d = 0; d < 12; ++d) q[d] = q[d + 1];
        q[12] = (active && z + 7 < G::S) ? col[(z + 7) * G::PLANE] : T(0);
    }
    acc_a = aa;
    acc_b = ab;
}

template <typename T>
__device__ inline void load_weights(const GridParams& g, T (&wd)[FD_NO + 1])
{
#pragma unroll
    for (int d = 0; d <= FD_NO; ++d) wd[d] = (T)(-0.5 * g.w[d]);
}

// ------------------------------------------------------------------------
// Chebyshev moments kernel (Section 3.2, Eqs. Rec:FD and rhoqj).
// ------------------------------------------------------------------------
template <typename T, int M, bool DB>
__global__ void __launch_bounds__(Geo<M>::NT)
moments_kernel(RegionArgs<T> a)
{
    using G = Geo<M>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* bufA = reinterpret_cast<T*>(smem_raw);
    __shared__ double red[64];
    __shared__ int red_i[33];
    __shared__ double s_mom[MAX_NPL / 2 + 2];
    __shared__ double s_d2[MAX_NPL / 2 + 2];
    __shared__ double s_d1[MAX_NPL / 2 + 2];
    __shared__ T s_centre;

    const int tid = threadIdx.x;
    const CtaScratch<T> sc = cta_scratch(a, M);
    T* bufB = DB ? bufA + G::ELEMS : sc.buf;
    T wd[FD_NO + 1];
    load_weights(a.g, wd);
    const int half = a.npl / 2;
    const bool has_nl = a.nl.n_atoms > 0;

    for (long long node = blockIdx.x; node < a.g.Nd; node += gridDim.x) {
        const int qi = (int)(node % a.g.n1);
        const int qj = (int)((node / a.g.n1) % a.g.n2);
        const int qk = (int)(node / ((long long)a.g.n1 * a.g.n2));
        const double chi = a.chi[node], zeta = a.zeta[node];
        const T dshift = (T)(-3.0 * a.g.w[0] - chi);
        const T s1 = (T)(1.0 / zeta), s2 = (T)(2.0 / zeta);
        const T* vwin = a.Vp + ((size_t)qk * a.g.P2 + qj) * a.g.P1 + qi;

        // t^0 = e_q (Eq. Rec:FD), t^{-1} = 0
        for (int i = tid; i < G::ELEMS; i += G::NT) bufA[i] = 0;
        if (DB) for (int i = tid; i < G::ELEMS; i += G::NT) bufB[i] = 0;
        else for (int i = tid; i < G::NS; i += G::NT) bufB[i] = 0;
        __syncthreads();
        if (tid == 0) {
            bufA[G::LEAD + M * G::PLANE + M * G::PX + M] = 1;
            s_mom[0] = 1.0;
        }
        int ncand = 0;
        if (has_nl) ncand = nl_setup<T, M>(a, sc, qi, qj, qk, red_i);
        __syncthreads();

        T* cur = bufA;
        T* sec = bufB;
        for (int i = 0; i < half; ++i) {
            const T s = (i == 0) ? s1 : s2;
            if (has_nl) {
                nl_dots<T, M>(a, sc, cur, ncand);
                __syncthreads();
                nl_prepass<T, M, DB>(a, sc, sec, T(1), i == 0, s);
                __syncthreads();
            }
            T aa, ab;
            stencil_sweep<T, M, true, DB>(a, cur, sec, vwin, s, dshift, wd, aa, ab, &s_centre);
            double d2 = (double)aa, d1 = (double)ab;
            block_sum2<G::NW>(d2, d1, red);        // includes the barrier that publishes the sweep
            if (tid == 0) {
                s_mom[i + 1] = (double)s_centre;
                s_d2[i + 1] = d2;                  // t^{i+1} . t^{i+1}
                s_d1[i + 1] = d1;                  // t^{i+1} . t^i
            }
            if (DB) { T* t = cur; cur = sec; sec = t; }
        }
        __syncthreads();
        double* out = a.moments + node * (long long)(a.npl + 1);
        for (int j = tid; j <= a.npl; j += G::NT) {
            double r;
            if (j <= half) r = s_mom[j];
            else if ((j & 1) == 0) r = 2.0 * s_d2[j / 2] - s_mom[0];        // rho^{2a} = 2 t^a.t^a - rho^0
            else r = 2.0 * s_d1[(j + 1) / 2] - s_mom[1];                     // rho^{2a+1} = 2 t^{a+1}.t^a - rho^1
            out[j] = r;
            if (!(fabs(r) <= 1.0 + a.mom_tol)) atomicOr(a.err, ERR_BOUNDS);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------
// Lanczos kernel (Section 3.2: extreme eigenvalues of H_q).  Start vector
// uniform 1/sqrt(Ns) on the region, n_lanczos steps without
// re-orthogonalisation, stop early on breakdown beta <= 1e-10 * scale.
// Writes alpha[0..k-1], beta[0..k-2] and k per node; the tridiagonal's
// extremes are found by tridiag_bounds_kernel.
// ------------------------------------------------------------------------
template <typename T, int M, bool DB>
__global__ void __launch_bounds__(Geo<M>::NT)
lanczos_kernel(RegionArgs<T> a)
{
    using G = Geo<M>;
    using SV = Sec<M, DB>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    __shared__ double red[64];
    __shared__ int red_i[33];
    __shared__ T s_dummy;

    const int tid = threadIdx.x;
    const bool active = tid < G::S * G::S;
    const int x = tid % G::S, y = tid / G::S;
    const CtaScratch<T> sc = cta_scratch(a, M);
    T* sec = DB ? sm + G::ELEMS : sc.buf;
    T wd[FD_NO + 1];
    load_weights(a.g, wd);
    const bool has_nl = a.nl.n_atoms > 0;
    const T dshift = (T)(-3.0 * a.g.w[0]);
    const T v0 = (T)(1.0 / sqrt((double)G::NS));

    for (long long node = blockIdx.x; node < a.g.Nd; node += gridDim.x) {
        const int qi = (int)(node % a.g.n1);
        const int qj = (int)((node / a.g.n1) % a.g.n2);
        const int qk = (int)(node / ((long long)a.g.n1 * a.g.n2));
        const T* vwin = a.Vp + ((size_t)qk * a.g.P2 + qj) * a.g.P1 + qi;
        for (int i = tid; i < G::ELEMS; i += G::NT) sm[i] = 0;
        if (DB) for (int i = tid; i < G::ELEMS; i += G::NT) sec[i] = 0;
        else for (int i = tid; i < G::NS; i += G::NT) sec[i] = 0;
        __syncthreads();
        T* col = sm + G::LEAD + y * G::PX + x;
        T* bcol = SV::col(sec, x, y);
        if (active)
            for (int z = 0; z < G::S; ++z) col[z * G::PLANE] = v0;
        int ncand = 0;
        if (has_nl) ncand = nl_setup<T, M>(a, sc, qi, qj, qk, red_i);
        __syncthreads();

        double* alpha = a.alpha + node * (long long)a.nl_cap;
        double* beta = a.beta + node * (long long)a.nl_cap;
        double bprev = 0.0, scale = 0.0;
        int k = 0;
        for (int it = 0; it < a.n_lanczos; ++it) {
            // w = H v - beta_prev v_old  (v_old and then w live in sec)
            if (has_nl) {
                nl_dots<T, M>(a, sc, sm, ncand);
                __syncthreads();
                nl_prepass<T, M, DB>(a, sc, sec, (T)bprev, false, T(1));
                __syncthreads();
            } else if (it > 0) {
                if (active)
                    for (int z = 0; z < G::S; ++z) bcol[z * SV::ZS] *= (T)bprev;
            }
            T aa, ab;
            stencil_sweep<T, M, false, DB>(a, sm, sec, vwin, T(1), dshift, wd, aa, ab, &s_dummy);
            double al = block_sum<G::NW>((double)ab, red);
            // w -= alpha v ; beta = |w|
            T acc = 0;
            const T alT = (T)al;
            if (active)
                for (int z = 0; z < G::S; ++z) {
                    T w = bcol[z * SV::ZS] - alT * col[z * G::PLANE];
                    bcol[z * SV::ZS] = w;
                    acc += w * w;
                }
            double b2 = block_sum<G::NW>((double)acc, red);
            double b = sqrt(b2);
            if (tid == 0) alpha[it] = al;
            k = it + 1;
            if (it == a.n_lanczos - 1) break;
            if (fabs(al) + bprev > scale) scale = fabs(al) + bprev;
            if (b <= 1e-10 * scale) break;
            if (tid == 0) beta[it] = b;
            // v_old <- v, v <- w / beta
            const T inv = (T)(1.0 / b);
            if (active)
                for (int z = 0; z < G::S; ++z) {
                    T w = bcol[z * SV::ZS];
                    T v = col[z * G::PLANE];
                    bcol[z * SV::ZS] = v;
                    col[z * G::PLANE] = w * inv;
                }
            bprev = b;
            __syncthreads();
        }
        if (tid == 0) a.klen[node] = k;
        __syncthreads();
    }
}

template <typename T, int M>
size_t region_smem()
{
    return (fits_double_buffer<T, M>() ? 2 : 1) * (size_t)Geo<M>::ELEMS * sizeof(T);
}

}  // namespace sq
