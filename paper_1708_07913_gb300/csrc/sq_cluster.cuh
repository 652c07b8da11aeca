// sq_cluster.cuh -- FP32 region kernels on thread-block clusters: the
// Chebyshev recurrence with moments (Section 3.2, Eqs. Rec:FD and rhoqj) and
// the Lanczos spectral bounds (Section 3.2, text after Eq. rhoqj).
//
// One cluster of NC CTAs owns one node at a time (persistent grid, nodes
// strided by the number of clusters).  The node's region is cut into NC slabs
// of planes z; CTA k of the cluster holds planes [z0(k), z0(k+1)) of both
// recurrence vectors in its own shared memory, so both vectors of a 29^3
// region stay on chip (two padded copies of a whole 29^3 region would not fit
// one CTA).  The layout of a slab is the padded layout of the single-CTA
// kernels (rows of pitch S+6, planes of S+6 rows, shared zero halos), so the x
// and y neighbours of the 37-point stencil are compile-time offsets; the z
// neighbours come from a 13-deep register queue, filled from the CTA's own
// planes and, across a slab boundary, from the partner CTA's planes through
// distributed shared memory (ld.shared::cluster).
//
// The nonlocal term (Eq. Hamiltonian, V_nl restricted to the region, Section
// 3.1) is split in two passes per step:
//   * inner products P_c = <chi_c, t> of every projector candidate c: the
//     entries (candidate, region row) of the CTA's own rows are cut into
//     chunks of 32 (one entry per lane, all lanes of a chunk the same
//     candidate), each entry reduces its row along x with the candidate's
//     separable Gaussian profile, and the CTA's partial sums go to shared
//     memory; the partial sums of the NC CTAs are then added in rank order
//     after one cluster barrier, so every CTA holds the same P;
//   * the update V_nl t is folded into the stencil sweep that produces the
//     next vector: the warp of row (y, z) walks that row's entries and each
//     lane adds G_x b0 + DG_x b1 of the entries whose x-interval holds it,
//     with b0 = cs f0 S_c + cp (f1 Y_c + f2 Z_c), b1 = cp f0 X_c computed
//     once per entry and step.  Every point therefore sums its projector
//     terms in one fixed order (no atomics).
//
// Per Chebyshev step: sweep (stencil + projector update, writing t^{i+1}
// over t^{i-1}) -> CTA barrier -> inner products of t^{i+1} -> cluster
// barrier -> partial sums combined, per-entry b0/b1 -> CTA barrier.  The
// dot products t^i.t^i and t^i.t^{i-1} of the product rule are accumulated
// during sweep i (which reads both vectors anyway).
//
// Per Lanczos step (w = H v - beta v_old, alpha = v.w, beta = |w - alpha v|):
// the sweep writes w over beta v_old and accumulates v.w, w.w and v.v, from
// which beta^2 = w.w - 2 alpha v.w + alpha^2 v.v after a cluster barrier; a
// pointwise pass forms v' = (w - alpha v)/beta and beta v, and the inner
// products of v' are taken from v' itself (recombining them from those of w
// and v would amplify their rounding by |alpha/beta| every step) before a
// second cluster barrier.
#pragma once
#include "sq_region.cuh"

namespace sq {

constexpr int CL_ECAP = 16;          // projector entries a region row may hold (FCC Al at h ~ 0.48: up to 16)
constexpr int CL_ESTR = 17;          // slot stride per row (odd, so rows fall in different banks)

template <int M, int NC>
struct CGeo {
    static constexpr int S = 2 * M + 1;
    static constexpr int PX = S + 6;
    static constexpr int PY = S + 6;
    static constexpr int PLANE = PX * PY;
    static constexpr int LEAD = 6 * PX + 6;
    static constexpr int NZMAX = (S + NC - 1) / NC;      // planes of the largest slab
    static constexpr int ELEMS = LEAD + NZMAX * PLANE;   // floats per vector slab
    static constexpr int ROWS = S * NZMAX;               // region rows of the largest slab
    static constexpr int NT = 32 * S;                    // warp y owns row y of every own plane, lane = x
    static constexpr int NW = S;
    static constexpr int BITW = (ROWS + 31) / 32;        // words of a per-candidate row bitmap
    __host__ __device__ static constexpr int z0(int k) { return (k * S) / NC; }
    __host__ __device__ static constexpr int owner(int z) { return ((z + 1) * NC - 1) / S; }
};

// Shared-memory carving of one CTA (byte offsets; identical on host and device).
struct ClLayout {
    size_t bufA, bufB, rec, rec2, row_n, cidx, bits, cand, clen, TX, Ploc, Pc, cstart, chunk, mom, part, total;
};
__host__ __device__ inline ClLayout cl_layout(int S, int nzmax, int ccap, int npl)
{
    const size_t px = S + 6, plane = px * px, lead = 6 * px + 6;
    const size_t elems = lead + (size_t)nzmax * plane;
    const size_t rows = (size_t)S * nzmax;
    ClLayout L;
    size_t o = 0;
    L.bufA = o;   o = align16(o + elems * 4);
    L.bufB = o;   o = align16(o + elems * 4);
    L.rec = o;    o = align16(o + rows * CL_ESTR * 16);
    L.rec2 = o;   o = align16(o + rows * CL_ESTR * 8);
    L.row_n = o;  o = align16(o + rows);
    L.cidx = o;   o = align16(o + rows * CL_ECAP * 2);
    L.bits = o;   o = align16(o + (size_t)ccap * ((rows + 31) / 32) * 4);
    L.cand = o;   o = align16(o + (size_t)ccap * 16);
    L.clen = o;   o = align16(o + (size_t)ccap * 4);
    L.TX = o;     o = align16(o + (size_t)ccap * S * 8);
    L.Ploc = o;   o = align16(o + (size_t)2 * ccap * 16);
    L.Pc = o;     o = align16(o + (size_t)ccap * 16);
    L.cstart = o; o = align16(o + (size_t)(ccap + 1) * 4);
    L.chunk = o;  o = align16(o + (size_t)(ccap + 1) * 4);
    L.mom = o;    o = align16(o + (size_t)3 * (npl / 2 + 2) * 8);
    L.part = o;   o = align16(o + (size_t)2 * 4 * 8);
    L.total = o;
    return L;
}

// ---- cluster primitives (PTX) ----------------------------------------------
__device__ __forceinline__ unsigned cl_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Every thread of every CTA of the cluster arrives; writes to shared memory
// (own or a partner's) before the barrier are visible to reads after it.
__device__ __forceinline__ void cl_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ unsigned cl_map(const void* p, unsigned rank)
{
    unsigned a = (unsigned)__cvta_generic_to_shared(p), r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ float cl_ld_f32(unsigned addr)
{
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ float4 cl_ld_v4(unsigned addr)
{
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}
__device__ __forceinline__ double cl_ld_f64(unsigned addr)
{
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr));
    return v;
}

// Pointers into one CTA's shared memory.
struct ClSmem {
    float* A;            // current vector slab (t^i / Lanczos v)
    float* B;            // second vector slab (t^{i-1} / beta v_old, then the sweep's output)
    float4* rec;         // [row][CL_ESTR]: (meta bits, f0, b0, b1)
    float2* rec2;        // [row][CL_ESTR]: (f1, f2)
    uint8_t* row_n;      // entries of each own row
    uint16_t* cidx;      // own entries in candidate order (slot indices)
    unsigned* bits;      // [cand][BITW]: own rows holding an entry of the candidate
    int4* cand;          // (atom, bx, by, bz): box start relative to the region
    int* clen;           // len_x | len_y << 8 | len_z << 16
    float2* TX;          // [cand][S]: (G_x, DG_x) at region column x (0 outside the box)
    float4* Ploc;        // [2][cand]: this CTA's partial inner products (S, X, Y, Z), by step parity
    float4* Pc;          // combined inner products of the vector the next sweep applies V_nl to
    int* cstart;         // [cand+1]: first own entry of each candidate in cidx
    int* chunk;          // [cand+1]: first 32-entry chunk of each candidate
    double* mom;         // centre values rho^i, t^i.t^i, t^i.t^{i-1} (npl/2 + 2 each)
    double* part;        // [2][4]: Lanczos partial sums (v.w, w.w, v.v) by step parity
};

__device__ inline ClSmem cl_smem(unsigned char* base, int S, int nzmax, int ccap, int npl)
{
    const ClLayout L = cl_layout(S, nzmax, ccap, npl);
    ClSmem s;
    s.A = reinterpret_cast<float*>(base + L.bufA);
    s.B = reinterpret_cast<float*>(base + L.bufB);
    s.rec = reinterpret_cast<float4*>(base + L.rec);
    s.rec2 = reinterpret_cast<float2*>(base + L.rec2);
    s.row_n = reinterpret_cast<uint8_t*>(base + L.row_n);
    s.cidx = reinterpret_cast<uint16_t*>(base + L.cidx);
    s.bits = reinterpret_cast<unsigned*>(base + L.bits);
    s.cand = reinterpret_cast<int4*>(base + L.cand);
    s.clen = reinterpret_cast<int*>(base + L.clen);
    s.TX = reinterpret_cast<float2*>(base + L.TX);
    s.Ploc = reinterpret_cast<float4*>(base + L.Ploc);
    s.Pc = reinterpret_cast<float4*>(base + L.Pc);
    s.cstart = reinterpret_cast<int*>(base + L.cstart);
    s.chunk = reinterpret_cast<int*>(base + L.chunk);
    s.mom = reinterpret_cast<double*>(base + L.mom);
    s.part = reinterpret_cast<double*>(base + L.part);
    return s;
}

// ------------------------------------------------------------------------
// Projector bookkeeping of one node for this CTA's rows (Section 3.1: V_nl
// restricted to the region).  Candidates: the atom images of the node's
// tile whose box meets the region, in tile-list order (the same list in
// every CTA of the cluster).  Entries: (candidate, own region row) pairs
// whose clipped support interval in x is non-empty, with the row's y/z
// Gaussian factors f0 = G_y G_z, f1 = DG_y G_z, f2 = G_y DG_z; stored by row
// (candidates ascending) and indexed by candidate (rows ascending).
// Returns the candidate count.
// ------------------------------------------------------------------------
template <int M, int NC>
__device__ int cl_setup(const RegionArgs<float>& a, const ClSmem& sm, int qi, int qj, int qk, int Z0, int NZ,
                        int* red_i)
{
    using G = CGeo<M, NC>;
    const NLParams<float>& nl = a.nl;
    const int tid = threadIdx.x;
    const int lb = nl.lb;
    const int lim = nl.ccap;
    int tile = (qi / TILE) + nl.ntile[0] * ((qj / TILE) + nl.ntile[1] * (qk / TILE));
    int beg = nl.tile_start[tile], end = nl.tile_start[tile + 1];
    // (1) candidates: ordered compaction of the tile list
    int ncand = 0;
    for (int c0 = beg; c0 < end; c0 += G::NT) {
        const int c = c0 + tid;
        int keep = 0, ln = 0;
        int4 rc = make_int4(0, 0, 0, 0);
        if (c < end) {
            const int4 tc = nl.tile_cand[c];
            const AtomTab at = nl.atoms[tc.x];
            const int bx = tc.y - (qi - M), by = tc.z - (qj - M), bz = tc.w - (qk - M);
            keep = (bx < G::S && bx + at.len[0] > 0 && by < G::S && by + at.len[1] > 0 && bz < G::S &&
                    bz + at.len[2] > 0);
            rc = make_int4(tc.x, bx, by, bz);
            ln = at.len[0] | (at.len[1] << 8) | (at.len[2] << 16);
        }
        int tot;
        const int pos = block_excl_scan<G::NW>(keep, red_i, tot);
        if (keep) {
            if (ncand + pos < lim) {
                sm.cand[ncand + pos] = rc;
                sm.clen[ncand + pos] = ln;
            } else {
                atomicOr(a.err, ERR_CAPACITY);
            }
        }
        ncand += tot;
    }
    if (ncand > lim) ncand = lim;
    const int rows = NZ * G::S;
    for (int i = tid; i < ncand * G::BITW; i += G::NT) sm.bits[i] = 0u;
    for (int c = tid; c <= ncand; c += G::NT) sm.cstart[c] = 0;
    __syncthreads();
    // (2) x-profiles of the candidates in region columns
    for (int i = tid; i < ncand * G::S; i += G::NT) {
        const int c = i / G::S, x = i % G::S;
        const int4 cr = sm.cand[c];
        const int ii = x - cr.y;
        float g = 0.f, dg = 0.f;
        if (ii >= 0 && ii < (sm.clen[c] & 255)) {
            g = nl.G[(size_t)cr.x * 3 * lb + ii];
            dg = nl.DG[(size_t)cr.x * 3 * lb + ii];
        }
        sm.TX[i] = make_float2(g, dg);
    }
    // (3) row entries: one thread per own row (y, z) tests the candidates in
    // order; counts every candidate's entries and marks its rows
    for (int r = tid; r < rows; r += G::NT) {
        const int y = r % G::S, z = Z0 + r / G::S;
        float4* out = sm.rec + (size_t)r * CL_ESTR;
        float2* out2 = sm.rec2 + (size_t)r * CL_ESTR;
        int n = 0;
        for (int c = 0; c < ncand; ++c) {
            const int4 cr = sm.cand[c];
            const int ln = sm.clen[c];
            const int jj = y - cr.z, kk = z - cr.w;
            if (jj < 0 || jj >= ((ln >> 8) & 255) || kk < 0 || kk >= (ln >> 16)) continue;
            int xlo, xhi;
            if (!nl_row_interval<float, M>(nl, cr.x, cr.y, jj, kk, xlo, xhi)) continue;
            if (n < CL_ECAP) {
                const float* Gt = nl.G + (size_t)cr.x * 3 * lb;
                const float* Dt = nl.DG + (size_t)cr.x * 3 * lb;
                const float gy = Gt[lb + jj], dgy = Dt[lb + jj], gz = Gt[2 * lb + kk], dgz = Dt[2 * lb + kk];
                const unsigned meta = (unsigned)c | ((unsigned)xlo << 10) | ((unsigned)xhi << 15);
                out[n] = make_float4(__uint_as_float(meta), gy * gz, 0.f, 0.f);
                out2[n] = make_float2(dgy * gz, gy * dgz);
                atomicAdd(&sm.cstart[c], 1);
                atomicOr(&sm.bits[c * G::BITW + (r >> 5)], 1u << (r & 31));
            } else {
                atomicOr(a.err, ERR_CAPACITY);
            }
            ++n;
        }
        sm.row_n[r] = (uint8_t)min(n, CL_ECAP);
    }
    __syncthreads();
    // (4) entry offsets and 32-entry chunk offsets per candidate (exclusive scans)
    {
        int run = 0, runk = 0;
        for (int c0 = 0; c0 < ncand; c0 += G::NT) {
            const int c = c0 + tid;
            const int v = (c < ncand) ? sm.cstart[c] : 0;
            int tot, totk;
            const int off = block_excl_scan<G::NW>(v, red_i, tot);
            const int offk = block_excl_scan<G::NW>((v + 31) >> 5, red_i, totk);
            if (c < ncand) {
                sm.cstart[c] = run + off;
                sm.chunk[c] = runk + offk;
            }
            run += tot;
            runk += totk;
        }
        if (tid == 0) {
            sm.cstart[ncand] = run;
            sm.chunk[ncand] = runk;
        }
    }
    __syncthreads();
    // (5) candidate-ordered index: an entry's place among its candidate's rows
    // is the number of lower own rows holding the candidate
    for (int r = tid; r < rows; r += G::NT) {
        const int n = sm.row_n[r];
        for (int k = 0; k < n; ++k) {
            const unsigned meta = __float_as_uint(sm.rec[(size_t)r * CL_ESTR + k].x);
            const int c = meta & 1023u;
            const unsigned* b = sm.bits + c * G::BITW;
            int below = __popc(b[r >> 5] & ((1u << (r & 31)) - 1u));
            for (int w = 0; w < (r >> 5); ++w) below += __popc(b[w]);
            sm.cidx[sm.cstart[c] + below] = (uint16_t)(r * CL_ESTR + k);
        }
    }
    __syncthreads();
    return ncand;
}

// Inner products of the vector slab `vec` with every candidate over this
// CTA's rows (trapezoidal rule, Eq. IntApprox, without the h^3 which sits in
// cs/cp): S_c = sum G t, X_c = sum DG_x G t, Y_c = sum DG_y G t, Z_c = sum
// DG_z G t.  Each entry reduces its row along x with the candidate's x
// profile (box-relative slots, so every lane of a chunk reads the same
// profile value), weighted by the row's factors; a warp's sums for a
// candidate are added to Ploc (shared-memory atomics).
template <int M, int NC>
__device__ void cl_dots(const RegionArgs<float>& a, const ClSmem& sm, const float* vec, float4* Ploc, int ncand)
{
    using G = CGeo<M, NC>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int K = sm.chunk[ncand];
    const int Q = (K + G::NW - 1) / G::NW;
    const int j0 = warp * Q, j1 = min(K, j0 + Q);
    if (j0 >= j1) return;
    int lo = 0, hi = ncand - 1;                       // last candidate with chunk <= j0
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sm.chunk[mid] <= j0) lo = mid;
        else hi = mid - 1;
    }
    const bool unrolled = a.nl.lb <= LBMAX;
    int c = lo;
    float aS = 0.f, aX = 0.f, aY = 0.f, aZ = 0.f;
    for (int j = j0; j < j1; ++j) {
        while (j >= sm.chunk[c + 1]) ++c;
        const int e = sm.cstart[c] + (j - sm.chunk[c]) * 32 + lane;
        if (e < sm.cstart[c + 1]) {
            const int slot = sm.cidx[e];
            const float4 r4 = sm.rec[slot];
            const float2 r2 = sm.rec2[slot];
            const unsigned meta = __float_as_uint(r4.x);
            const int xlo = (meta >> 10) & 31u, xhi = (meta >> 15) & 31u;
            const int r = slot / CL_ESTR;
            const float* row = vec + G::LEAD + (r / G::S) * G::PLANE + (r % G::S) * G::PX;
            const float2* tx = sm.TX + (size_t)c * G::S;
            float u = 0.f, u2 = 0.f;
            if (unrolled) {
                const int bx = sm.cand[c].y;
                const uint32_t mask = ((2u << (xhi - bx)) - 1u) & ~((1u << (xlo - bx)) - 1u);
#pragma unroll
                for (int k = 0; k < LBMAX; ++k)
                    if (mask & (1u << k)) {
                        const float2 g = tx[bx + k];
                        const float tv = row[bx + k];
                        u += g.x * tv;
                        u2 += g.y * tv;
                    }
            } else {
                for (int x = xlo; x <= xhi; ++x) {
                    const float2 g = tx[x];
                    const float tv = row[x];
                    u += g.x * tv;
                    u2 += g.y * tv;
                }
            }
            aS += r4.y * u;
            aX += r4.y * u2;
            aY += r2.x * u;
            aZ += r2.y * u;
        }
        if (j + 1 >= j1 || j + 1 >= sm.chunk[c + 1]) {   // warp-uniform: candidate done in this warp
            aS = warp_sumf(aS);
            aX = warp_sumf(aX);
            aY = warp_sumf(aY);
            aZ = warp_sumf(aZ);
            if (lane == 0) {
                atomicAdd(&Ploc[c].x, aS);
                atomicAdd(&Ploc[c].y, aX);
                atomicAdd(&Ploc[c].z, aY);
                atomicAdd(&Ploc[c].w, aZ);
            }
            aS = aX = aY = aZ = 0.f;
        }
    }
}

// P = sum over the cluster's CTAs (in rank order) of their partial sums.
template <int NC>
__device__ inline float4 cl_gather_P(const float4* Ploc, int c)
{
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const float4 v = cl_ld_v4(cl_map(Ploc + c, (unsigned)k));
        s.x += v.x;
        s.y += v.y;
        s.z += v.z;
        s.w += v.w;
    }
    return s;
}

// b0 = cs f0 S + cp (f1 Y + f2 Z), b1 = cp f0 X for every own entry, from P.
template <int M, int NC>
__device__ void cl_bpass(const RegionArgs<float>& a, const ClSmem& sm, const float4* P, int rows)
{
    using G = CGeo<M, NC>;
    const float cs = a.nl.cs, cp = a.nl.cp;
    for (int r = threadIdx.x; r < rows; r += G::NT) {
        const int n = sm.row_n[r];
        for (int k = 0; k < n; ++k) {
            float4* e = sm.rec + (size_t)r * CL_ESTR + k;
            const float4 r4 = *e;
            const float2 r2 = sm.rec2[(size_t)r * CL_ESTR + k];
            const float4 p = P[__float_as_uint(r4.x) & 1023u];
            e->z = cs * r4.y * p.x + cp * (r2.x * p.z + r2.y * p.w);
            e->w = cp * r4.y * p.y;
        }
    }
}

// One value of the current vector at plane zz of column (x, y), from this
// CTA's slab or, across a slab boundary, from the owner's (zero outside the
// region or for idle lanes).
template <int M, int NC>
__device__ __forceinline__ float cl_plane_value(const float* buf, int x, int y, int zz, int Z0, int NZ, bool active)
{
    using G = CGeo<M, NC>;
    if (!active || zz < 0 || zz >= G::S) return 0.f;
    if (zz >= Z0 && zz < Z0 + NZ) return buf[G::LEAD + (zz - Z0) * G::PLANE + y * G::PX + x];
    const int k = G::owner(zz);
    return cl_ld_f32(cl_map(buf + G::LEAD + (zz - G::z0(k)) * G::PLANE + y * G::PX + x, (unsigned)k));
}

// ------------------------------------------------------------------------
// Stencil sweep over this CTA's planes with the projector term folded in:
//   out(p) = s * [ (-3 w_0 + V(p) - shift) t(p) - 1/2 sum_d w_d (6 nbrs at d)
//                  + sum_e (G_x b0_e + DG_x b1_e) ] - sec(p)
// (the last sum over the entries e of p's row whose x-interval holds p).
// out replaces sec pointwise.  Accumulates over the thread's column
// acc_cc = t.t, acc_cs = t.sec (both before the update), acc_co = t.out,
// acc_oo = out.out; the centre value of out goes to *centre.
// ------------------------------------------------------------------------
template <int M, int NC>
__device__ void cl_sweep(const RegionArgs<float>& a, const ClSmem& sm, const float* cur, float* sec,
                         const float* vwin, float s, float dshift, int Z0, int NZ, float& acc_cc, float& acc_cs,
                         float& acc_co, float& acc_oo, double* centre)
{
    using G = CGeo<M, NC>;
    const int x = threadIdx.x & 31, y = threadIdx.x >> 5;
    const bool active = x < G::S;
    const int xs = active ? x : 0;
    const size_t vplane = (size_t)a.g.P1 * a.g.P2;
    const float* vcol = vwin + (size_t)Z0 * vplane + (size_t)y * a.g.P1 + xs;
    float q[13];
#pragma unroll
    for (int d = 0; d < 13; ++d) q[d] = cl_plane_value<M, NC>(cur, xs, y, Z0 - 6 + d, Z0, NZ, active);
    constexpr int VD = 4;
    float vq[VD];
#pragma unroll
    for (int d = 0; d < VD; ++d) vq[d] = (d < NZ) ? vcol[d * vplane] : 0.f;
    float cc = 0.f, cs = 0.f, co = 0.f, oo = 0.f;
#pragma unroll
    for (int lz = 0; lz < G::NZMAX; ++lz) {
        if (lz < NZ) {
            const float c = q[6];
            const float vz = vq[lz % VD];
            if (lz + VD < NZ) vq[lz % VD] = vcol[(lz + VD) * vplane];
            const float* p = cur + G::LEAD + lz * G::PLANE + y * G::PX + xs;
            float lap = 0.f;
#pragma unroll
            for (int d = 1; d <= FD_NO; ++d) {
                const float nb = (p[d] + p[-d]) + (p[d * G::PX] + p[-d * G::PX]) + (q[6 + d] + q[6 - d]);
                lap += a.wd[d] * nb;
            }
            const float hv = (vz + dshift) * c + lap;
            // projector term of this row (warp-uniform entry list)
            const int r = lz * G::S + y;
            const int n = sm.row_n[r];
            const float4* er = sm.rec + (size_t)r * CL_ESTR;
            const float2* tx0 = sm.TX + xs;
            float nlv = 0.f;
            for (int k = 0; k < n; ++k) {
                const float4 e = er[k];
                const unsigned meta = __float_as_uint(e.x);
                const int xlo = (meta >> 10) & 31u, xhi = (meta >> 15) & 31u;
                if (x >= xlo && x <= xhi) {
                    const float2 g = tx0[(size_t)(meta & 1023u) * G::S];
                    nlv += g.x * e.z + g.y * e.w;
                }
            }
            float* sp = sec + G::LEAD + lz * G::PLANE + y * G::PX + xs;
            const float sv = *sp;
            const float out = s * (hv + nlv) - sv;
            if (active) {
                *sp = out;
                cc += c * c;
                cs += c * sv;
                co += c * out;
                oo += out * out;
                if (x == M && y == M && Z0 + lz == M) *centre = (double)out;
            }
        }
#pragma unroll
        for (int d = 0; d < 12; ++d) q[d] = q[d + 1];
        q[12] = cl_plane_value<M, NC>(cur, xs, y, Z0 + lz + 7, Z0, NZ, active);
    }
    acc_cc = cc;
    acc_cs = cs;
    acc_co = co;
    acc_oo = oo;
}

// Zero this CTA's two slabs (halos included) and the per-node arrays.
template <int M, int NC>
__device__ inline void cl_zero_slabs(const ClSmem& sm)
{
    using G = CGeo<M, NC>;
    for (int i = threadIdx.x; i < G::ELEMS; i += G::NT) {
        sm.A[i] = 0.f;
        sm.B[i] = 0.f;
    }
}

// ------------------------------------------------------------------------
// Chebyshev moments on a cluster (FP32 vectors, FP64 moments).
// ------------------------------------------------------------------------
template <int M, int NC>
__global__ void __cluster_dims__(NC, 1, 1) __launch_bounds__(CGeo<M, NC>::NT, 1)
cl_moments_kernel(RegionArgs<float> a)
{
    using G = CGeo<M, NC>;
    extern __shared__ __align__(16) unsigned char cl_smem_raw[];
    __shared__ double red[2][4][32];
    __shared__ int red_i[33];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned rank = cl_rank();
    const int Z0 = G::z0((int)rank), NZ = G::z0((int)rank + 1) - Z0;
    const int rows = NZ * G::S;
    const ClSmem sm = cl_smem(cl_smem_raw, G::S, G::NZMAX, a.nl.ccap, a.npl);
    const int half = a.npl / 2;
    const bool has_nl = a.nl.n_atoms > 0;
    const unsigned crank = (unsigned)G::owner(M);   // the CTA holding the node's own plane
    const long long nclusters = gridDim.x / NC;
    double* s_mom = sm.mom;
    double* s_d2 = sm.mom + (half + 2);
    double* s_d1 = sm.mom + 2 * (half + 2);
    cl_sync();                                      // every CTA of the cluster runs before DSMEM is used
    cl_zero_slabs<M, NC>(sm);
    if (!has_nl)
        for (int r = tid; r < G::ROWS; r += G::NT) sm.row_n[r] = 0;
    __syncthreads();

    for (long long node = blockIdx.x / NC; node < a.g.Nd; node += nclusters) {
        const int qi = (int)(node % a.g.n1);
        const int qj = (int)((node / a.g.n1) % a.g.n2);
        const int qk = (int)(node / ((long long)a.g.n1 * a.g.n2));
        const double chi = a.chi[node], zeta = a.zeta[node];
        const float dshift = (float)(-3.0 * a.g.w[0] - chi);
        const float s1 = (float)(1.0 / zeta), s2 = (float)(2.0 / zeta);
        const float* vwin = a.Vp + ((size_t)qk * a.g.P2 + qj) * a.g.P1 + qi;

        // t^0 = e_q, t^{-1} = 0 (interior of both slabs; halos stay zero)
        for (int i = tid; i < rows * G::S; i += G::NT) {
            const int x = i % G::S, r = i / G::S;
            const int o = G::LEAD + (r / G::S) * G::PLANE + (r % G::S) * G::PX + x;
            sm.A[o] = 0.f;
            sm.B[o] = 0.f;
        }
        int ncand = 0;
        if (has_nl) ncand = cl_setup<M, NC>(a, sm, qi, qj, qk, Z0, NZ, red_i);
        for (int c = tid; c < 2 * ncand; c += G::NT) sm.Ploc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (tid == 0) s_mom[0] = 1.0;
        __syncthreads();
        if (rank == (unsigned)G::owner(M) && tid == 0)
            sm.A[G::LEAD + (M - Z0) * G::PLANE + M * G::PX + M] = 1.f;
        __syncthreads();
        if (has_nl) cl_dots<M, NC>(a, sm, sm.A, sm.Ploc, ncand);
        cl_sync();
        if (has_nl) {
            for (int c = tid; c < ncand; c += G::NT) sm.Pc[c] = cl_gather_P<NC>(sm.Ploc, c);
            __syncthreads();
            cl_bpass<M, NC>(a, sm, sm.Pc, rows);
        }
        __syncthreads();

        float* cur = sm.A;
        float* sec = sm.B;
        for (int i = 0; i < half; ++i) {
            const float s = (i == 0) ? s1 : s2;
            float cc, cs, co, oo;
            cl_sweep<M, NC>(a, sm, cur, sec, vwin, s, dshift, Z0, NZ, cc, cs, co, oo, &s_mom[i + 1]);
            const int par = i & 1;
            const double w2 = warp_total(cc), w1 = warp_total(cs);
            if (lane == 0) {
                red[par][0][warp] = w2;
                red[par][1][warp] = w1;
            }
            { float* t = cur; cur = sec; sec = t; }     // cur = t^{i+1}, sec = t^i
            __syncthreads();                             // the sweep's output is complete in this CTA
            if (tid == 0) {
                double d2 = 0.0, d1 = 0.0;
                for (int w = 0; w < G::NW; ++w) {
                    d2 += red[par][0][w];
                    d1 += red[par][1][w];
                }
                s_d2[i] = d2;                            // t^i . t^i   (this CTA's planes)
                s_d1[i] = d1;                            // t^i . t^{i-1}
            }
            const int pn = (i + 1) & 1;                  // parity of the partial sums of t^{i+1}
            if (has_nl && i + 1 < half) cl_dots<M, NC>(a, sm, cur, sm.Ploc + pn * ncand, ncand);
            cl_sync();                                   // partial sums and every slab of t^{i+1} complete
            if (has_nl && i + 1 < half) {
                for (int c = tid; c < ncand; c += G::NT) {
                    sm.Pc[c] = cl_gather_P<NC>(sm.Ploc + pn * ncand, c);
                    sm.Ploc[(1 - pn) * ncand + c] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                __syncthreads();
                cl_bpass<M, NC>(a, sm, sm.Pc, rows);
            }
            __syncthreads();
        }
        // t^{half}.t^{half} and t^{half}.t^{half-1} over this CTA's planes
        {
            float aa = 0.f, ab = 0.f;
            if (lane < G::S)
                for (int lz = 0; lz < NZ; ++lz) {
                    const int o = G::LEAD + lz * G::PLANE + warp * G::PX + lane;
                    const float u = cur[o], v = sec[o];
                    aa += u * u;
                    ab += u * v;
                }
            const double w2 = warp_total(aa), w1 = warp_total(ab);
            if (lane == 0) {
                red[0][2][warp] = w2;
                red[0][3][warp] = w1;
            }
            __syncthreads();
            if (tid == 0) {
                double d2 = 0.0, d1 = 0.0;
                for (int w = 0; w < G::NW; ++w) {
                    d2 += red[0][2][w];
                    d1 += red[0][3][w];
                }
                s_d2[half] = d2;
                s_d1[half] = d1;
            }
        }
        cl_sync();                                       // every CTA's sums are final
        if (rank == crank) {
            double* out = a.moments + node * (long long)(a.npl + 1);
            for (int j = tid; j <= a.npl; j += G::NT) {
                double r;
                if (j <= half) {
                    r = s_mom[j];
                } else {
                    const bool even = (j & 1) == 0;
                    const int idx = even ? j / 2 : (j + 1) / 2;
                    const double* arr = even ? s_d2 : s_d1;
                    double t = 0.0;
                    for (int k = 0; k < NC; ++k) t += cl_ld_f64(cl_map(arr + idx, (unsigned)k));
                    r = even ? 2.0 * t - s_mom[0] : 2.0 * t - s_mom[1];   // product rule (corrected sign)
                }
                out[j] = r;
                if (!(fabs(r) <= 1.0 + a.mom_tol)) atomicOr(a.err, ERR_BOUNDS);
            }
        }
        cl_sync();                                       // partners' sums read before the next node reuses them
    }
}

// ------------------------------------------------------------------------
// Lanczos on a cluster (FP32 vectors, FP64 coefficients).  Start vector
// uniform 1/sqrt(Ns) on the region, n_lanczos steps without
// re-orthogonalisation, early stop on breakdown beta <= 1e-10 * scale.
// Writes alpha[0..k-1], beta[0..k-2] and k per node.
// ------------------------------------------------------------------------
template <int M, int NC>
__global__ void __cluster_dims__(NC, 1, 1) __launch_bounds__(CGeo<M, NC>::NT, 1)
cl_lanczos_kernel(RegionArgs<float> a)
{
    using G = CGeo<M, NC>;
    extern __shared__ __align__(16) unsigned char cl_smem_raw[];
    __shared__ double red[3][32];
    __shared__ int red_i[33];
    __shared__ float s_alpha, s_inv, s_beta;
    __shared__ int s_stop;
    __shared__ double s_dummy;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned rank = cl_rank();
    const int Z0 = G::z0((int)rank), NZ = G::z0((int)rank + 1) - Z0;
    const int rows = NZ * G::S;
    const ClSmem sm = cl_smem(cl_smem_raw, G::S, G::NZMAX, a.nl.ccap, 0);
    const bool has_nl = a.nl.n_atoms > 0;
    const long long nclusters = gridDim.x / NC;
    const float dshift = (float)(-3.0 * a.g.w[0]);
    const float v0 = (float)(1.0 / sqrt((double)(G::S * G::S * G::S)));
    cl_sync();
    cl_zero_slabs<M, NC>(sm);
    if (!has_nl)
        for (int r = tid; r < G::ROWS; r += G::NT) sm.row_n[r] = 0;
    __syncthreads();

    for (long long node = blockIdx.x / NC; node < a.g.Nd; node += nclusters) {
        const int qi = (int)(node % a.g.n1);
        const int qj = (int)((node / a.g.n1) % a.g.n2);
        const int qk = (int)(node / ((long long)a.g.n1 * a.g.n2));
        const float* vwin = a.Vp + ((size_t)qk * a.g.P2 + qj) * a.g.P1 + qi;
        for (int i = tid; i < rows * G::S; i += G::NT) {
            const int x = i % G::S, r = i / G::S;
            const int o = G::LEAD + (r / G::S) * G::PLANE + (r % G::S) * G::PX + x;
            sm.A[o] = v0;
            sm.B[o] = 0.f;
        }
        int ncand = 0;
        if (has_nl) ncand = cl_setup<M, NC>(a, sm, qi, qj, qk, Z0, NZ, red_i);
        for (int c = tid; c < 2 * ncand; c += G::NT) sm.Ploc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        // the start vector's partial sums take parity 1, so step 0 (parity 0) starts from zero
        if (has_nl) cl_dots<M, NC>(a, sm, sm.A, sm.Ploc + ncand, ncand);
        cl_sync();
        if (has_nl) {
            for (int c = tid; c < ncand; c += G::NT) sm.Pc[c] = cl_gather_P<NC>(sm.Ploc + ncand, c);
            __syncthreads();
            cl_bpass<M, NC>(a, sm, sm.Pc, rows);
        }
        __syncthreads();

        double* alpha = a.alpha + node * (long long)a.nl_cap;
        double* beta = a.beta + node * (long long)a.nl_cap;
        double bprev = 0.0, scale = 0.0;
        for (int it = 0; it < a.n_lanczos; ++it) {
            const int par = it & 1;
            // w = H v - beta_prev v_old  (sec holds beta_prev v_old, then w)
            float cc, cs, co, oo;
            cl_sweep<M, NC>(a, sm, sm.A, sm.B, vwin, 1.f, dshift, Z0, NZ, cc, cs, co, oo, &s_dummy);
            const double wa = warp_total(co), ww = warp_total(oo), wv = warp_total(cc);
            if (lane == 0) {
                red[0][warp] = wa;
                red[1][warp] = ww;
                red[2][warp] = wv;
            }
            __syncthreads();
            if (tid == 0) {
                double pa = 0.0, pw = 0.0, pv = 0.0;
                for (int w = 0; w < G::NW; ++w) {
                    pa += red[0][w];
                    pw += red[1][w];
                    pv += red[2][w];
                }
                sm.part[par * 4 + 0] = pa;
                sm.part[par * 4 + 1] = pw;
                sm.part[par * 4 + 2] = pv;
            }
            cl_sync();                                   // every CTA's partial sums of this step are final
            // v.w, w.w, v.v over the region, added in rank order (the same in every CTA)
            double va = 0.0, wsq = 0.0, vsq = 0.0;
            for (int k = 0; k < NC; ++k) {
                va += cl_ld_f64(cl_map(sm.part + par * 4 + 0, (unsigned)k));
                wsq += cl_ld_f64(cl_map(sm.part + par * 4 + 1, (unsigned)k));
                vsq += cl_ld_f64(cl_map(sm.part + par * 4 + 2, (unsigned)k));
            }
            const double al = va;
            const double b2 = wsq - 2.0 * al * va + al * al * vsq;   // |w - alpha v|^2
            const double b = sqrt(b2 > 0.0 ? b2 : 0.0);
            if (fabs(al) + bprev > scale) scale = fabs(al) + bprev;
            const int stop = (it == a.n_lanczos - 1) || (b <= 1e-10 * scale);
            if (rank == 0 && tid == 0) {
                alpha[it] = al;
                if (!stop) beta[it] = b;
                else a.klen[node] = it + 1;
            }
            bprev = b;
            if (stop) {
                cl_sync();                               // partners' sums read before the next node
                break;
            }
            // v' = (w - alpha v) / beta, sec = beta v
            const float alT = (float)al, inv = (float)(1.0 / b), bT = (float)b;
            if (lane < G::S)
                for (int lz = 0; lz < NZ; ++lz) {
                    const int o = G::LEAD + lz * G::PLANE + warp * G::PX + lane;
                    const float v = sm.A[o], w = sm.B[o];
                    sm.A[o] = (w - alT * v) * inv;
                    sm.B[o] = bT * v;
                }
            __syncthreads();
            // inner products of v' itself (its own rounding, not a recombination)
            if (has_nl) cl_dots<M, NC>(a, sm, sm.A, sm.Ploc + par * ncand, ncand);
            cl_sync();                                   // v' complete in every slab, partial sums final
            if (has_nl) {
                for (int c = tid; c < ncand; c += G::NT) {
                    sm.Pc[c] = cl_gather_P<NC>(sm.Ploc + par * ncand, c);
                    sm.Ploc[(1 - par) * ncand + c] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                __syncthreads();
                cl_bpass<M, NC>(a, sm, sm.Pc, rows);
            }
            __syncthreads();
        }
    }
    (void)s_alpha; (void)s_inv; (void)s_beta; (void)s_stop;
}

}  // namespace sq
