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
// boundary of Section 3.1 for free).  Warp y owns row y of every plane (lane
// = x), so each stencil load of a warp is one contiguous, bank-conflict-free
// row segment; thread (x, y) marches in z, keeping the 13 z-values it needs in
// a register queue.  The second vector (t^{i-1} / Lanczos v_old) is touched only
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
    static constexpr int NT = 32 * S;     // one warp per region row y, lane = x (lanes >= S idle)
    static constexpr int NW = S;
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

// CTAs of a region kernel that fit one SM by shared memory and threads; used
// as the min-blocks hint of __launch_bounds__ so ptxas sizes registers for the
// occupancy that shared memory allows anyway.
template <typename T, int M>
constexpr int region_min_blocks()
{
    size_t smem = (fits_double_buffer<T, M>() ? 2 : 1) * (size_t)Geo<M>::ELEMS * sizeof(T) + 8192;
    int by_smem = (int)(232448 / smem);
    int by_threads = 2048 / Geo<M>::NT;
    int by_regs = 65536 / (Geo<M>::NT * 64);      // keep >= 64 registers per thread
    int b = by_smem < by_threads ? by_smem : by_threads;
    b = b < by_regs ? b : by_regs;
    return b < 1 ? 1 : b;
}

// Per-CTA scratch carving (identical on host and device).
struct ScratchLayout {
    size_t buf, cand, P, TX, ent_meta, ent_f, cent_meta, cent_f, row_start, row_fill, cand_start, total;
};
__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
__host__ __device__ inline ScratchLayout scratch_layout(int m, size_t tsize)
{
    int S = 2 * m + 1;
    ScratchLayout L;
    size_t off = 0;
    const size_t cap = (size_t)S * S * ENTRIES_PER_ROW;
    L.buf = off;        off = align256(off + (size_t)S * S * S * tsize);
    L.cand = off;       off = align256(off + (size_t)MAX_CAND * sizeof(int4));
    L.P = off;          off = align256(off + (size_t)MAX_CAND * 4 * tsize);
    L.TX = off;         off = align256(off + (size_t)MAX_CAND * S * 2 * tsize);
    L.ent_meta = off;   off = align256(off + cap * sizeof(uint32_t));
    L.ent_f = off;      off = align256(off + cap * 4 * tsize);
    L.cent_meta = off;  off = align256(off + cap * sizeof(uint32_t));
    L.cent_f = off;     off = align256(off + cap * 4 * tsize);
    L.row_start = off;  off = align256(off + (size_t)(S * S + 1) * sizeof(int));
    L.row_fill = off;   off = align256(off + (size_t)S * S * sizeof(int));
    L.cand_start = off; off = align256(off + (size_t)(MAX_CAND + 1) * sizeof(int));
    L.total = off;
    return L;
}

template <typename T>
struct RegionArgs {
    GridParams g;
    T wd[FD_NO + 1];                 // -w_d/2 in precision T (kernel parameters: constant-bank operands)
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
    s.TX = reinterpret_cast<T*>(base + L.TX);
    s.ent_meta = reinterpret_cast<uint32_t*>(base + L.ent_meta);
    s.ent_f = reinterpret_cast<T*>(base + L.ent_f);
    s.cent_meta = reinterpret_cast<uint32_t*>(base + L.cent_meta);
    s.cent_f = reinterpret_cast<T*>(base + L.cent_f);
    s.row_start = reinterpret_cast<int*>(base + L.row_start);
    s.row_fill = reinterpret_cast<int*>(base + L.row_fill);
    s.cand_start = reinterpret_cast<int*>(base + L.cand_start);
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

// Error-free sum of two floats (Knuth's TwoSum): a + b = s + e exactly.
__device__ inline void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Warp sum of per-thread column partials, returned in FP64 on every lane.
// FP32: a compensated FP32 tree (value + running error) -- no FP64 arithmetic
// per lane, which matters on GB300's narrow FP64 pipe; FP64: a plain tree.
__device__ inline double warp_total(float v)
{
    float s = v, c = 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float t = __shfl_xor_sync(0xffffffffu, s, o);
        float tc = __shfl_xor_sync(0xffffffffu, c, o);
        float e;
        two_sum(s, t, s, e);
        c = c + (tc + e);
    }
    return (double)s + (double)c;
}
__device__ inline double warp_total(double v) { return warp_sum(v); }

// Block sums: lane 0 of each warp stores its warp total in red[w]; after the
// barrier one thread adds the warp totals in index order (fixed order, FP64).

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
// region, kept in tile-list order.  Entries: one per (candidate, region row
// (y,z)) whose clipped support interval in x is non-empty, with the row's
// y/z Gaussian factors.  Both entry orders are fixed (rows ascending within a
// candidate; candidates ascending within a row), so every sum below has a
// fixed order and results are bitwise reproducible.
// ------------------------------------------------------------------------
template <typename T, int M>
__device__ int nl_setup(const RegionArgs<T>& a, const CtaScratch<T>& sc, int qi, int qj, int qk,
                        int* red_i)
{
    using G = Geo<M>;
    const NLParams<T>& nl = a.nl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lb = nl.lb;
    int tile = (qi / TILE) + nl.ntile[0] * ((qj / TILE) + nl.ntile[1] * (qk / TILE));
    int beg = nl.tile_start[tile], end = nl.tile_start[tile + 1];
    // (1) candidates, ordered compaction of the tile list
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
    const int nrow = G::S * G::S;
    const int cap = nrow * ENTRIES_PER_ROW;
    for (int r = tid; r < nrow; r += G::NT) sc.row_fill[r] = 0;
    __syncthreads();
    // (2) x-tables of the candidates in region columns
    for (int i = tid; i < ncand * G::S; i += G::NT) {
        int c = i / G::S, x = i % G::S;
        int4 rec = sc.cand[c];
        int ii = x - rec.y;
        T g = 0, dg = 0;
        if (ii >= 0 && ii < nl.atoms[rec.x].len[0]) {
            g = nl.G[(size_t)rec.x * 3 * lb + ii];
            dg = nl.DG[(size_t)rec.x * 3 * lb + ii];
        }
        sc.TX[2 * i] = g;
        sc.TX[2 * i + 1] = dg;
    }
    // (3) entries: count per row and per candidate, scan, then fill (warp per
    // candidate; rows of its box clipped to the region, ascending r)
    for (int pass = 0; pass < 2; ++pass) {
        for (int c = warp; c < ncand; c += G::NW) {
            int4 rec = sc.cand[c];
            AtomTab at = nl.atoms[rec.x];
            const T* Gt = nl.G + (size_t)rec.x * 3 * lb;
            const T* Dt = nl.DG + (size_t)rec.x * 3 * lb;
            int j0 = max(0, -rec.z), j1 = min(at.len[1], G::S - rec.z);
            int k0 = max(0, -rec.w), k1 = min(at.len[2], G::S - rec.w);
            int nj = j1 - j0;
            int nrows = (nj > 0 && k1 > k0) ? nj * (k1 - k0) : 0;
            int cbase = pass ? sc.cand_start[c] : 0;
            int cnt = 0;
            for (int r0 = 0; r0 < nrows; r0 += 32) {
                int rr = r0 + lane;
                int ok = 0, xlo = 0, xhi = 0, row = 0, jj = 0, kk = 0;
                if (rr < nrows) {
                    jj = j0 + rr % nj;
                    kk = k0 + rr / nj;
                    const uint8_t* iv = nl.ivl + (((size_t)rec.x * lb + jj) * lb + kk) * 2;
                    xlo = max((int)iv[0] + rec.y, 0);
                    xhi = min((int)iv[1] + rec.y, G::S - 1);
                    ok = (iv[0] <= iv[1]) && (xlo <= xhi);
                    row = (rec.z + jj) + G::S * (rec.w + kk);
                }
                unsigned bal = __ballot_sync(0xffffffffu, ok);
                if (ok) {
                    if (!pass) {
                        atomicAdd(&sc.row_fill[row], 1);
                    } else {
                        T gy = Gt[lb + jj], dgy = Dt[lb + jj], gz = Gt[2 * lb + kk], dgz = Dt[2 * lb + kk];
                        int ce = cbase + cnt + __popc(bal & ((1u << lane) - 1u));
                        if (ce < cap) {
                            sc.cent_meta[ce] = (uint32_t)row | ((uint32_t)xlo << 10) | ((uint32_t)xhi << 15);
                            sc.cent_f[4 * ce + 0] = gy * gz;
                            sc.cent_f[4 * ce + 1] = dgy * gz;
                            sc.cent_f[4 * ce + 2] = gy * dgz;
                            sc.cent_f[4 * ce + 3] = 0;
                        }
                        int se = sc.row_start[row] + atomicAdd(&sc.row_fill[row], 1);
                        if (se < cap) {
                            sc.ent_meta[se] = (uint32_t)c | ((uint32_t)xlo << 10) | ((uint32_t)xhi << 15);
                            sc.ent_f[4 * se + 0] = gy * gz;
                            sc.ent_f[4 * se + 1] = dgy * gz;
                            sc.ent_f[4 * se + 2] = gy * dgz;
                            sc.ent_f[4 * se + 3] = 0;
                        }
                    }
                }
                cnt += __popc(bal);
            }
            if (!pass && lane == 0) sc.cand_start[c] = cnt;
        }
        __syncthreads();
        if (!pass) {
            // exclusive scans: rows (counts in row_fill) and candidates
            int run = 0;
            for (int r0 = 0; r0 < nrow; r0 += G::NT) {
                int r = r0 + tid;
                int v = (r < nrow) ? sc.row_fill[r] : 0;
                int tot;
                int off = block_excl_scan<G::NW>(v, red_i, tot);
                if (r < nrow) sc.row_start[r] = min(run + off, cap);
                run += tot;
            }
            if (tid == 0) {
                sc.row_start[nrow] = min(run, cap);
                if (run > cap) atomicOr(a.err, ERR_CAPACITY);
            }
            run = 0;
            for (int c0 = 0; c0 < ncand; c0 += G::NT) {
                int c = c0 + tid;
                int v = (c < ncand) ? sc.cand_start[c] : 0;
                int tot;
                int off = block_excl_scan<G::NW>(v, red_i, tot);
                if (c < ncand) sc.cand_start[c] = min(run + off, cap);
                run += tot;
            }
            if (tid == 0) sc.cand_start[ncand] = min(run, cap);
            __syncthreads();
            for (int r = tid; r < nrow; r += G::NT) sc.row_fill[r] = 0;
            __syncthreads();
        }
    }
    // (4) order each row's entries by candidate (a handful per row)
    for (int r = tid; r < nrow; r += G::NT) {
        int b = sc.row_start[r], n = sc.row_start[r + 1] - b;
        uint32_t* Mt = sc.ent_meta + b;
        T* F = sc.ent_f + 4 * (size_t)b;
        for (int i = 1; i < n; ++i) {
            uint32_t v = Mt[i];
            T f0 = F[4 * i], f1 = F[4 * i + 1], f2 = F[4 * i + 2];
            int j = i - 1;
            while (j >= 0 && (Mt[j] & 1023u) > (v & 1023u)) {
                Mt[j + 1] = Mt[j];
                F[4 * (j + 1)] = F[4 * j];
                F[4 * (j + 1) + 1] = F[4 * j + 1];
                F[4 * (j + 1) + 2] = F[4 * j + 2];
                --j;
            }
            Mt[j + 1] = v;
            F[4 * (j + 1)] = f0;
            F[4 * (j + 1) + 1] = f1;
            F[4 * (j + 1) + 2] = f2;
        }
    }
    __syncthreads();
    return ncand;
}

// Projector inner products of the shared-memory vector (trapezoidal rule,
// Eq. IntApprox, without the h^3 which sits in cs/cp):
//   S_c = sum G t, X_c = sum D_x G t, Y_c = sum D_y G t, Z_c = sum D_z G t
// over the support of candidate c inside the region.  The Gaussian factorises
// per axis: each row is reduced along x with the x-table, then weighted by the
// row's y/z factors.  One warp per candidate, lanes over its rows, a
// warp-uniform x loop (table values are broadcasts), warp tree at the end.
template <typename T, int M>
__device__ void nl_dots(const RegionArgs<T>& a, const CtaScratch<T>& sc, const T* cur, int ncand)
{
    using G = Geo<M>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = warp; c < ncand; c += G::NW) {
        int4 rec = sc.cand[c];
        const int x0 = max(rec.y, 0), x1 = min(rec.y + a.nl.atoms[rec.x].len[0], G::S) - 1;
        const T* tx = sc.TX + (size_t)c * G::S * 2;
        const int e0 = sc.cand_start[c], e1 = sc.cand_start[c + 1];
        T aS = 0, aX = 0, aY = 0, aZ = 0;
        for (int eb = e0; eb < e1; eb += 32) {
            const int e = eb + lane;
            const bool valid = e < e1;
            uint32_t mt = valid ? sc.cent_meta[e] : 0u;
            int r = mt & 1023u, xlo = valid ? (int)((mt >> 10) & 31u) : 1, xhi = (mt >> 15) & 31u;
            int y = r % G::S, z = r / G::S;
            const T* row = cur + G::LEAD + z * G::PLANE + y * G::PX;
            T u = 0, u2 = 0;
            for (int x = x0; x <= x1; ++x) {
                T g = tx[2 * x], dg = tx[2 * x + 1];
                T tv = (x >= xlo && x <= xhi) ? row[x] : T(0);
                u += g * tv;
                u2 += dg * tv;
            }
            if (valid) {
                T f0 = sc.cent_f[4 * e], f1 = sc.cent_f[4 * e + 1], f2 = sc.cent_f[4 * e + 2];
                aS += f0 * u;
                aX += f0 * u2;
                aY += f1 * u;
                aZ += f2 * u;
            }
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

// V_nl t at region column x of row r (warp-uniform loop over the row's
// entries; candidates in fixed order):
//   sum_c h^3 G_x [ f0 (gamma_s A_s^2 S_c + ...) ] =
//   sum_e TX_c(x) . (b0, b1),  b0 = cs f0 S + cp (f1 Y + f2 Z),  b1 = cp f0 X
template <typename T, int M>
__device__ inline T nl_row_apply(const RegionArgs<T>& a, const CtaScratch<T>& sc, int r, int x)
{
    using G = Geo<M>;
    const int e0 = sc.row_start[r], e1 = sc.row_start[r + 1];
    const T cs = a.nl.cs, cp = a.nl.cp;
    T acc = 0;
    for (int e = e0; e < e1; ++e) {
        uint32_t mt = sc.ent_meta[e];
        int c = mt & 1023u, xlo = (mt >> 10) & 31u, xhi = (mt >> 15) & 31u;
        T f0 = sc.ent_f[4 * e], f1 = sc.ent_f[4 * e + 1], f2 = sc.ent_f[4 * e + 2];
        T pS = sc.P[4 * c], pX = sc.P[4 * c + 1], pY = sc.P[4 * c + 2], pZ = sc.P[4 * c + 3];
        T b0 = cs * f0 * pS + cp * (f1 * pY + f2 * pZ);
        T b1 = cp * f0 * pX;
        const T* tx = sc.TX + ((size_t)c * G::S + x) * 2;
        T g = (x >= xlo && x <= xhi) ? tx[0] : T(0);
        T dg = (x >= xlo && x <= xhi) ? tx[1] : T(0);
        acc += g * b0 + dg * b1;
    }
    return acc;
}

// ------------------------------------------------------------------------
// Stencil sweep of H (Eq. FD:Laplacian + V, plus the projector term):
//   out(p) = s * [ (-3 w_0 + V(p) - shift) t(p) - 1/2 sum_d w_d (6 nbrs at d)
//                  + (V_nl t)(p) ] - a_old * sec(p)
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
__device__ void stencil_sweep(const RegionArgs<T>& a, const CtaScratch<T>& sc, bool has_nl, T* cur, T* sec,
                              const T* vwin, T s, T a_old, T dshift, T& acc_a, T& acc_b, double* centre_out)
{
    using G = Geo<M>;
    using SV = Sec<M, DB>;
    const int x = threadIdx.x & 31, y = threadIdx.x >> 5;
    const bool active = x < G::S;
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
                lap += a.wd[d] * nb;
            }
            T vz = vcol[z * vplane];
            T hv = (vz + dshift) * c + lap;
            if (has_nl) hv += nl_row_apply<T, M>(a, sc, y + G::S * z, x);
            out = s * hv - a_old * bcol[z * SV::ZS];
        }
        if (RECUR && !DB) __syncthreads();
        if (active) {
            if (RECUR) {
                if (!DB) col[z * G::PLANE] = out;
                bcol[z * SV::ZS] = DB ? out : c;
                aa += out * out;
                ab += out * c;
                if (x == M && y == M && z == M) *centre_out = (double)out;
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

// ------------------------------------------------------------------------
// Chebyshev moments kernel (Section 3.2, Eqs. Rec:FD and rhoqj).
// ------------------------------------------------------------------------
template <typename T, int M, bool DB>
__global__ void __launch_bounds__(Geo<M>::NT, (region_min_blocks<T, M>()))
moments_kernel(RegionArgs<T> a)
{
    using G = Geo<M>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* bufA = reinterpret_cast<T*>(smem_raw);
    __shared__ double red[2][2][32];          // [step parity][d2, d1][warp]
    __shared__ int red_i[33];
    __shared__ double s_mom[MAX_NPL / 2 + 2];
    __shared__ double s_d2[MAX_NPL / 2 + 2];
    __shared__ double s_d1[MAX_NPL / 2 + 2];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const CtaScratch<T> sc = cta_scratch(a, M);
    T* bufB = DB ? bufA + G::ELEMS : sc.buf;
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
            }
            T aa, ab;
            stencil_sweep<T, M, true, DB>(a, sc, has_nl, cur, sec, vwin, s, (i == 0) ? T(0) : T(1), dshift, aa,
                                          ab, &s_mom[i + 1]);
            // t^{i+1}.t^{i+1} and t^{i+1}.t^i: column sums in T, warp trees, FP64 across warps
            const int par = i & 1;
            double w2 = warp_total(aa), w1 = warp_total(ab);
            if (lane == 0) { red[par][0][warp] = w2; red[par][1][warp] = w1; }
            __syncthreads();                       // also publishes the sweep and rho^{i+1}
            if (tid == 0) {
                double d2 = 0.0, d1 = 0.0;
                for (int w = 0; w < G::NW; ++w) { d2 += red[par][0][w]; d1 += red[par][1][w]; }
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
// extremes are found by tridiag_bounds_kernel.  The scalar recurrence
// (alpha, beta, breakdown test) runs on thread 0 in FP64 and is broadcast.
// ------------------------------------------------------------------------
template <typename T, int M, bool DB>
__global__ void __launch_bounds__(Geo<M>::NT, (region_min_blocks<T, M>()))
lanczos_kernel(RegionArgs<T> a)
{
    using G = Geo<M>;
    using SV = Sec<M, DB>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    __shared__ double red_a[32], red_b[32];  // alpha and beta partials (separate: no reuse race)
    __shared__ int red_i[33];
    __shared__ T s_alpha, s_inv, s_bprev;
    __shared__ int s_stop;
    __shared__ double s_dummy;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x = lane, y = warp;
    const bool active = x < G::S;
    const CtaScratch<T> sc = cta_scratch(a, M);
    T* sec = DB ? sm + G::ELEMS : sc.buf;
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
        double bprev = 0.0, scale = 0.0;           // thread 0 only
        T bprevT = 0;
        for (int it = 0; it < a.n_lanczos; ++it) {
            // w = H v - beta_prev v_old  (v_old and then w live in sec)
            if (has_nl) {
                nl_dots<T, M>(a, sc, sm, ncand);
                __syncthreads();
            }
            T aa, ab;
            stencil_sweep<T, M, false, DB>(a, sc, has_nl, sm, sec, vwin, T(1), bprevT, dshift, aa, ab, &s_dummy);
            double wt = warp_total(ab);
            if (lane == 0) red_a[warp] = wt;
            __syncthreads();
            if (tid == 0) {
                double al = 0.0;
                for (int w = 0; w < G::NW; ++w) al += red_a[w];
                alpha[it] = al;
                s_alpha = (T)al;
                if (fabs(al) + bprev > scale) scale = fabs(al) + bprev;
            }
            __syncthreads();
            // w -= alpha v ; beta = |w|
            const T alT = s_alpha;
            T acc = 0;
            if (active)
                for (int z = 0; z < G::S; ++z) {
                    T w = bcol[z * SV::ZS] - alT * col[z * G::PLANE];
                    bcol[z * SV::ZS] = w;
                    acc += w * w;
                }
            wt = warp_total(acc);
            if (lane == 0) red_b[warp] = wt;
            __syncthreads();
            if (tid == 0) {
                double b2 = 0.0;
                for (int w = 0; w < G::NW; ++w) b2 += red_b[w];
                double b = sqrt(b2);
                int stop = (it == a.n_lanczos - 1) || (b <= 1e-10 * scale);
                if (!stop) beta[it] = b;
                else a.klen[node] = it + 1;
                s_stop = stop;
                s_inv = (T)(1.0 / b);
                s_bprev = (T)b;
                bprev = b;
            }
            __syncthreads();
            if (s_stop) break;
            // v_old <- v, v <- w / beta
            const T inv = s_inv;
            bprevT = s_bprev;
            if (active)
                for (int z = 0; z < G::S; ++z) {
                    T w = bcol[z * SV::ZS];
                    T v = col[z * G::PLANE];
                    bcol[z * SV::ZS] = v;
                    col[z * G::PLANE] = w * inv;
                }
            __syncthreads();
        }
        __syncthreads();
    }
}

template <typename T, int M>
size_t region_smem()
{
    return (fits_double_buffer<T, M>() ? 2 : 1) * (size_t)Geo<M>::ELEMS * sizeof(T);
}

}  // namespace sq
