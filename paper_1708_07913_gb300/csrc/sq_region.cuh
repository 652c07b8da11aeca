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
#include <math.h>
#include <string.h>

#include "sq_internal.cuh"

namespace sq {

template <int M>
struct Geo {
    static constexpr int S = 2 * M + 1;
    // Compact form for 27^3 and 29^3 regions (m = 13, 14): rows of pitch S+2
    // (2 zero columns) and planes of exactly S rows, so that two vectors and
    // the hot projector tables fit a CTA's shared memory (two fully padded
    // 29^3 vectors would not fit at all); the stencil then masks the x
    // neighbours at distance 3 to 6 of the edge columns and the y neighbours
    // that fall outside the region, instead of reading zero halos.  LEAD and
    // the 6-element tail keep every x-neighbour address inside the buffer.
    static constexpr bool CY = (M == 13 || M == 14);
    static constexpr int PX = CY ? S + 2 : S + 6;
    static constexpr int PY = CY ? S : S + 6;
    static constexpr int PLANE = PX * PY;
    static constexpr int LEAD = CY ? 6 : 6 * PX + 6;
    static constexpr int ELEMS = LEAD + S * PLANE + (CY ? 6 : 0);
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

// Dynamic shared memory of the region vectors.
template <typename T, int M>
__host__ __device__ constexpr size_t region_smem()
{
    return (fits_double_buffer<T, M>() ? 2 : 1) * (size_t)Geo<M>::ELEMS * sizeof(T);
}

// Per-CTA scratch carving (identical on host and device).
struct ScratchLayout {
    size_t buf, cand, clen, P, TX, seg, cent, rec, cand_start, chunk_first, row_n, total;
};
__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
__host__ __device__ inline size_t rec_size(size_t tsize) { return tsize == 4 ? 16 : 32; }   // sizeof(EntRec<T>)
__host__ __device__ inline ScratchLayout scratch_layout(int m, size_t tsize)
{
    int S = 2 * m + 1;
    ScratchLayout L;
    size_t off = 0;
    const size_t cap = (size_t)S * S * ENTRIES_PER_ROW;
    L.buf = off;         off = align256(off + (size_t)S * S * S * tsize);
    L.cand = off;        off = align256(off + (size_t)MAX_CAND * sizeof(int4));
    L.clen = off;        off = align256(off + (size_t)MAX_CAND * sizeof(int));
    L.P = off;           off = align256(off + (size_t)MAX_CAND * 4 * tsize);
    L.TX = off;          off = align256(off + (size_t)MAX_CAND * NL_BOX * 2 * tsize);
    L.seg = off;         off = align256(off + (size_t)(MAX_CAND + 32) * 4 * tsize);
    L.cent = off;        off = align256(off + cap * rec_size(tsize));
    L.rec = off;         off = align256(off + cap * rec_size(tsize));
    L.cand_start = off;  off = align256(off + (size_t)(MAX_CAND + 1) * sizeof(int));
    L.chunk_first = off; off = align256(off + (size_t)(MAX_CAND + 1) * sizeof(int));
    L.row_n = off;       off = align256(off + (size_t)S * S);
    L.total = off;
    return L;
}

// Shared-memory placement of the per-candidate tables for ccap candidates
// with x-tables of lb box columns (offsets from a 16-byte aligned base; total
// includes 16 bytes of slack for aligning that base).  NL_ALL: every table;
// NL_HOT: only those read every step (inner products, x-tables, chunk and
// entry offsets), the rest staying in global scratch, for regions whose
// vectors leave too little room for all of them.
enum : int { NL_GLOBAL = 0, NL_ALL = 1, NL_HOT = 2 };
struct NLSmem {
    size_t cand, P, TX, seg, clen, cand_start, chunk_first, row_n, total;
};
__host__ __device__ inline NLSmem nl_smem_layout(int mode, int ccap, int S, int lb, size_t tsize)
{
    NLSmem L;
    size_t o = 0;
    L.P = o;           o = align16(o + (size_t)ccap * 4 * tsize);
    L.TX = o;          o = align16(o + (size_t)ccap * 2 * lb * tsize);
    L.cand_start = o;  o = align16(o + (size_t)(ccap + 1) * sizeof(int));
    L.chunk_first = o; o = align16(o + (size_t)(ccap + 1) * sizeof(int));
    L.cand = L.seg = L.clen = L.row_n = 0;
    if (mode == NL_ALL) {
        L.cand = o;    o = align16(o + (size_t)ccap * sizeof(int4));
        L.seg = o;     o = align16(o + (size_t)(ccap + 32) * 4 * tsize);
        L.clen = o;    o = align16(o + (size_t)ccap * sizeof(int));
        L.row_n = o;   o = align16(o + (size_t)S * S);
    }
    L.total = o + 16;
    return L;
}
__host__ __device__ inline size_t nl_smem_bytes(int mode, int ccap, int S, int lb, size_t tsize)
{
    return nl_smem_layout(mode, ccap, S, lb, tsize).total;
}

// Per-node moment scratch of the moments kernel in dynamic shared memory:
// rho^i (centre values) and the two product sums, npl/2 + 2 each.
__host__ __device__ inline size_t mom_smem_bytes(int npl) { return 16 + (size_t)3 * (npl / 2 + 2) * sizeof(double); }

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

// The region-kernel arguments of a context (host).
template <typename T>
inline RegionArgs<T> region_args(const sq_ctx* c)
{
    RegionArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.g = c->g;
    for (int d = 0; d <= FD_NO; ++d) a.wd[d] = (T)(-0.5 * c->g.w[d]);
    a.Vp = (const T*)c->Vp;
    a.nl.n_atoms = (c->has_s || c->has_p) ? c->n_atoms : 0;
    a.nl.atoms = c->d_atoms;
    a.nl.G = (const T*)c->d_G;
    a.nl.DG = (const T*)c->d_DG;
    a.nl.ivl = c->d_ivl;
    a.nl.lb = c->lb;
    a.nl.ccap = c->ccap;
    a.nl.smem = c->nl_mode;
    a.nl.tile_start = c->d_tile_start;
    a.nl.tile_cand = c->d_tile_cand;
    for (int i = 0; i < 3; ++i) a.nl.ntile[i] = c->ntile[i];
    const double h3 = c->g.h * c->g.h * c->g.h;
    const double As2 = pow(M_PI * c->rc * c->rc, -1.5);          // A_s^2
    const double Ap2 = 2.0 / (c->rc * c->rc) * As2;              // A_p^2
    a.nl.cs = (T)(c->has_s ? h3 * c->gamma_s * As2 : 0.0);
    a.nl.cp = (T)(c->has_p ? h3 * c->gamma_p * Ap2 : 0.0);
    a.scratch = (char*)c->d_scratch;
    a.scratch_stride = c->scratch_bytes_per_cta;
    a.err = c->d_err;
    a.npl = c->npl;
    a.mom_tol = c->precision == SQ_FP32 ? 1e-4 : 1e-6;
    return a;
}

template <typename T>
__device__ inline CtaScratch<T> cta_scratch(const RegionArgs<T>& a, int m)
{
    ScratchLayout L = scratch_layout(m, sizeof(T));
    char* base = a.scratch + (size_t)blockIdx.x * a.scratch_stride;
    CtaScratch<T> s;
    s.buf = reinterpret_cast<T*>(base + L.buf);
    s.cand = reinterpret_cast<int4*>(base + L.cand);
    s.clen = reinterpret_cast<int*>(base + L.clen);
    s.P = reinterpret_cast<T*>(base + L.P);
    s.TX = reinterpret_cast<T*>(base + L.TX);
    s.seg = reinterpret_cast<T*>(base + L.seg);
    s.cent = reinterpret_cast<EntRec<T>*>(base + L.cent);
    s.rec = reinterpret_cast<EntRec<T>*>(base + L.rec);
    s.cand_start = reinterpret_cast<int*>(base + L.cand_start);
    s.chunk_first = reinterpret_cast<int*>(base + L.chunk_first);
    s.row_n = reinterpret_cast<uint8_t*>(base + L.row_n);
    return s;
}

// Move the per-candidate tables of placement `mode` (NL_ALL or NL_HOT) into
// shared memory at p (at least nl_smem_bytes(mode, ...) bytes available).
template <typename T>
__device__ inline void nl_tables_in_smem(CtaScratch<T>& s, void* p_, int mode, int ccap, int S, int lb)
{
    char* p = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(p_) + 15) & ~uintptr_t(15));
    const NLSmem L = nl_smem_layout(mode, ccap, S, lb, sizeof(T));
    s.P = reinterpret_cast<T*>(p + L.P);
    s.TX = reinterpret_cast<T*>(p + L.TX);
    s.cand_start = reinterpret_cast<int*>(p + L.cand_start);
    s.chunk_first = reinterpret_cast<int*>(p + L.chunk_first);
    if (mode == NL_ALL) {
        s.cand = reinterpret_cast<int4*>(p + L.cand);
        s.seg = reinterpret_cast<T*>(p + L.seg);
        s.clen = reinterpret_cast<int*>(p + L.clen);
        s.row_n = reinterpret_cast<uint8_t*>(p + L.row_n);
    }
}

template <typename T>
__device__ inline EntRec<T> ld_rec(const EntRec<T>* p);
template <>
__device__ inline EntRec<float> ld_rec<float>(const EntRec<float>* p)
{
    float4 v = *reinterpret_cast<const float4*>(p);
    EntRec<float> r;
    r.meta = __float_as_uint(v.x);
    r.f0 = v.y;
    r.f1 = v.z;
    r.f2 = v.w;
    return r;
}
template <>
__device__ inline EntRec<double> ld_rec<double>(const EntRec<double>* p)
{
    double2 u = reinterpret_cast<const double2*>(p)[0], v = reinterpret_cast<const double2*>(p)[1];
    EntRec<double> r;
    r.meta = (uint32_t)__double_as_longlong(u.x);
    r.f0 = u.y;
    r.f1 = v.x;
    r.f2 = v.y;
    return r;
}
template <typename T>
__device__ inline void st_rec(EntRec<T>* p, uint32_t meta, T f0, T f1, T f2)
{
    p->meta = meta;
    p->f0 = f0;
    p->f1 = f1;
    p->f2 = f2;
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
// y/z Gaussian factors.  Both entry orders are fixed (rows ascending within
// a candidate; candidates ascending within a row), so every sum below has a
// fixed order and results are bitwise reproducible.  Returns the candidate
// count.
// ------------------------------------------------------------------------

// Clipped x-interval [xlo, xhi] (region columns) of box row (jj, kk) of a
// candidate whose box starts at region column bx; false if empty.
template <typename T, int M>
__device__ inline bool nl_row_interval(const NLParams<T>& nl, int atom, int bx, int jj, int kk, int& xlo, int& xhi)
{
    const uchar2 iv = *reinterpret_cast<const uchar2*>(nl.ivl + (((size_t)atom * nl.lb + jj) * nl.lb + kk) * 2);
    xlo = max((int)iv.x + bx, 0);
    xhi = min((int)iv.y + bx, Geo<M>::S - 1);
    return iv.x <= iv.y && xlo <= xhi;
}

template <typename T, int M>
__device__ int nl_setup(const RegionArgs<T>& a, const CtaScratch<T>& sc, int qi, int qj, int qk, int* red_i)
{
    using G = Geo<M>;
    const NLParams<T>& nl = a.nl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lb = nl.lb;
    const int lim = nl.smem ? nl.ccap : MAX_CAND;
    const int cap = G::S * G::S * ENTRIES_PER_ROW;
    int tile = (qi / TILE) + nl.ntile[0] * ((qj / TILE) + nl.ntile[1] * (qk / TILE));
    int beg = nl.tile_start[tile], end = nl.tile_start[tile + 1];
    // (1) candidates, ordered compaction of the tile list
    int ncand = 0;
    for (int c0 = beg; c0 < end; c0 += G::NT) {
        int c = c0 + tid;
        int keep = 0, ln = 0;
        int4 rec = make_int4(0, 0, 0, 0);
        if (c < end) {
            int4 tc = nl.tile_cand[c];
            AtomTab at = nl.atoms[tc.x];
            int bx = tc.y - (qi - M), by = tc.z - (qj - M), bz = tc.w - (qk - M);
            keep = (bx < G::S && bx + at.len[0] > 0 && by < G::S && by + at.len[1] > 0 &&
                    bz < G::S && bz + at.len[2] > 0);
            rec = make_int4(tc.x, bx, by, bz);
            ln = at.len[0] | (at.len[1] << 8) | (at.len[2] << 16);
        }
        int tot;
        int pos = block_excl_scan<G::NW>(keep, red_i, tot);
        if (keep) {
            if (ncand + pos < lim) {
                sc.cand[ncand + pos] = rec;
                sc.clen[ncand + pos] = ln;
            } else {
                atomicOr(a.err, ERR_CAPACITY);
            }
        }
        ncand += tot;
    }
    if (ncand > lim) ncand = lim;
    for (int c = tid; c <= ncand; c += G::NT) sc.cand_start[c] = 0;     // entry counts first
    __syncthreads();
    // (2) x-tables of the candidates by box column k (lb per candidate; zero
    // beyond the box)
    for (int i = tid; i < ncand * lb; i += G::NT) {
        const int c = i / lb, k = i % lb;
        T g = 0, dg = 0;
        if (k < (sc.clen[c] & 255)) {
            const int atom = sc.cand[c].x;
            g = nl.G[(size_t)atom * 3 * lb + k];
            dg = nl.DG[(size_t)atom * 3 * lb + k];
        }
        sc.TX[2 * i] = g;
        sc.TX[2 * i + 1] = dg;
    }
    // (3) row-ordered entries: thread (lane = y, warp = z) tests the
    // candidates in order for row (y, z); also counts every candidate's entries
    if (lane < G::S) {
        const int y = lane, z = warp;
        const int r = y + G::S * z;
        EntRec<T>* out = sc.rec + (size_t)r * ENTRIES_PER_ROW;
        int n = 0;
        for (int c = 0; c < ncand; ++c) {
            const int4 cr = sc.cand[c];
            const int ln = sc.clen[c];
            const int jj = y - cr.z, kk = z - cr.w;
            if (jj < 0 || jj >= ((ln >> 8) & 255) || kk < 0 || kk >= (ln >> 16)) continue;
            int xlo, xhi;
            if (!nl_row_interval<T, M>(nl, cr.x, cr.y, jj, kk, xlo, xhi)) continue;
            if (n < ENTRIES_PER_ROW) {
                const T* Gt = nl.G + (size_t)cr.x * 3 * lb;
                const T* Dt = nl.DG + (size_t)cr.x * 3 * lb;
                const T gy = Gt[lb + jj], dgy = Dt[lb + jj], gz = Gt[2 * lb + kk], dgz = Dt[2 * lb + kk];
                st_rec<T>(out + n, (uint32_t)c | ((uint32_t)xlo << 10) | ((uint32_t)xhi << 15) |
                                       ((uint32_t)(cr.y + 32) << 20), gy * gz, dgy * gz, gy * dgz);
            } else {
                atomicOr(a.err, ERR_CAPACITY);
            }
            ++n;
            atomicAdd(&sc.cand_start[c], 1);
        }
        sc.row_n[r] = (uint8_t)min(n, ENTRIES_PER_ROW);
    }
    __syncthreads();
    // (4) candidate offsets and chunk offsets (exclusive scans of the counts)
    {
        int run = 0, runk = 0;
        for (int c0 = 0; c0 < ncand; c0 += G::NT) {
            const int c = c0 + tid;
            const int v = (c < ncand) ? sc.cand_start[c] : 0;
            int tot, totk;
            const int off = block_excl_scan<G::NW>(v, red_i, tot);
            const int offk = block_excl_scan<G::NW>((v + 31) >> 5, red_i, totk);
            if (c < ncand) {
                sc.cand_start[c] = min(run + off, cap);
                sc.chunk_first[c] = runk + offk;
            }
            run += tot;
            runk += totk;
        }
        if (tid == 0) {
            if (run > cap) atomicOr(a.err, ERR_CAPACITY);
            sc.cand_start[ncand] = min(run, cap);
            sc.chunk_first[ncand] = runk;
        }
    }
    __syncthreads();
    // (5) candidate-ordered entries: warp per candidate, its box rows clipped
    // to the region in ascending r, compacted with a ballot
    for (int c = warp; c < ncand; c += G::NW) {
        const int4 cr = sc.cand[c];
        const int ln = sc.clen[c];
        const T* Gt = nl.G + (size_t)cr.x * 3 * lb;
        const T* Dt = nl.DG + (size_t)cr.x * 3 * lb;
        const int j0 = max(0, -cr.z), j1 = min((ln >> 8) & 255, G::S - cr.z);
        const int k0 = max(0, -cr.w), k1 = min(ln >> 16, G::S - cr.w);
        const int nj = j1 - j0;
        const int nrows = (nj > 0 && k1 > k0) ? nj * (k1 - k0) : 0;
        const int cbase = sc.cand_start[c], cend = sc.cand_start[c + 1];
        int cnt = 0;
        for (int r0 = 0; r0 < nrows; r0 += 32) {
            const int rr = r0 + lane;
            int ok = 0, xlo = 0, xhi = 0, jj = 0, kk = 0;
            if (rr < nrows) {
                jj = j0 + rr % nj;
                kk = k0 + rr / nj;
                ok = nl_row_interval<T, M>(nl, cr.x, cr.y, jj, kk, xlo, xhi);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const int ce = cbase + cnt + __popc(bal & ((1u << lane) - 1u));
                if (ce < cend) {
                    const int row = (cr.z + jj) + G::S * (cr.w + kk);
                    const T gy = Gt[lb + jj], dgy = Dt[lb + jj], gz = Gt[2 * lb + kk], dgz = Dt[2 * lb + kk];
                    st_rec<T>(sc.cent + ce, (uint32_t)row | ((uint32_t)xlo << 10) | ((uint32_t)xhi << 15) |
                                                ((uint32_t)(cr.y + 32) << 20), gy * gz, dgy * gz, gy * dgz);
                }
            }
            cnt += __popc(bal);
        }
    }
    __syncthreads();
    return ncand;
}

// Projector inner products of the shared-memory vector (trapezoidal rule,
// Eq. IntApprox, without the h^3 which sits in cs/cp):
//   S_c = sum G t, X_c = sum D_x G t, Y_c = sum D_y G t, Z_c = sum D_z G t
// over the support of candidate c inside the region.  The Gaussian factorises
// per axis: each row is reduced along x with the candidate's x-profile, then
// weighted by the row's y/z factors.  The candidate-ordered entries are cut
// into chunks of 32 (one entry per lane) and each warp takes a contiguous run
// of chunks, so the warps carry equal work whatever the candidates' sizes;
// the next chunk's records are fetched while the current one is reduced.  A
// warp's partial sums for candidate c go to seg[c + warp] -- distinct for
// every (candidate, warp) pair that occurs, because both rise along the chunk
// order -- and nl_collect adds them in warp order, so the order is fixed.
constexpr int LBMAX = 20;    // unrolled box width (longer boxes take the plain loop)

template <typename T>
struct Pair2;
template <> struct Pair2<float> { using type = float2; };
template <> struct Pair2<double> { using type = double2; };

template <typename T, int M>
__device__ void nl_dots(const RegionArgs<T>& a, const CtaScratch<T>& sc, const T* cur, int ncand)
{
    using G = Geo<M>;
    using P2 = typename Pair2<T>::type;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int K = sc.chunk_first[ncand];
    const int Q = (K + G::NW - 1) / G::NW;
    const int j0 = warp * Q, j1 = min(K, j0 + Q);
    if (j0 >= j1) return;
    int lo = 0, hi = ncand - 1;                       // last candidate with chunk_first <= j0
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sc.chunk_first[mid] <= j0) lo = mid;
        else hi = mid - 1;
    }
    const int lb = a.nl.lb;
    const bool unrolled = lb <= LBMAX;
    // records of chunks j+1 and j+2 are in flight while chunk j is reduced
    auto fetch = [&](int j, int c, EntRec<T>& r, bool& v) {
        const int e = sc.cand_start[c] + (j - sc.chunk_first[c]) * 32 + lane;
        v = e < sc.cand_start[c + 1];
        if (v) r = ld_rec(sc.cent + e);
    };
    EntRec<T> rA, rB;
    rA.meta = rB.meta = 0;
    rA.f0 = rA.f1 = rA.f2 = rB.f0 = rB.f1 = rB.f2 = 0;
    bool vA = false, vB = false;
    int cA = lo, cB = lo;
    fetch(j0, cA, rA, vA);
    if (j0 + 1 < j1) {
        while (j0 + 1 >= sc.chunk_first[cB + 1]) ++cB;
        fetch(j0 + 1, cB, rB, vB);
    }
    T aS = 0, aX = 0, aY = 0, aZ = 0;
    for (int j = j0; j < j1; ++j) {
        const EntRec<T> rc = rA;
        const bool val = vA;
        const int c = cA;
        rA = rB;
        vA = vB;
        cA = cB;
        if (j + 2 < j1) {
            while (j + 2 >= sc.chunk_first[cB + 1]) ++cB;
            fetch(j + 2, cB, rB, vB);
        }
        if (val) {
            const int r = rc.meta & 1023u, xlo = (rc.meta >> 10) & 31u, xhi = (rc.meta >> 15) & 31u;
            const int bx = (int)((rc.meta >> 20) & 63u) - 32;
            const int y = r % G::S, z = r / G::S;
            const T* row = cur + G::LEAD + z * G::PLANE + y * G::PX;
            // slots k of the candidate's box, x = bx + k: every lane of the
            // chunk reads the same (G, DG) pair, and rows of one plane sit in
            // distinct banks
            const P2* txp = reinterpret_cast<const P2*>(sc.TX) + (size_t)c * lb;
            const T* rowp = row + bx;
            T u = 0, u2 = 0;
            if (unrolled) {
                const uint32_t mask = ((2u << (xhi - bx)) - 1u) & ~((1u << (xlo - bx)) - 1u);
#pragma unroll
                for (int k = 0; k < LBMAX; ++k)
                    if (mask & (1u << k)) {
                        const P2 g = txp[k];
                        const T tv = rowp[k];
                        u += g.x * tv;
                        u2 += g.y * tv;
                    }
            } else {
                for (int k = xlo - bx; k <= xhi - bx; ++k) {
                    const P2 g = txp[k];
                    const T tv = rowp[k];
                    u += g.x * tv;
                    u2 += g.y * tv;
                }
            }
            aS += rc.f0 * u;
            aX += rc.f0 * u2;
            aY += rc.f1 * u;
            aZ += rc.f2 * u;
        }
        if (j + 1 >= j1 || cA != c) {                 // warp-uniform: candidate done in this warp
            aS = warp_sumT<T>(aS);                    // xor tree: every lane holds the totals
            aX = warp_sumT<T>(aX);
            aY = warp_sumT<T>(aY);
            aZ = warp_sumT<T>(aZ);
            if (lane == 0) {
                T* sg = sc.seg + (size_t)(c + warp) * 4;
                sg[0] = aS;
                sg[1] = aX;
                sg[2] = aY;
                sg[3] = aZ;
            }
            aS = aX = aY = aZ = 0;
        }
    }
}

// P_c = sum over the warps that reduced part of candidate c of their partial
// sums, in warp order.
template <typename T, int M>
__device__ void nl_collect(const CtaScratch<T>& sc, int ncand)
{
    using G = Geo<M>;
    const int K = sc.chunk_first[ncand];
    const int Q = (K + G::NW - 1) / G::NW;
    for (int c = threadIdx.x; c < ncand; c += G::NT) {
        T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
        const int f0 = sc.chunk_first[c], f1 = sc.chunk_first[c + 1];
        if (f1 > f0)
            for (int w = f0 / Q; w <= (f1 - 1) / Q; ++w) {
                const T* sg = sc.seg + (size_t)(c + w) * 4;
                s0 += sg[0];
                s1 += sg[1];
                s2 += sg[2];
                s3 += sg[3];
            }
        sc.P[4 * c + 0] = s0;
        sc.P[4 * c + 1] = s1;
        sc.P[4 * c + 2] = s2;
        sc.P[4 * c + 3] = s3;
    }
}

// The four inner products of candidate c (one 16-byte load in FP32).
template <typename T>
__device__ inline void load_P(const T* P, int c, T& pS, T& pX, T& pY, T& pZ);
template <>
__device__ inline void load_P<float>(const float* P, int c, float& pS, float& pX, float& pY, float& pZ)
{
    const float4 v = reinterpret_cast<const float4*>(P)[c];
    pS = v.x;
    pX = v.y;
    pY = v.z;
    pZ = v.w;
}
template <>
__device__ inline void load_P<double>(const double* P, int c, double& pS, double& pX, double& pY, double& pZ)
{
    const double2 u = reinterpret_cast<const double2*>(P)[2 * c], v = reinterpret_cast<const double2*>(P)[2 * c + 1];
    pS = u.x;
    pX = u.y;
    pY = v.x;
    pZ = v.y;
}

// sec <- sec - coef * V_nl t, candidate-ordered per point (FP64; the FP32
// form uses nl_update_red below).  Thread (lane = y, warp = z) owns
// region row (y, z) and walks its entries (candidates ascending); the lanes
// of a warp take their k-th entries together, and each entry's x-interval is
// covered by predicated slots, loads first and stores after, so every entry
// costs a fixed, overlapped instruction sequence.  Per entry
//   b0 = coef (cs f0 S_c + cp (f1 Y_c + f2 Z_c)),  b1 = coef cp f0 X_c,
// and each point of the interval gets  -= G_x b0 + DG_x b1.  The lanes own
// neighbouring rows of one plane, whose candidates and intervals nearly
// coincide, so their shared-memory accesses spread over distinct banks.
template <typename T, int M, bool DB>
__device__ void nl_update(const RegionArgs<T>& a, const CtaScratch<T>& sc, T* sec, T coef)
{
    using G = Geo<M>;
    using P2 = typename Pair2<T>::type;
    constexpr int GRP = sizeof(T) == 4 ? 5 : 4;       // slots loaded together (divides LBMAX)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool own = lane < G::S;
    const int r = (own ? lane : 0) + G::S * warp;
    T* brow = Sec<M, DB>::row(sec, own ? lane : 0, warp);
    const int n = own ? sc.row_n[r] : 0;
    const int nmax = __reduce_max_sync(0xffffffffu, (unsigned)n);
    if (nmax == 0) return;
    const bool unrolled = a.nl.lb <= LBMAX;
    const T cs = a.nl.cs * coef, cp = a.nl.cp * coef;
    const P2* tx2 = reinterpret_cast<const P2*>(sc.TX);
    const EntRec<T>* rrow = sc.rec + (size_t)r * ENTRIES_PER_ROW;
    EntRec<T> r0, r1;
    r0.meta = r1.meta = 0;
    r0.f0 = r0.f1 = r0.f2 = r1.f0 = r1.f1 = r1.f2 = 0;
    if (n > 0) r0 = ld_rec(rrow);
    if (n > 1) r1 = ld_rec(rrow + 1);
    for (int k = 0; k < nmax; ++k) {
        const EntRec<T> rc = r0;
        r0 = r1;
        if (k + 2 < n) r1 = ld_rec(rrow + k + 2);
        if (k >= n) continue;
        const int c = rc.meta & 1023u, xlo = (rc.meta >> 10) & 31u, xhi = (rc.meta >> 15) & 31u;
        const int bx = (int)((rc.meta >> 20) & 63u) - 32;
        T pS, pX, pY, pZ;
        load_P<T>(sc.P, c, pS, pX, pY, pZ);
        const T b0 = cs * rc.f0 * pS + cp * (rc.f1 * pY + rc.f2 * pZ);
        const T b1 = cp * rc.f0 * pX;
        const P2* tx = tx2 + (size_t)c * a.nl.lb + (xlo - bx);
        T* bp = brow + xlo;
        const int len = xhi - xlo;                    // slots 0..len
        bool done = false;
        if constexpr (sizeof(T) == 4) {               // FP64 takes the plain loop: registers matter more there
            if (unrolled) {
#pragma unroll
                for (int h = 0; h < LBMAX / GRP; ++h) {
                    if (h * GRP > len) break;
                    P2 g[GRP];
                    T v[GRP];
#pragma unroll
                    for (int s = 0; s < GRP; ++s)
                        if (h * GRP + s <= len) {
                            g[s] = tx[h * GRP + s];
                            v[s] = bp[h * GRP + s];
                        }
#pragma unroll
                    for (int s = 0; s < GRP; ++s)
                        if (h * GRP + s <= len) bp[h * GRP + s] = v[s] - (g[s].x * b0 + g[s].y * b1);
                }
                done = true;
            }
        }
        if (!done) {
            for (int s = 0; s <= len; ++s) {
                const P2 g = tx[s];
                bp[s] -= g.x * b0 + g.y * b1;
            }
        }
    }
}

// sec <- sec - coef * V_nl t for the FP32 form: the update walks the
// candidate-ordered entries exactly like nl_dots (equal runs of 32-entry
// chunks per warp, one entry per lane, slots from the candidate's box start,
// records two chunks ahead), and adds each point's contribution with a
// shared-memory atomic add.  Lanes of a chunk own distinct rows; points
// covered by several candidates receive their contributions in an order
// that varies from run to run, so this form is reproducible to FP32
// rounding rather than bitwise (the FP64 form keeps the fixed order).
template <typename T, int M, bool DB>
__device__ void nl_update_red(const RegionArgs<T>& a, const CtaScratch<T>& sc, T* sec, int ncand, T coef)
{
    using G = Geo<M>;
    using P2 = typename Pair2<T>::type;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int K = sc.chunk_first[ncand];
    const int Q = (K + G::NW - 1) / G::NW;
    const int j0 = warp * Q, j1 = min(K, j0 + Q);
    if (j0 >= j1) return;
    int lo = 0, hi = ncand - 1;                       // last candidate with chunk_first <= j0
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sc.chunk_first[mid] <= j0) lo = mid;
        else hi = mid - 1;
    }
    const int lb = a.nl.lb;
    const bool unrolled = lb <= LBMAX;
    const T cs = a.nl.cs * coef, cp = a.nl.cp * coef;
    auto fetch = [&](int j, int c, EntRec<T>& r, bool& v) {
        const int e = sc.cand_start[c] + (j - sc.chunk_first[c]) * 32 + lane;
        v = e < sc.cand_start[c + 1];
        if (v) r = ld_rec(sc.cent + e);
    };
    EntRec<T> rA, rB;
    rA.meta = rB.meta = 0;
    rA.f0 = rA.f1 = rA.f2 = rB.f0 = rB.f1 = rB.f2 = 0;
    bool vA = false, vB = false;
    int cA = lo, cB = lo;
    fetch(j0, cA, rA, vA);
    if (j0 + 1 < j1) {
        while (j0 + 1 >= sc.chunk_first[cB + 1]) ++cB;
        fetch(j0 + 1, cB, rB, vB);
    }
    for (int j = j0; j < j1; ++j) {
        const EntRec<T> rc = rA;
        const bool val = vA;
        const int c = cA;
        rA = rB;
        vA = vB;
        cA = cB;
        if (j + 2 < j1) {
            while (j + 2 >= sc.chunk_first[cB + 1]) ++cB;
            fetch(j + 2, cB, rB, vB);
        }
        if (!val) continue;
        const int r = rc.meta & 1023u, xlo = (rc.meta >> 10) & 31u, xhi = (rc.meta >> 15) & 31u;
        const int bx = (int)((rc.meta >> 20) & 63u) - 32;
        T pS, pX, pY, pZ;
        load_P<T>(sc.P, c, pS, pX, pY, pZ);
        const T b0 = cs * rc.f0 * pS + cp * (rc.f1 * pY + rc.f2 * pZ);
        const T b1 = cp * rc.f0 * pX;
        T* rowp = Sec<M, DB>::row(sec, r % G::S, r / G::S) + bx;
        const P2* txp = reinterpret_cast<const P2*>(sc.TX) + (size_t)c * lb;
        if (unrolled) {
            const uint32_t mask = ((2u << (xhi - bx)) - 1u) & ~((1u << (xlo - bx)) - 1u);
#pragma unroll
            for (int k = 0; k < LBMAX; ++k)
                if (mask & (1u << k)) {
                    const P2 g = txp[k];
                    const T d = -(g.x * b0 + g.y * b1);
                    if constexpr (DB) {
                        const unsigned addr = (unsigned)__cvta_generic_to_shared(rowp + k);
                        asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(addr), "f"(d) : "memory");
                    } else {
                        atomicAdd(rowp + k, d);
                    }
                }
        } else {
            for (int k = xlo - bx; k <= xhi - bx; ++k) {
                const P2 g = txp[k];
                atomicAdd(rowp + k, -(g.x * b0 + g.y * b1));
            }
        }
    }
}

// ------------------------------------------------------------------------
// Stencil sweep of H (local part, Eq. FD:Laplacian + V):
//   out(p) = s * [ (-3 w_0 + V(p) - shift) t(p) - 1/2 sum_d w_d (6 nbrs at d) ] - sec(p)
// (the projector term, when present, has already been folded into sec by
// the projector update)
// RECUR = true (Chebyshev step): out = t^{i+1} and sec holds t^{i-1}.
//   DB:  out replaces t^{i-1} in sec (pointwise, no barrier); the caller
//        swaps the two buffers after the sweep.
//   !DB: out replaces t^i in shared memory plane by plane (one barrier per
//        plane keeps the neighbours of the next plane intact) and t^i goes
//        to sec, which becomes t^{i-1}.
//   The thread accumulates out.out and out.t^i over its column.
// RECUR = false (Lanczos): out = w goes to sec; t is left in place; the
//   thread accumulates out.out, out.t and t.t.
// ------------------------------------------------------------------------
// ACCD (recurrence only): also D += cd * t^{i+1} at every point, D being an
// unpadded S^3 array (x fastest) that only the point's own thread touches.
template <typename T, int M, bool RECUR, bool DB, bool YEDGE = false, bool ACCD = false>
__device__ void stencil_sweep(const RegionArgs<T>& a, T* cur, T* sec, const T* vwin, T s, T dshift,
                              T& acc_a, T& acc_b, T& acc_c, double* centre_out, T* D = nullptr, T cd = T(0))
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
    // the potential comes from global memory: keep VD planes in flight
    constexpr int VD = 4;
    T vq[VD];
#pragma unroll
    for (int d = 0; d < VD; ++d) vq[d] = (active && d < G::S) ? vcol[d * vplane] : T(0);
    T aa = 0, ab = 0, ac = 0;
#pragma unroll
    for (int z = 0; z < G::S; ++z) {
        T out = 0;
        const T c = q[6];
        const T vz = vq[z % VD];
        if (z + VD < G::S) vq[z % VD] = active ? vcol[(z + VD) * vplane] : T(0);
        if (active) {
            const T* p = col + z * G::PLANE;
            T lap = 0;
#pragma unroll
            for (int d = 1; d <= FD_NO; ++d) {
                T xp = p[d], xm = p[-d];
                if constexpr (G::CY) {                 // beyond the zero columns: the next/previous row
                    if (d > G::PX - G::S) {
                        if (x + d >= G::S) xp = T(0);
                        if (x < d) xm = T(0);
                    }
                }
                T yp, ym;
                if constexpr (G::CY && YEDGE) {        // no zero rows: outside the region is zero
                    yp = (y + d < G::S) ? p[d * G::PX] : T(0);
                    ym = (y >= d) ? p[-d * G::PX] : T(0);
                } else {
                    yp = p[d * G::PX];
                    ym = p[-d * G::PX];
                }
                T nb = (xp + xm) + (yp + ym) + (q[6 + d] + q[6 - d]);
                lap += a.wd[d] * nb;
            }
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
                if (x == M && y == M && z == M) *centre_out = (double)out;
                if constexpr (ACCD) D[((size_t)z * G::S + y) * G::S + x] += cd * out;
            } else {
                bcol[z * SV::ZS] = out;
                aa += out * out;
                ab += out * c;
                ac += c * c;
            }
        }
#pragma unroll
        for (int d = 0; d < 12; ++d) q[d] = q[d + 1];
        q[12] = (active && z + 7 < G::S) ? col[(z + 7) * G::PLANE] : T(0);
    }
    acc_a = aa;
    acc_b = ab;
    acc_c = ac;
}

// ------------------------------------------------------------------------
// Chebyshev moments kernel (Section 3.2, Eqs. Rec:FD and rhoqj).
// ------------------------------------------------------------------------
template <typename T, int M, bool DB>
__device__ void moments_node(const RegionArgs<T>& a, unsigned char* smem_raw, long long node)
{
    using G = Geo<M>;
    // the compact form picks its sweep per warp, which is only legal without
    // the per-plane barriers of the single-buffer sweep
    static_assert(!G::CY || DB, "compact regions must keep both vectors in shared memory");
    T* bufA = reinterpret_cast<T*>(smem_raw);
    __shared__ double red[2][2][32];          // [step parity][d2, d1][warp]
    __shared__ int red_i[33];
    // after the region vectors: rho^i and the two product sums (npl/2 + 2 each), then the projector tables
    double* s_mom = reinterpret_cast<double*>(smem_raw + align16(region_smem<T, M>()));
    double* s_d2 = s_mom + (a.npl / 2 + 2);
    double* s_d1 = s_d2 + (a.npl / 2 + 2);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    CtaScratch<T> sc = cta_scratch(a, M);
    if (a.nl.smem) nl_tables_in_smem(sc, s_d1 + (a.npl / 2 + 2), a.nl.smem, a.nl.ccap, G::S, a.nl.lb);
    T* bufB = DB ? bufA + G::ELEMS : sc.buf;
    const int half = a.npl / 2;
    const bool has_nl = a.nl.n_atoms > 0;

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
            nl_collect<T, M>(sc, ncand);
            __syncthreads();
            if constexpr (sizeof(T) == 4) nl_update_red<T, M, DB>(a, sc, sec, ncand, s);
            else nl_update<T, M, DB>(a, sc, sec, s);
            __syncthreads();
        }
        T aa, ab, unused;
        if (G::CY && (warp < FD_NO || warp >= G::S - FD_NO))   // warp-uniform
            stencil_sweep<T, M, true, DB, true>(a, cur, sec, vwin, s, dshift, aa, ab, unused, &s_mom[i + 1]);
        else
            stencil_sweep<T, M, true, DB, false>(a, cur, sec, vwin, s, dshift, aa, ab, unused, &s_mom[i + 1]);
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

template <typename T, int M, bool DB>
__global__ void __launch_bounds__(Geo<M>::NT, (region_min_blocks<T, M>()))
moments_kernel(RegionArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (long long node = blockIdx.x; node < a.g.Nd; node += gridDim.x) moments_node<T, M, DB>(a, smem_raw, node);
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
__device__ void lanczos_node(const RegionArgs<T>& a, unsigned char* smem_raw, long long node)
{
    using G = Geo<M>;
    static_assert(!G::CY || DB, "compact regions must keep both vectors in shared memory");
    using SV = Sec<M, DB>;
    T* sm = reinterpret_cast<T*>(smem_raw);
    __shared__ double red_a[32], red_b[32], red_c[32];  // v.w, w.w and v.v partials
    __shared__ int red_i[33];
    __shared__ T s_alpha, s_inv, s_bprev;
    __shared__ int s_stop, s_explicit;
    __shared__ double s_dummy;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x = lane, y = warp;
    const bool active = x < G::S;
    CtaScratch<T> sc = cta_scratch(a, M);
    if (a.nl.smem) nl_tables_in_smem(sc, smem_raw + region_smem<T, M>(), a.nl.smem, a.nl.ccap, G::S, a.nl.lb);
    T* sec = DB ? sm + G::ELEMS : sc.buf;
    const bool has_nl = a.nl.n_atoms > 0;
    const T dshift = (T)(-3.0 * a.g.w[0]);
    const T v0 = (T)(1.0 / sqrt((double)G::NS));

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
    for (int it = 0; it < a.n_lanczos; ++it) {
        // w = H v - beta_prev v_old  (sec holds beta_prev v_old, then w)
        if (has_nl) {
            nl_dots<T, M>(a, sc, sm, ncand);
            __syncthreads();
            nl_collect<T, M>(sc, ncand);
            __syncthreads();
            if constexpr (sizeof(T) == 4) nl_update_red<T, M, DB>(a, sc, sec, ncand, T(1));
            else nl_update<T, M, DB>(a, sc, sec, T(1));
            __syncthreads();
        }
        T ww, vw, vv;
        if (G::CY && (warp < FD_NO || warp >= G::S - FD_NO))   // warp-uniform
            stencil_sweep<T, M, false, DB, true>(a, sm, sec, vwin, T(1), dshift, ww, vw, vv, &s_dummy);
        else
            stencil_sweep<T, M, false, DB, false>(a, sm, sec, vwin, T(1), dshift, ww, vw, vv, &s_dummy);
        // alpha = v.w and beta^2 = |w - alpha v|^2 = w.w - 2 alpha v.w + alpha^2 v.v from the
        // sweep's sums, which saves a pass over w; where that difference cancels (beta below a
        // tenth of |w|: near breakdown, e.g. tiny regions) beta is taken from w - alpha v itself
        const double wa = warp_total(vw), wb = warp_total(ww), wc = warp_total(vv);
        if (lane == 0) {
            red_a[warp] = wa;
            red_b[warp] = wb;
            red_c[warp] = wc;
        }
        __syncthreads();
        if (tid == 0) {
            double al = 0.0, w2 = 0.0, v2 = 0.0;
            for (int w = 0; w < G::NW; ++w) {
                al += red_a[w];
                w2 += red_b[w];
                v2 += red_c[w];
            }
            alpha[it] = al;
            if (fabs(al) + bprev > scale) scale = fabs(al) + bprev;
            const double b2 = w2 - 2.0 * al * al + al * al * v2;
            s_alpha = (T)al;
            s_explicit = !(b2 > 0.01 * w2);
            if (!s_explicit) {
                const double b = sqrt(b2);
                const int stop = (it == a.n_lanczos - 1) || (b <= 1e-10 * scale);
                if (!stop) beta[it] = b;
                else a.klen[node] = it + 1;
                s_stop = stop;
                s_inv = (T)(1.0 / b);
                s_bprev = (T)b;
                bprev = b;
            }
        }
        __syncthreads();
        const T alT = s_alpha;
        if (s_explicit) {                              // block-uniform
            // w -= alpha v ; beta = |w|
            T acc = 0;
            if (active)
                for (int z = 0; z < G::S; ++z) {
                    T w = bcol[z * SV::ZS] - alT * col[z * G::PLANE];
                    bcol[z * SV::ZS] = w;
                    acc += w * w;
                }
            const double wt = warp_total(acc);
            if (lane == 0) red_b[warp] = wt;
            __syncthreads();
            if (tid == 0) {
                double b2 = 0.0;
                for (int w = 0; w < G::NW; ++w) b2 += red_b[w];
                const double b = sqrt(b2);
                const int stop = (it == a.n_lanczos - 1) || (b <= 1e-10 * scale);
                if (!stop) beta[it] = b;
                else a.klen[node] = it + 1;
                s_stop = stop;
                s_inv = (T)(1.0 / b);
                s_bprev = (T)b;
                bprev = b;
            }
            __syncthreads();
            if (s_stop) break;
            // sec <- beta v (the next step's beta_prev v_old), v <- w / beta
            const T inv = s_inv, bT = s_bprev;
            if (active)
                for (int z = 0; z < G::S; ++z) {
                    T w = bcol[z * SV::ZS];
                    T v = col[z * G::PLANE];
                    bcol[z * SV::ZS] = bT * v;
                    col[z * G::PLANE] = w * inv;
                }
        } else {
            if (s_stop) break;
            // sec <- beta v, v <- (w - alpha v) / beta
            const T inv = s_inv, bT = s_bprev;
            if (active)
                for (int z = 0; z < G::S; ++z) {
                    T w = bcol[z * SV::ZS];
                    T v = col[z * G::PLANE];
                    bcol[z * SV::ZS] = bT * v;
                    col[z * G::PLANE] = (w - alT * v) * inv;
                }
        }
        __syncthreads();
    }
    __syncthreads();
}

template <typename T, int M, bool DB>
__global__ void __launch_bounds__(Geo<M>::NT, (region_min_blocks<T, M>()))
lanczos_kernel(RegionArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (long long node = blockIdx.x; node < a.g.Nd; node += gridDim.x) lanczos_node<T, M, DB>(a, smem_raw, node);
}

}  // namespace sq
