// sq_cnn_tc.cuh -- the warm-start network's 32 -> 32-channel 3^3 convolution
// (the middle layer) as an implicit GEMM on the fifth-generation tensor cores
// (tcgen05), bfloat16 operands, FP32 accumulation in tensor memory (TMEM):
//
//   z2[p][o] = b2[o] + sum_{d < 27} sum_{i < 32} W2[d][i][o] a1[p + d][i],  a2 = silu(z2)
//
// GEMM view per tile of 128 nodes: D (128 x 32) = A (128 x 864) B (864 x 32),
// row m of A = the 27 neighbour rows of node p_m (32 channels each, periodic
// wrap), B = W2 with k = d * 32 + i.  Per tap d the kernel gathers A_d (128 x
// 32 bfloat16, 8 KB) into shared memory and one thread issues two
// tcgen05.mma (M = 128, N = 32, K = 16); the accumulator (128 lanes x 32
// FP32 columns) stays in TMEM over the 27 taps and four warps read it back
// with tcgen05.ld for the epilogue (bias, SiLU, stores).  The weights (27 x
// 32 x 32 bfloat16) are staged once per CTA; A_d uses a two-stage ring, so
// gathering tap d+1 overlaps the MMAs of tap d; each stage has an mbarrier
// that tcgen05.commit arrives on when its MMAs complete.
//
// Operand layout (shared memory, no swizzle, K-major): 8 x 8 "core
// matrices" of 8 rows x 16 bytes stored contiguously; core matrices
// adjacent along K are LBO = 128 bytes apart, 8-row groups SBO = 512 bytes
// apart (32 channels = 4 core matrices per row group).  The second K-half of
// a tap starts 256 bytes in.
//
// Every wait on an mbarrier has an iteration limit; on expiry the kernel
// latches an error bit, stops issuing, waits (with a limit) for what it
// issued, frees its TMEM columns and returns.
#pragma once
#include "sq_cnn.cuh"

namespace sq {

constexpr int TC_M = 128;                    // nodes per tile (MMA M)
constexpr int TC_TAPS = 27;
constexpr int TC_ABYTES = TC_M * CNN_C * 2;  // one tap of A: 8 KB
constexpr int TC_BBYTES = CNN_C * CNN_C * 2; // one tap of B: 2 KB
constexpr unsigned TC_ERR_TIMEOUT = 1u;
constexpr long long TC_WAIT_LIMIT = 1ll << 26;   // mbarrier polls before giving up

// shared memory: B (27 taps), A ring (2 stages), mbarriers, TMEM address
constexpr int TC_SMEM = TC_TAPS * TC_BBYTES + 2 * TC_ABYTES + 64;

__device__ __forceinline__ uint32_t tc_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4 (16-29),
// SBO >> 4 (32-45), descriptor version 1 (46-47), no swizzle (61-63 = 0).
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1),
// A and B bfloat16 (7-9 = 1, 10-12 = 1), both K-major, N >> 3 (17-22),
// M >> 4 (24-28).
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(CNN_C >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ void tc_mbar_init(uint32_t mbar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
}

// Wait for phase `parity` of the mbarrier, at most TC_WAIT_LIMIT polls;
// false on expiry.
__device__ __forceinline__ bool tc_mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (long long i = 0; i < TC_WAIT_LIMIT; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(TC_IDESC), "r"(accumulate) : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// z2 and a2 of one layer: the forward of conv3(32 -> 32) + bias + SiLU on
// tensor cores.  128 threads (4 warps) per CTA, persistent over tiles.
__global__ void __launch_bounds__(128, 1) cnn_conv2_tc_kernel(CnnGrid g, const Bf16* __restrict__ x,
                                                             const Bf16* __restrict__ W,
                                                             const float* __restrict__ b,
                                                             float* __restrict__ z, Bf16* __restrict__ a,
                                                             unsigned* __restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char* sB = tc_smem;                                  // 27 x 2 KB
    unsigned char* sA = tc_smem + TC_TAPS * TC_BBYTES;            // 2 x 8 KB
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sA + 2 * TC_ABYTES);
    uint32_t* s_taddr = reinterpret_cast<uint32_t*>(mbar + 2);
    const int tid = threadIdx.x, warp = tid >> 5;

    // B: element (n = o, k = i) of tap d at core matrix (n / 8, i / 8), row n % 8, column i % 8
    for (int e = tid; e < TC_TAPS * CNN_C * CNN_C; e += 128) {
        const int d = e / (CNN_C * CNN_C), i = (e / CNN_C) % CNN_C, o = e % CNN_C;
        const int off = d * TC_BBYTES + ((o >> 3) * 4 + (i >> 3)) * 128 + (o & 7) * 16 + (i & 7) * 2;
        *reinterpret_cast<uint16_t*>(sB + off) = W[e].u;
    }
    if (tid == 0) {
        tc_mbar_init(tc_smem_u32(&mbar[0]));
        tc_mbar_init(tc_smem_u32(&mbar[1]));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {                                               // 32 TMEM columns: the 128 x 32 accumulator
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(tc_smem_u32(s_taddr))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // B visible to the tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = *s_taddr;
    const uint32_t sA0 = tc_smem_u32(sA), sB0 = tc_smem_u32(sB);
    uint32_t phase[2] = {0u, 0u};
    int pending[2] = {0, 0};                                       // commits not yet waited for, per stage
    bool ok = true;

    const long long ntiles = (g.N + TC_M - 1) / TC_M;
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const long long p = tile * TC_M + tid;                     // thread = row of A = node
        const bool valid = p < g.N;
        int pi = 0, pj = 0, pk = 0;
        if (valid) cnn_ijk(g, p, pi, pj, pk);
        for (int d = 0; d < TC_TAPS; ++d) {
            const int s = d & 1;
            if (pending[s]) {                                      // MMAs of tap d - 2 have read this stage
                if (tid == 0) ok = tc_mbar_wait(tc_smem_u32(&mbar[s]), phase[s]);
                ok = __syncthreads_and(ok);
                phase[s] ^= 1u;
                pending[s] = 0;
                if (!ok) break;
            }
            const int dz = d / 9 - 1, dy = (d / 3) % 3 - 1, dx = d % 3 - 1;
            uint4 v[4] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
            if (valid) {
                const uint4* src = reinterpret_cast<const uint4*>(x + cnn_nb(g, pi, pj, pk, dx, dy, dz) * CNN_C);
#pragma unroll
                for (int c = 0; c < 4; ++c) v[c] = src[c];
            }
            unsigned char* dst = sA + s * TC_ABYTES + (tid >> 3) * 512 + (tid & 7) * 16;
#pragma unroll
            for (int c = 0; c < 4; ++c) *reinterpret_cast<uint4*>(dst + c * 128) = v[c];   // core matrix (row/8, c)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = sA0 + s * TC_ABYTES, b0 = sB0 + d * TC_BBYTES;
                tc_mma(taddr, tc_desc(a0, 128, 512), tc_desc(b0, 128, 512), d > 0 ? 1u : 0u);
                tc_mma(taddr, tc_desc(a0 + 256, 128, 512), tc_desc(b0 + 256, 128, 512), 1u);
                tc_commit(tc_smem_u32(&mbar[s]));
            }
            pending[s] = 1;
        }
        // wait for the last two commits (taps 25 and 26), then read the accumulator
        for (int s = 0; s < 2 && ok; ++s)
            if (pending[s]) {
                if (tid == 0) ok = tc_mbar_wait(tc_smem_u32(&mbar[s]), phase[s]);
                ok = __syncthreads_and(ok);
                phase[s] ^= 1u;
                pending[s] = 0;
            }
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t r[32];
        const uint32_t ta = taddr + ((uint32_t)(warp * 32) << 16);   // lanes 32 warp .. 32 warp + 31
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
              "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (valid) {
#pragma unroll
            for (int o = 0; o < CNN_C; ++o) {
                const float zz = __uint_as_float(r[o]) + b[o];
                z[p * CNN_C + o] = zz;
                stv(a[p * CNN_C + o], cnn_silu(zz));
            }
        }
        // every warp has read the accumulator before the next tile's first MMA overwrites it
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (!ok) {
        if (tid == 0) atomicOr(err, TC_ERR_TIMEOUT);
        for (int s = 0; s < 2; ++s)                                // what was issued, with a limit too
            if (pending[s] && tid == 0) tc_mbar_wait(tc_smem_u32(&mbar[s]), phase[s]);
        __syncthreads();
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(taddr) : "memory");
}

}  // namespace sq
