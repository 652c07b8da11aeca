// sq_queue.cuh -- persistent region kernels fed from a device work queue, for
// a batch of systems that share one region half-width m (the batched launch
// of uneven systems; the paper treats one system at a time).
//
// The grid is one wave of resident CTAs.  Each CTA takes the next item of a
// host-built list with one atomic add on a counter and runs it; it stops when
// the list is exhausted, so systems of different size, degree and projector
// density share the SMs without a tail per system.  Items:
//   QI_VPAD   copy a slab of a system's potential into its padded window
//             (the periodic index map of Section 3.1);
//   QI_NODES  the Lanczos recurrence (Section 3.2) or the Chebyshev moments
//             (Eqs. Rec:FD and rhoqj) of a run of consecutive nodes.
// In the Lanczos queue every QI_VPAD item precedes every QI_NODES item, and a
// QI_NODES item first waits until all QI_VPAD items of its system are done:
// thread 0 polls the system's completion count with acquire loads for at most
// `budget` SM clock cycles.  The producers of a count are items taken
// earlier, which no wait holds up, so the count is reached unless something
// is wrong; if the budget runs out the CTA latches ERR_TIMEOUT in the
// system's error word, writes a one-step zero tridiagonal for the item's
// nodes (so every later kernel of the step reads defined values) and goes on
// with the next item.  The host reports that as SQ_ETIMEOUT.
#pragma once
#include "sq_region.cuh"

namespace sq {

constexpr int QMAX = 8;              // systems per queue launch

enum : int { QI_VPAD = 0, QI_NODES = 1 };

struct QItem {
    int sys;                         // index into QueueArgs::sys
    int kind;                        // QI_VPAD or QI_NODES
    long long begin, end;            // padded-potential elements or nodes [begin, end)
};

template <typename T>
struct QueueArgs {
    RegionArgs<T> sys[QMAX];         // per system, as for the single-system kernels
    const double* V[QMAX];           // QI_VPAD: the system's potential (n1 x n2 x n3)
    int need[QMAX];                  // QI_VPAD items of each system
    const QItem* items;
    int n_items;
    unsigned* next;                  // dequeue counter, zero before the launch
    unsigned* done;                  // [QMAX] finished QI_VPAD items, zero before the launch
    long long budget;                // SM clock cycles one wait may take
    int unset;                       // 1: wait for one QI_VPAD item more than exist (exercises the time-out)
};
static_assert(sizeof(QueueArgs<double>) <= 4000, "queue arguments must fit the kernel parameter space");

// Thread 0 takes the next item index; every thread returns it.
__device__ inline int queue_take(unsigned* next, int* slot)
{
    if (threadIdx.x == 0) *slot = (int)atomicAdd(next, 1u);
    __syncthreads();
    const int it = *slot;
    __syncthreads();                 // read by all before thread 0 overwrites it
    return it;
}

// Poll *count (acquire, GPU scope) until it reaches target or `budget` SM
// cycles have passed; true if reached.  Called by one thread.
__device__ inline bool wait_count(const unsigned* count, unsigned target, long long budget)
{
    const long long t0 = clock64();
    for (;;) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
        if (v >= target) return true;
        if (clock64() - t0 >= budget) return false;
        __nanosleep(256);
    }
}

template <typename T, int M, bool DB>
__global__ void __launch_bounds__(Geo<M>::NT, (region_min_blocks<T, M>()))
lanczos_queue_kernel(const __grid_constant__ QueueArgs<T> q)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item, s_go;
    const int tid = threadIdx.x;
    for (;;) {
        const int it = queue_take(q.next, &s_item);
        if (it >= q.n_items) break;
        const QItem w = q.items[it];
        const RegionArgs<T>& a = q.sys[w.sys];
        if (w.kind == QI_VPAD) {
            for (long long t = w.begin + tid; t < w.end; t += Geo<M>::NT)
                vpad_elem<T>(q.V[w.sys], const_cast<T*>(a.Vp), a.g.n1, a.g.n2, a.g.n3, a.g.m, t, a.err);
            __syncthreads();
            if (tid == 0) {
                __threadfence();             // the slab before the count (cumulative over the CTA's writes)
                atomicAdd(q.done + w.sys, 1u);
            }
            continue;
        }
        if (tid == 0) {
            const bool ok = wait_count(q.done + w.sys, (unsigned)(q.need[w.sys] + q.unset), q.budget);
            if (!ok) atomicOr(a.err, ERR_TIMEOUT);
            s_go = ok;
        }
        __syncthreads();
        if (s_go) {
            for (long long node = w.begin; node < w.end; ++node) lanczos_node<T, M, DB>(a, smem_raw, node);
        } else {
            for (long long node = w.begin + tid; node < w.end; node += Geo<M>::NT) {
                a.klen[node] = 1;
                a.alpha[node * (long long)a.nl_cap] = 0.0;
            }
        }
        __syncthreads();
    }
}

template <typename T, int M, bool DB>
__global__ void __launch_bounds__(Geo<M>::NT, (region_min_blocks<T, M>()))
moments_queue_kernel(const __grid_constant__ QueueArgs<T> q)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    for (;;) {
        const int it = queue_take(q.next, &s_item);
        if (it >= q.n_items) break;
        const QItem w = q.items[it];
        const RegionArgs<T>& a = q.sys[w.sys];
        for (long long node = w.begin; node < w.end; ++node) moments_node<T, M, DB>(a, smem_raw, node);
    }
}

}  // namespace sq
