// The persistent batched kernel: a CTA takes (instance, query tile) work items from a device queue
// (atomic ticket, no waits) and runs the exhaustive search (process_item) or the sorted sweep
// (process_item_sweep) on each. DLO..DHI: embedding dimensions compiled in (one specialised d = 1..8,
// or all of 1..5 with a switch); Q: queries per thread; KS: top-k slots (k + 1 rounded up).
#pragma once

#include "te_sweep.cuh"

namespace te {

template <int DLO, int DHI, int Q, int KS, bool SWEEP>
__global__ void __launch_bounds__(kBatchedMaxThreads) batched_kernel(const BatchArgs a) {
    extern __shared__ __align__(16) float sm[];
    __shared__ double sred[64];
    __shared__ float sbnd[64];
    __shared__ int s_item;
    __shared__ int s_wblock;
    if constexpr (SWEEP) work_reset();
    for (;;) {
        __syncthreads();  // everyone is done with s_item / sred of the previous item
        if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
        __syncthreads();
        const int ticket = s_item;
        if (ticket >= a.n_items) break;
        const int it = a.item_base + ticket;
        const WorkItem w = a.items[it];
        const InstDesc I = a.insts[w.inst];
        const int part = I.part_begin + (it - I.item_begin);
#define TE_PROCESS(DD)                                                                    \
    do {                                                                                  \
        if constexpr (SWEEP) {                                                            \
            if (I.warp_mode)                                                              \
                process_instance_sweep_warps<DD, Q, KS>(a, I, w.q0, sm, &s_wblock);       \
            else if (I.strips > 1)                                                        \
                process_item_sweep_strips<DD, Q, KS>(a, I, w.q0, part, sm, sred, sbnd);   \
            else                                                                          \
                process_item_sweep<DD, Q, KS>(a, I, w.q0, part, sm, sred, sbnd);          \
        } else {                                                                          \
            process_item<DD, Q, KS>(a, I, w.q0, part, sm, sred);                          \
        }                                                                                 \
    } while (0)
        if constexpr (DLO == DHI) {
            TE_PROCESS(DLO);
        } else {
            switch (I.d) {
                case 1: if constexpr (DLO <= 1 && 1 <= DHI) TE_PROCESS(1); break;
                case 2: if constexpr (DLO <= 2 && 2 <= DHI) TE_PROCESS(2); break;
                case 3: if constexpr (DLO <= 3 && 3 <= DHI) TE_PROCESS(3); break;
                case 4: if constexpr (DLO <= 4 && 4 <= DHI) TE_PROCESS(4); break;
                case 5: if constexpr (DLO <= 5 && 5 <= DHI) TE_PROCESS(5); break;
                default: break;
            }
        }
#undef TE_PROCESS
    }
    if constexpr (SWEEP) work_flush(a);
}

// Sweep kernel for batches whose every estimate is staged whole in shared memory (warp mode)
// with d <= 2: without the tiled path it fits 64 registers, so a CTA can have 1024 threads, twice
// the warps per SM when one large instance (an AR(1) window of 15,000 points) fills shared memory.
template <int DD, int Q, int KS>
__global__ void __launch_bounds__(kSweepWarpThreads) sweep_warp_kernel(const BatchArgs a) {
    extern __shared__ __align__(16) float sm[];
    __shared__ int s_item;
    __shared__ int s_wblock;
    work_reset();
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
        __syncthreads();
        const int ticket = s_item;
        if (ticket >= a.n_items) break;
        const WorkItem w = a.items[a.item_base + ticket];
        const InstDesc I = a.insts[w.inst];
        process_instance_sweep_warps<DD, Q, KS>(a, I, w.q0, sm, &s_wblock);
    }
    work_flush(a);
}

#define TE_SWEEP_WARP_PTR_FN(NAME, DD)                                                           \
    const void* NAME(int ks, int q) {                                                            \
        if (ks != 5) return nullptr;                                                             \
        if (q == 2) return (const void*)sweep_warp_kernel<DD, 2, 5>;                             \
        if (q == 1) return (const void*)sweep_warp_kernel<DD, 1, 5>;                             \
        return nullptr;                                                                          \
    }

// kernel pointer of one variant (defined in te_batched_*.cu); k > 4 runs with 2 queries per
// thread only (17 slots x 4 queries would not fit the register budget)
#define TE_BATCHED_PTR_FN(NAME, DLO, DHI)                                                        \
    const void* NAME(int ks, int q, bool sweep) {                                                \
        if (q == 2) {                                                                            \
            if (ks == 5) return sweep ? (const void*)batched_kernel<DLO, DHI, 2, 5, true>        \
                                      : (const void*)batched_kernel<DLO, DHI, 2, 5, false>;      \
            if (ks == 17) return sweep ? (const void*)batched_kernel<DLO, DHI, 2, 17, true>      \
                                       : (const void*)batched_kernel<DLO, DHI, 2, 17, false>;    \
        } else if (q == 4) {                                                                     \
            if (ks == 5) return sweep ? (const void*)batched_kernel<DLO, DHI, 4, 5, true>        \
                                      : (const void*)batched_kernel<DLO, DHI, 4, 5, false>;      \
        }                                                                                        \
        return nullptr;                                                                          \
    }

// d = 6..8 (joint dimension 13..17): one query per thread (the duplicated coordinates of two
// queries plus four references' would not fit the register budget)
#define TE_BATCHED_PTR_FN_WIDE(NAME, DD)                                                         \
    const void* NAME(int ks, int q, bool sweep) {                                                \
        if (q != 1) return nullptr;                                                              \
        if (ks == 5) return sweep ? (const void*)batched_kernel<DD, DD, 1, 5, true>              \
                                  : (const void*)batched_kernel<DD, DD, 1, 5, false>;            \
        if (ks == 17) return sweep ? (const void*)batched_kernel<DD, DD, 1, 17, true>            \
                                   : (const void*)batched_kernel<DD, DD, 1, 17, false>;          \
        return nullptr;                                                                          \
    }

}  // namespace te
