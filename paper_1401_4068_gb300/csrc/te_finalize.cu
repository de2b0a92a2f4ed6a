// Per-instance TE from the work items' partial sums (Eq. 9 / Eq. 10: psi(k) plus the mean of
// the per-point digamma terms) and the surrogate p-value ("TE calculation and statistical
// testing against surrogate data": share of surrogate TE values >= the original TE).
// Both run in FP64 in a fixed order, so results do not depend on the queue's schedule.
#include "te_batched.cuh"

namespace te {

namespace {

__global__ void finalize_te_kernel(const InstDesc* __restrict__ insts, int n_inst,
                                   const double* __restrict__ partial,
                                   const double* __restrict__ partial_abs, double psi_k,
                                   double err_coef, double* __restrict__ te,
                                   double* __restrict__ err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_inst) return;
    const InstDesc I = insts[i];
    double s = 0.0, sa = 0.0;
    for (int m = 0; m < I.n_parts; ++m) {
        s += partial[I.part_begin + m];
        sa += partial_abs[I.part_begin + m];
    }
    te[i] = psi_k + s / (double)I.N;
    if (err) err[i] = sa * err_coef / (double)I.N + fabs(psi_k) * 0x1p-52;
}

// one block per (series, time point) group laid out as [original, surrogate 0 .. S-1]
__global__ void finalize_groups_kernel(const double* __restrict__ te_all, int S,
                                       double* __restrict__ te_orig, double* __restrict__ te_surr,
                                       double* __restrict__ p) {
    const int g = blockIdx.x;
    const double* v = te_all + (size_t)g * (S + 1);
    const double t0 = v[0];
    int n = 0;
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        const double ts = v[1 + s];
        te_surr[(size_t)g * S + s] = ts;
        n += ts >= t0 ? 1 : 0;
    }
    __shared__ int sc[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0) sc[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sc[w];
        te_orig[g] = t0;
        p[g] = S > 0 ? (double)tot / (double)S : __longlong_as_double(0x7ff8000000000000LL);
    }
}

// Eq. 5: the reconstructed delay of each analysis start is the scanned u of largest TE
// (strictly larger wins, so ties go to the smaller u; NaN never wins)
__global__ void delay_argmax_kernel(const double* __restrict__ te, int n_u, int n_t, int u_lo,
                                    int32_t* __restrict__ u_best) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_t) return;
    double best = te[j];
    int bu = 0;
    for (int iu = 1; iu < n_u; ++iu) {
        const double v = te[(size_t)iu * n_t + j];
        if (v > best || (best != best && v == v)) {
            best = v;
            bu = iu;
        }
    }
    u_best[j] = u_lo + bu;
}

}  // namespace

cudaError_t launch_delay_argmax(const double* te, int n_u, int n_t, int u_lo, int32_t* u_best, cudaStream_t s) {
    delay_argmax_kernel<<<(n_t + 127) / 128, 128, 0, s>>>(te, n_u, n_t, u_lo, u_best);
    return cudaGetLastError();
}

const void* batched_kernel_ptr(const BatchedVariant& v) {
    if (v.warp_only) {
        if (!v.sweep || v.dlo != v.dhi) return nullptr;
        if (v.dlo == 1) return sweep_warp_ptr_d1(v.ks, v.qpt);
        if (v.dlo == 2) return sweep_warp_ptr_d2(v.ks, v.qpt);
        return nullptr;
    }
    if (v.dlo == v.dhi) {
        switch (v.dlo) {
            case 1: return batched_ptr_d1(v.ks, v.qpt, v.sweep);
            case 2: return batched_ptr_d2(v.ks, v.qpt, v.sweep);
            case 3: return batched_ptr_d3(v.ks, v.qpt, v.sweep);
            case 4: return batched_ptr_d4(v.ks, v.qpt, v.sweep);
            case 5: return batched_ptr_d5(v.ks, v.qpt, v.sweep);
            case 6: return batched_ptr_d6(v.ks, v.qpt, v.sweep);
            case 7: return batched_ptr_d7(v.ks, v.qpt, v.sweep);
            case 8: return batched_ptr_d8(v.ks, v.qpt, v.sweep);
            default: return nullptr;
        }
    }
    return v.dhi <= 5 ? batched_ptr_mix(v.ks, v.qpt, v.sweep) : nullptr;
}

cudaError_t launch_batched(const BatchedVariant& v, const BatchArgs& a, int grid, int threads,
                           size_t smem, cudaStream_t s) {
    const void* fn = batched_kernel_ptr(v);
    if (!fn) return cudaErrorInvalidDeviceFunction;
    void* args[] = {const_cast<BatchArgs*>(&a)};
    return cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, s);
}

cudaError_t launch_finalize_te(const InstDesc* insts, int n_inst, const double* partial,
                               const double* partial_abs, double psi_k, double err_coef,
                               double* te, double* err, cudaStream_t s) {
    finalize_te_kernel<<<(n_inst + 127) / 128, 128, 0, s>>>(insts, n_inst, partial, partial_abs,
                                                            psi_k, err_coef, te, err);
    return cudaGetLastError();
}

cudaError_t launch_finalize_groups(const double* te_all, int n_groups, int S, double* te_orig,
                                   double* te_surr, double* p, cudaStream_t s) {
    finalize_groups_kernel<<<n_groups, 256, 0, s>>>(te_all, S, te_orig, te_surr, p);
    return cudaGetLastError();
}

}  // namespace te
