// The lane kernel's pre-passes (sorted target parts, member-minor source arrays) and launchers;
// its instantiations are in te_lanes_d2.cu .. te_lanes_d8.cu (one embedding dimension each).
#include <algorithm>

#include "te_lanes.cuh"

namespace te {

// Pre-pass: the sorted target part and (r, w) of every point of every lane group.
__global__ void lane_stage_kernel(const LaneGroup* __restrict__ groups, int n_groups,
                                  const int32_t* __restrict__ sorted_idx, float2* __restrict__ tpart,
                                  int32_t* __restrict__ rw, float* __restrict__ ckey) {
    for (int g = blockIdx.y; g < n_groups; g += gridDim.y) {
        const LaneGroup G = groups[g];
        const int NP = (G.N + 31) & ~31;
        const int DA = 1 + G.d, DA2 = (G.d + 2) / 2;
        for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < NP; p += gridDim.x * blockDim.x) {
            float2* tp = tpart + G.tp_off + (size_t)(p >> 5) * (DA2 * 32) + (p & 31);  // chunk-major
            // positions past N (and the strip padding, index -1, which lies there) are padding
            const int i = p < G.N ? __ldg(sorted_idx + G.sort_off + p) : -1;
            if (i >= 0) {
                const int r = i / G.W, w = i - r * G.W;
                const int t = G.t_start + w;
                const float* y = G.tgt + (size_t)r * G.T;
                for (int c2 = 0; c2 < DA2; ++c2) {
                    const int c0 = 2 * c2, c1 = 2 * c2 + 1 < DA ? 2 * c2 + 1 : 1;
                    const float v0 = c0 == 0 ? __ldg(y + t) : __ldg(y + t - 1 - (c0 - 1) * G.tau);
                    const float v1 = __ldg(y + t - 1 - (c1 - 1) * G.tau);
                    tp[c2 * 32] = make_float2(v0, v1);
                }
                rw[G.rw_off + p] = (int32_t)(((uint32_t)r << 16) | (uint32_t)w);
                if ((p & 31) == 0) ckey[G.ck_off + (p >> 5)] = __ldg(y + t - 1);
            } else {
                for (int c2 = 0; c2 < DA2; ++c2) tp[c2 * 32] = make_float2(f_inf(), f_inf());
                rw[G.rw_off + p] = 0;
                if ((p & 31) == 0) ckey[G.ck_off + (p >> 5)] = f_inf();
            }
        }
    }
}

// Pre-pass: the member-minor source arrays of the lane blocks (LaneXBlock); a permutation entry
// outside 0..R-1 raises the flag and reads repetition 0.
__global__ void lane_x_kernel(const LaneXBlock* __restrict__ blocks, int n_blocks, float* __restrict__ X,
                              int32_t* flags) {
    for (int b = blockIdx.y; b < n_blocks; b += gridDim.y) {
        const LaneXBlock& B = blocks[b];
        const int64_t total = (int64_t)B.R * B.ncols * 32;
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
             e += (int64_t)gridDim.x * blockDim.x) {
            const int lane = (int)(e & 31);
            const int64_t rc = e >> 5;
            const int r = (int)(rc / B.ncols);
            const int c = (int)(rc - (int64_t)r * B.ncols);
            const int32_t* perm = B.perm[lane];
            int rs = perm ? __ldg(perm + r) : r;
            if ((unsigned)rs >= (unsigned)B.R) {
                atomicOr(flags, kFlagBadPerm);
                rs = 0;
            }
            X[B.off + e] = __ldg(B.src[lane] + (size_t)rs * B.T + B.t0 + c);
        }
    }
}

const void* lane_kernel_ptr(int d, int ks, int tc) {
    switch (d) {
        case 2: return lane_ptr_d2(ks, tc);
        case 3: return lane_ptr_d3(ks, tc);
        case 4: return lane_ptr_d4(ks, tc);
        case 5: return lane_ptr_d5(ks, tc);
        case 6: return lane_ptr_d6(ks, tc);
        case 7: return lane_ptr_d7(ks, tc);
        case 8: return lane_ptr_d8(ks, tc);
        default: return nullptr;
    }
}

cudaError_t launch_lanes(int d, int ks, int tc, const BatchArgs& a, int grid, cudaStream_t s) {
    const void* fn = lane_kernel_ptr(d, ks, tc);
    if (!fn) return cudaErrorInvalidDeviceFunction;
    void* args[] = {const_cast<BatchArgs*>(&a)};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kLaneThreads), args, 0, s);
}

cudaError_t launch_lane_stage(const LaneGroup* groups, int n_groups, int max_np, const int32_t* sorted_idx,
                              float2* tpart, int32_t* lane_rw, float* lane_ckey, const LaneXBlock* xblocks,
                              int n_xblocks, int64_t max_x, float* lane_x, int32_t* flags, cudaStream_t s) {
    if (n_groups <= 0) return cudaSuccess;
    const int threads = 256;
    const dim3 grid((unsigned)std::min(64, (max_np + threads - 1) / threads), (unsigned)std::min(n_groups, 65535));
    lane_stage_kernel<<<grid, threads, 0, s>>>(groups, n_groups, sorted_idx, tpart, lane_rw, lane_ckey);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || n_xblocks <= 0) return e;
    const dim3 gx((unsigned)std::min<int64_t>(1024, (max_x + threads - 1) / threads),
                  (unsigned)std::min(n_xblocks, 65535));
    lane_x_kernel<<<gx, threads, 0, s>>>(xblocks, n_xblocks, lane_x, flags);
    return cudaGetLastError();
}

}  // namespace te
