// te_surrogate_test_static: the surrogate test for callers that cannot allocate GPU memory.
//
// Some callers must not call cudaMalloc: code that runs inside another runtime's memory pool
// or a fixed memory budget (an inference server, a plugin host), code that may not trigger an
// implicit device synchronisation, or a process whose allocator is owned by someone else.
// This entry point allocates nothing, on the device or the host. Its scratch space (work-queue
// head, per-item partial sums, per-estimate TE values and the digamma table) is one
// file-scope static device array of fixed size. The CUDA driver maps it, with this file's
// kernels, when the module is first used on a device (with lazy module loading: the first call
// of this entry point there), and every GPU keeps it until the process exits. The caller still
// provides inputs and outputs.
//
// Limits (checked before any launch, TE_ENOTIMPL with a message when exceeded):
//   one series, k <= 4, d = 1..5, N = R * window <= 8192 points, n_t <= 256 start points,
//   n_t * (S + 1) <= 65536 estimates, <= 131072 work items.
// Scratch size: kNaScratchBytes (about 2.6 MiB).
//
// The first call on a device sets that device up: with the device current it resolves the
// array's device address with cudaGetSymbolAddress (the array's name in host code is only a
// host-side stand-in), fills the digamma table with a small kernel, waits for it on the
// caller's stream and sets the kernels' shared-memory attribute. That first call is where the
// driver maps the array (a device allocation of its own, possibly with a synchronisation), so
// make it where that is acceptable, and before any stream capture. Every later call
// reuses the same array and keeps the previous call's contents; the queue head is cleared at
// the start of each call, and every partial sum and TE value is rewritten before it is read.
// Calls whose work overlaps on the GPU (other streams, other host threads) race on the array.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <mutex>

#include "te_batched.cuh"

#define TE_EXPORT extern "C" __attribute__((visibility("default")))

namespace {

constexpr int kNaMaxN = 8192;
constexpr int kNaMaxT = 256;
constexpr int kNaMaxInst = 65536;
constexpr int kNaMaxItems = 131072;
constexpr int kNaMaxDevices = 64;
constexpr int kNaQ = 4;   // queries per thread
constexpr int kNaKS = 5;  // k + 1 slots for k <= 4

// byte offsets of the regions inside the scratch array (each 256-byte aligned)
constexpr size_t kOffWords = 0;                                               // queue, flags
constexpr size_t kOffPsi = 256;                                               // float2 [kNaMaxN + 2]
constexpr size_t kOffPartial = kOffPsi + (((kNaMaxN + 2) * 8 + 255) / 256) * 256;  // double [items]
constexpr size_t kOffPartialAbs = kOffPartial + (size_t)kNaMaxItems * 8;      // double [items]
constexpr size_t kOffTe = kOffPartialAbs + (size_t)kNaMaxItems * 8;           // double [inst]
constexpr size_t kNaScratchBytes = kOffTe + (size_t)kNaMaxInst * 8;

static __device__ __align__(256) unsigned char g_te_noalloc_scratch[kNaScratchBytes];

struct NaParams {
    const float* src;
    const float* tgt;
    const int32_t* perms;
    unsigned char* scratch;  // device address of g_te_noalloc_scratch
    int32_t R, T, d, tau, u, W, S, N, k, n_t, items_per_inst, n_items, smem_floats;
    int32_t t_starts[kNaMaxT];
};

// digamma(n), n = 1 .. kNaMaxN + 1, as (hi, lo) floats: -gamma + H_{n-1} below 16, the
// asymptotic series ln n - 1/(2n) - sum B_2k / (2k n^2k) from 16 on
__global__ void na_psi_kernel(unsigned char* scratch) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    float2* psi = reinterpret_cast<float2*>(scratch + kOffPsi);
    if (n == 0) psi[0] = make_float2(0.f, 0.f);
    if (n < 1 || n > kNaMaxN + 1) return;
    double v;
    if (n < 16) {
        v = -0.57721566490153286060651209;
        for (int m = 1; m < n; ++m) v += 1.0 / m;
    } else {
        const double x = n, r2 = 1.0 / (x * x);
        const double s =
            r2 * (1.0 / 12 - r2 * (1.0 / 120 - r2 * (1.0 / 252 - r2 * (1.0 / 240 - r2 * (1.0 / 132 - r2 * (691.0 / 32760))))));
        v = log(x) - 0.5 / x - s;
    }
    const float hi = (float)v;
    psi[n] = make_float2(hi, (float)(v - (double)hi));
}

// the persistent batched kernel with its estimate descriptors computed from the uniform
// surrogate-test layout instead of read from an uploaded table
template <int d>
__global__ void __launch_bounds__(te::kBatchedMaxThreads) na_batched_kernel(const NaParams p) {
    extern __shared__ __align__(16) float sm[];
    __shared__ double sred[64];
    __shared__ int s_item;
    int32_t* words = reinterpret_cast<int32_t*>(p.scratch + kOffWords);
    te::BatchArgs a{};
    a.n_items = p.n_items;
    a.item_base = 0;
    a.queue = words;
    a.flags = words + 1;
    a.psi = reinterpret_cast<const float2*>(p.scratch + kOffPsi);
    a.k = p.k;
    a.smem_floats = p.smem_floats;
    a.partial = reinterpret_cast<double*>(p.scratch + kOffPartial);
    a.partial_abs = reinterpret_cast<double*>(p.scratch + kOffPartialAbs);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= p.n_items) break;
        const int g = it / p.items_per_inst;          // estimate: t index major, [orig, surrogates]
        const int j = it - g * p.items_per_inst;
        const int ti = g / (p.S + 1);
        const int m = g - ti * (p.S + 1) - 1;         // -1: original pairing
        te::InstDesc I;
        I.src = p.src;
        I.tgt = p.tgt;
        I.perm = m >= 0 ? p.perms + (size_t)m * p.R : nullptr;
        I.R = p.R;
        I.T = p.T;
        I.W = p.W;
        I.t_start = p.t_starts[ti];
        I.tau = p.tau;
        I.u = p.u;
        I.d = d;
        I.N = p.N;
        I.pt_off = 0;
        I.item_begin = g * p.items_per_inst;
        I.n_items = p.items_per_inst;
        I.part_begin = I.item_begin;
        I.n_parts = I.n_items;
        I.warp_mode = 0;
        te::process_item<d, kNaQ, kNaKS>(a, I, j * (int)blockDim.x * kNaQ, it, sm, sred);
    }
}

__global__ void na_finalize_kernel(const NaParams p, double psi_k) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_inst = p.n_t * (p.S + 1);
    if (g >= n_inst) return;
    const double* partial = reinterpret_cast<const double*>(p.scratch + kOffPartial);
    double s = 0.0;
    for (int j = 0; j < p.items_per_inst; ++j) s += partial[(size_t)g * p.items_per_inst + j];
    reinterpret_cast<double*>(p.scratch + kOffTe)[g] = psi_k + s / (double)p.N;
}

const void* na_kernel(int d) {
    switch (d) {
        case 1: return (const void*)na_batched_kernel<1>;
        case 2: return (const void*)na_batched_kernel<2>;
        case 3: return (const void*)na_batched_kernel<3>;
        case 4: return (const void*)na_batched_kernel<4>;
        case 5: return (const void*)na_batched_kernel<5>;
        default: return nullptr;
    }
}

std::mutex g_na_mu;
unsigned char* g_na_ptr[kNaMaxDevices] = {};

te_status na_msg(char* msg, int32_t len, te_status st, const char* text) {
    if (msg && len > 0) snprintf(msg, (size_t)len, "%s", text);
    return st;
}

}  // namespace

// See include/te_gb300.h. Allocation-free variant of te_surrogate_test for one series.
TE_EXPORT te_status te_surrogate_test_static(const te_series* s, const int32_t* t_starts, int32_t n_t,
                                             int32_t window, int32_t S, int32_t k, double* te_orig,
                                             double* te_surr, double* p, void* stream, char* msg,
                                             int32_t msg_len) {
    char buf[256];
    if (msg && msg_len > 0) msg[0] = '\0';
    if (!s || !t_starts || !te_orig || !p || (S > 0 && !te_surr))
        return na_msg(msg, msg_len, TE_EINVAL, "null argument");
    if (!s->src || !s->tgt || s->R < 1 || s->T < 1 || s->tau < 1 || s->u < 0 || window < 1 || S < 0 ||
        (S > 0 && (!s->perms || s->S < S)))
        return na_msg(msg, msg_len, TE_EINVAL, "invalid series, window or surrogate count");
    if (k < 1 || k > kNaKS - 1 || s->d < 1 || s->d > 5) {
        snprintf(buf, sizeof buf, "k=%d d=%d: this entry point supports k <= %d and d = 1..5", k, s->d, kNaKS - 1);
        return na_msg(msg, msg_len, TE_ENOTIMPL, buf);
    }
    const int64_t N = (int64_t)s->R * window;
    const int64_t n_inst = (int64_t)n_t * (S + 1);
    if (n_t < 1 || n_t > kNaMaxT || N > kNaMaxN || n_inst > kNaMaxInst) {
        snprintf(buf, sizeof buf,
                 "size beyond the static scratch: n_t=%d (max %d), N=%lld (max %d), estimates=%lld (max %d)", n_t,
                 kNaMaxT, (long long)N, kNaMaxN, (long long)n_inst, kNaMaxInst);
        return na_msg(msg, msg_len, TE_ENOTIMPL, buf);
    }
    if (N < k + 1) return na_msg(msg, msg_len, TE_EINVAL, "N = R * window must be at least k + 1");
    for (int j = 0; j < n_t; ++j) {
        const int64_t t0 = t_starts[j];
        if (t0 < 0 || t0 + window - 1 > s->T - 1 || t0 - 1 - (int64_t)(s->d - 1) * s->tau < 0 ||
            t0 - s->u - (int64_t)(s->d - 1) * s->tau < 0) {
            snprintf(buf, sizeof buf, "t_starts[%d]=%lld: embedding reaches outside samples 0..%d", j, (long long)t0,
                     s->T - 1);
            return na_msg(msg, msg_len, TE_ERANGE, buf);
        }
    }
    // launch shape: 4 queries per thread, CTA size with the fewest padded query slots
    int threads = 256;
    {
        int64_t best = INT64_MAX;
        for (int m = 1; m <= 64; ++m) {
            int t = 32 * (int)((N + (int64_t)m * kNaQ * 32 - 1) / ((int64_t)m * kNaQ * 32));
            if (t < 64) t = 64;
            if (t > te::kBatchedMaxThreads) continue;
            const int64_t per = (int64_t)t * kNaQ, slots = ((N + per - 1) / per) * per;
            if (slots < best || (slots == best && t < threads)) {
                best = slots;
                threads = t;
            }
            if (t == 64) break;
        }
    }
    const int ipi = (int)((N + (int64_t)threads * kNaQ - 1) / ((int64_t)threads * kNaQ));
    if (n_inst * ipi > kNaMaxItems) {
        snprintf(buf, sizeof buf, "%lld work items exceed the static scratch (max %d)", (long long)(n_inst * ipi),
                 kNaMaxItems);
        return na_msg(msg, msg_len, TE_ENOTIMPL, buf);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return na_msg(msg, msg_len, TE_ECUDA, "no current device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int D = 1 + 2 * s->d;
    const int smem_floats = (int)std::min<int64_t>(16384, ((N + 3) & ~3LL) * D);
    {
        // once per device, with that device current: the array's device address, the digamma
        // table and the kernels' shared-memory limit
        std::lock_guard<std::mutex> lock(g_na_mu);
        if (!g_na_ptr[dev]) {
            void* ptr = nullptr;
            if ((e = cudaGetSymbolAddress(&ptr, g_te_noalloc_scratch)) != cudaSuccess) {
                snprintf(buf, sizeof buf, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
                return na_msg(msg, msg_len, TE_ECUDA, buf);
            }
            for (int dd = 1; dd <= 5; ++dd)
                if ((e = cudaFuncSetAttribute(na_kernel(dd), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              16384 * (int)sizeof(float))) != cudaSuccess)
                    return na_msg(msg, msg_len, TE_ECUDA, "cudaFuncSetAttribute failed");
            na_psi_kernel<<<(kNaMaxN + 2 + 255) / 256, 256, 0, st>>>(static_cast<unsigned char*>(ptr));
            // the table is complete before the device counts as set up: a later call on another
            // stream must not find it half written, and a failed fill must not be reused
            if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess)
                return na_msg(msg, msg_len, TE_ECUDA, cudaGetErrorString(e));
            g_na_ptr[dev] = static_cast<unsigned char*>(ptr);
        }
    }
    NaParams prm{};
    prm.src = s->src;
    prm.tgt = s->tgt;
    prm.perms = s->perms;
    prm.scratch = g_na_ptr[dev];
    prm.R = s->R;
    prm.T = s->T;
    prm.d = s->d;
    prm.tau = s->tau;
    prm.u = s->u;
    prm.W = window;
    prm.S = S;
    prm.N = (int32_t)N;
    prm.k = k;
    prm.n_t = n_t;
    prm.items_per_inst = ipi;
    prm.n_items = (int32_t)(n_inst * ipi);
    prm.smem_floats = smem_floats;
    for (int j = 0; j < n_t; ++j) prm.t_starts[j] = t_starts[j];

    const void* fn = na_kernel(s->d);
    int per_sm = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem_floats * sizeof(float))) !=
            cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return na_msg(msg, msg_len, TE_ECUDA, cudaGetErrorString(e));
    const int grid = (int)std::min<int64_t>((int64_t)std::max(per_sm, 1) * sms, prm.n_items);
    // the queue head and the flag word must start at zero; everything else is overwritten
    if ((e = cudaMemsetAsync(g_na_ptr[dev] + kOffWords, 0, 2 * sizeof(int32_t), st)) != cudaSuccess)
        return na_msg(msg, msg_len, TE_ECUDA, cudaGetErrorString(e));
    void* args[] = {&prm};
    if ((e = cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem_floats * sizeof(float), st)) != cudaSuccess)
        return na_msg(msg, msg_len, TE_ECUDA, cudaGetErrorString(e));
    double psi_k = -0.57721566490153286060651209;
    for (int m = 1; m < k; ++m) psi_k += 1.0 / m;
    na_finalize_kernel<<<(int)((n_inst + 255) / 256), 256, 0, st>>>(prm, psi_k);
    if ((e = cudaGetLastError()) != cudaSuccess) return na_msg(msg, msg_len, TE_ECUDA, cudaGetErrorString(e));
    if ((e = te::launch_finalize_groups(reinterpret_cast<const double*>(g_na_ptr[dev] + kOffTe), n_t, S, te_orig,
                                        te_surr, p, st)) != cudaSuccess)
        return na_msg(msg, msg_len, TE_ECUDA, cudaGetErrorString(e));
    return TE_OK;
}
