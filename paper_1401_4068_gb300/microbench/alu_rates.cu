// Throughput of the FP32 instruction forms the max-norm kernels are built from, on the GPU at
// hand. For each form: one wave of resident blocks (occupancy query), eight independent
// dependency chains per thread so that latency is hidden, rate = instructions / (event time x
// measured SM clock x SM count). Prints one JSON object:
//   warp_inst_per_sm_clk   warp instructions issued per SM per clock for the form;
//   coord_per_sm_clk       for the coordinate forms, (subtract + abs-max) coordinate
//                          evaluations per SM per clock (lanes x coordinates / clock).
// Forms: sub.f32, sub.f32x2 (two subtractions), max.f32, max.abs.f32 with three inputs (two new
// |x| per instruction), set.lt.f32.f32 (1.0f / 0.0f), fma.f32, and the coordinate pairs
//   one coordinate:   sub.f32 + abs + max.f32
//   two coordinates:  sub.f32x2 + max.abs.f32 (three inputs)
// and the count step: set.lt.f32.f32 + add.f32. Integer forms: add.u32, and.b32, min.u32,
// shr.u32 + add.u32 (a sign bit accumulated), and the count step written as an FP32 subtraction
// whose sign bit is accumulated: b < e exactly when fl(b - e) has its sign bit set (fl(b - e) is
// +0 when b == e), so [b < e] = sign(fl(b - e)); "count x2" is the n_xz form (two such
// subtractions, their sign bits ANDed, then accumulated).
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { \
    fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_)); return 1; } } while (0)

constexpr int kIters = 8192;
constexpr int kChains = 8;
constexpr int kThreads = 256;

enum Op { OP_FADD, OP_FSUB2, OP_FMAX, OP_FMAX3_ABS, OP_FSET, OP_FFMA, OP_COORD1, OP_COORD2, OP_COUNT,
          OP_IADD, OP_LOP, OP_IMIN, OP_SHRADD, OP_COUNT_SIGN, OP_COUNT_SIGN2 };

template <int OP>
__global__ void __launch_bounds__(kThreads) rate_kernel(float* out, float seed) {
    float a[kChains];
    unsigned ua[kChains];
    unsigned long long v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        a[c] = seed * (float)(threadIdx.x + c);
        ua[c] = threadIdx.x * 7u + c;
        v[c] = ((unsigned long long)__float_as_uint(a[c] + 1.5f) << 32) | __float_as_uint(a[c] + 0.5f);
    }
    const float b = seed * 0.5f, b2 = seed * 0.25f;
    const unsigned long long bb = ((unsigned long long)__float_as_uint(b2) << 32) | __float_as_uint(b);
    const unsigned ub = __float_as_uint(seed) | 1u;
#pragma unroll 1
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (OP == OP_FADD) asm volatile("sub.rn.f32 %0, %0, %1;" : "+f"(a[c]) : "f"(b));
            if (OP == OP_FSUB2) asm volatile("sub.rn.f32x2 %0, %0, %1;" : "+l"(v[c]) : "l"(bb));
            if (OP == OP_FMAX) asm volatile("max.f32 %0, %0, %1;" : "+f"(a[c]) : "f"(b));
            if (OP == OP_FMAX3_ABS) asm volatile("max.abs.f32 %0, %0, %1, %2;" : "+f"(a[c]) : "f"(b), "f"(b2));
            if (OP == OP_FSET) asm volatile("set.lt.f32.f32 %0, %0, %1;" : "+f"(a[c]) : "f"(b));
            if (OP == OP_FFMA) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[c]) : "f"(b), "f"(b2));
            // one coordinate: the difference depends on the chain, so nothing can be hoisted
            if (OP == OP_COORD1)
                asm volatile("{.reg .f32 t; sub.rn.f32 t, %1, %0; abs.f32 t, t; max.f32 %0, %0, t;}"
                             : "+f"(a[c]) : "f"(b));
            // two coordinates: the packed difference is a chain of its own, the max consumes it
            if (OP == OP_COORD2)
                asm volatile("{.reg .f32 lo, hi; sub.rn.f32x2 %1, %1, %2; mov.b64 {lo, hi}, %1;"
                             " max.abs.f32 %0, %0, lo, hi;}"
                             : "+f"(a[c]), "+l"(v[c]) : "l"(bb));
            if (OP == OP_COUNT)
                asm volatile("{.reg .f32 s; set.lt.f32.f32 s, %1, %2; add.rn.f32 %0, %0, s;}"
                             : "+f"(a[c]) : "f"(b2 + a[c]), "f"(b));
            if (OP == OP_IADD) asm volatile("add.u32 %0, %0, %1;" : "+r"(ua[c]) : "r"(ub));
            if (OP == OP_LOP) asm volatile("xor.b32 %0, %0, %1;" : "+r"(ua[c]) : "r"(ub));
            if (OP == OP_IMIN) asm volatile("min.u32 %0, %0, %1;" : "+r"(ua[c]) : "r"(ub + (unsigned)c));
            if (OP == OP_SHRADD)
                asm volatile("{.reg .u32 t; shr.u32 t, %1, 31; add.u32 %0, %0, t;}"
                             : "+r"(ua[c]) : "r"(ua[c] ^ ub));
            // the difference depends on the chain's previous value, so nothing is hoisted
            if (OP == OP_COUNT_SIGN)
                asm volatile("{.reg .f32 d; .reg .u32 t; sub.rn.f32 d, %1, %2; mov.b32 t, d; shr.u32 t, t, 31;"
                             " add.u32 %0, %0, t;}"
                             : "+r"(ua[c]) : "f"(__uint_as_float(ua[c] & 0x3fffffffu)), "f"(b));
            if (OP == OP_COUNT_SIGN2)
                asm volatile("{.reg .f32 d, e; .reg .u32 t, w; sub.rn.f32 d, %1, %2; sub.rn.f32 e, %3, %2;"
                             " mov.b32 t, d; mov.b32 w, e; and.b32 t, t, w; shr.u32 t, t, 31; add.u32 %0, %0, t;}"
                             : "+r"(ua[c]) : "f"(__uint_as_float(ua[c] & 0x3fffffffu)), "f"(b),
                               "f"(__uint_as_float((ua[c] >> 1) & 0x3fffffffu)));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c] + __uint_as_float((unsigned)v[c]) + (float)ua[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void clock_kernel(long long* c, unsigned long long* ns) {
    unsigned long long g0, g1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g0));
    const long long t0 = clock64();
    long long t = t0;
    while (t - t0 < 200000000LL) t = clock64();  // about 0.1 s, ends by itself
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g1));
    c[0] = t - t0;
    ns[0] = g1 - g0;
}

double g_mhz = 0;

int measure_clock() {
    long long* dc;
    unsigned long long* dn;
    CK(cudaMalloc(&dc, 8));
    CK(cudaMalloc(&dn, 8));
    clock_kernel<<<1, 1>>>(dc, dn);
    CK(cudaDeviceSynchronize());
    long long hc;
    unsigned long long hn;
    CK(cudaMemcpy(&hc, dc, 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&hn, dn, 8, cudaMemcpyDeviceToHost));
    g_mhz = (double)hc / (double)hn * 1e3;
    cudaFree(dc);
    cudaFree(dn);
    return 0;
}

template <int OP>
int run(const char* name, int sms, float* out, int first, int inst_per_step, int coords_per_step) {
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rate_kernel<OP>, kThreads, 0));
    const int blocks = sms * per_sm;  // one wave
    rate_kernel<OP><<<blocks, kThreads>>>(out, 1.0001f);
    CK(cudaDeviceSynchronize());
    if (measure_clock()) return 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0);
    rate_kernel<OP><<<blocks, kThreads>>>(out, 1.0001f);
    cudaEventRecord(e1);
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    const double steps = (double)blocks * (kThreads / 32) * kIters * kChains;  // warp steps
    const double clk = ms * 1e-3 * g_mhz * 1e6 * sms;                           // SM clocks
    printf("%s\"%s\": {\"warp_inst_per_sm_clk\": %.3f", first ? "" : ", ", name, steps * inst_per_step / clk);
    if (coords_per_step) printf(", \"coord_per_sm_clk\": %.1f", steps * 32.0 * coords_per_step / clk);
    printf(", \"blocks_per_sm\": %d, \"kernel_ms\": %.3f, \"sm_mhz\": %.0f}", per_sm, ms, g_mhz);
    return 0;
}

int main() {
    int sms = 0;
    CK(cudaSetDevice(0));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, 0));
    float* out;
    CK(cudaMalloc(&out, sizeof(float) * sms * 32 * kThreads));
    printf("{\"gpu\": \"%s\", \"sms\": %d, \"iters\": %d, \"chains\": %d, \"rates\": {", prop.name, sms, kIters,
           kChains);
    int rc = 0;
    rc |= run<OP_FADD>("sub.f32", sms, out, 1, 1, 0);
    rc |= run<OP_FSUB2>("sub.f32x2", sms, out, 0, 1, 0);
    rc |= run<OP_FMAX>("max.f32", sms, out, 0, 1, 0);
    rc |= run<OP_FMAX3_ABS>("max.abs.f32 (3 inputs)", sms, out, 0, 1, 0);
    rc |= run<OP_FSET>("set.lt.f32.f32", sms, out, 0, 1, 0);
    rc |= run<OP_FFMA>("fma.f32", sms, out, 0, 1, 0);
    rc |= run<OP_COORD1>("coordinate: sub + abs + max", sms, out, 0, 0, 1);
    rc |= run<OP_COORD2>("2 coordinates: sub.f32x2 + max.abs (3 inputs)", sms, out, 0, 0, 2);
    rc |= run<OP_COUNT>("count: set.lt.f32.f32 + add.f32", sms, out, 0, 2, 0);
    rc |= run<OP_IADD>("add.u32", sms, out, 0, 1, 0);
    rc |= run<OP_LOP>("xor.b32", sms, out, 0, 1, 0);
    rc |= run<OP_IMIN>("min.u32", sms, out, 0, 1, 0);
    rc |= run<OP_SHRADD>("shr.u32 31 + add.u32 (per pair)", sms, out, 0, 1, 0);
    rc |= run<OP_COUNT_SIGN>("count: sub.f32 + sign-bit accumulate (per count)", sms, out, 0, 1, 0);
    rc |= run<OP_COUNT_SIGN2>("count x2: 2 sub.f32 + and + sign accumulate (per count)", sms, out, 0, 1, 0);
    printf("}}\n");
    return rc;
}
