// probe.cu -- sl_measure_alu_peak: measured arithmetic peaks of the device,
// the denominators of the roofline fractions that bench.py reports for the
// ALU-bound kernels (the FP64 path, the FP32 contraction and interpolation).
//
// Each thread runs 8 independent multiply-add chains (enough to cover the
// pipe latency at full occupancy); a grid of 8 CTAs of 256 threads per SM runs
// for a fixed number of iterations, timed with CUDA events on a private
// stream, best of 3 after one warm-up launch.  The chains stay bounded
// (x <- x * m + c with m just below 1), and the result is written only when a
// runtime flag that the host always passes as 0 is set, so the arithmetic
// cannot be removed and the kernel touches no memory.
//   kind 0: FP64 fma.rn.f64, 2 flops each
//   kind 1: FP32 fma.rn.f32, 2 flops each
//   kind 2: FP32 fma.rn.f32x2 (two lanes per instruction), 4 flops each
#include "sl_internal.cuh"

namespace sl {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_peak_f64(int iters, int flag, double *out) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    const double m = 0.999999, a = 1e-6;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], m, a);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (flag) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_f32(int iters, int flag, float *out) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.f + 1e-3f * (threadIdx.x + c);
    const float m = 0.9999f, a = 1e-4f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], m, a);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (flag) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_f32x2(int iters, int flag, float *out) {
    unsigned long long x[kChains], m, a;
    const float m1 = 0.9999f, a1 = 1e-4f;
    asm("mov.b64 %0, {%1, %1};" : "=l"(m) : "f"(m1));
    asm("mov.b64 %0, {%1, %1};" : "=l"(a) : "f"(a1));
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        const float lo = 1.f + 1e-3f * (threadIdx.x + c), hi = lo + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(lo), "f"(hi));
    }
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(m), "l"(a));
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    if (flag) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace sl

using namespace sl;

extern "C" sl_status sl_measure_alu_peak(int device, int kind, double *flops_per_s) {
    if (!flops_per_s) return set_error(SL_ERR_ARG, "sl_measure_alu_peak: NULL output");
    if (kind < 0 || kind > 2) return set_error(SL_ERR_ARG, "sl_measure_alu_peak: kind %d not in 0..2", kind);
    sl_status st = cuda_check(cudaSetDevice(device), "cudaSetDevice");
    if (st != SL_OK) return st;
    int nsm = 0;
    if ((st = cuda_check(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device), "SM count")) != SL_OK)
        return st;
    const int blocks = nsm * 8, threads = 256;
    // about 17-20 ms per launch on GB300 (1.06 / 77.8 / 79.2 TFLOP/s measured)
    const int iters = kind == 0 ? 4096 : (kind == 1 ? 262144 : 131072);
    const double flops_per_fma = kind == 2 ? 4.0 : 2.0;
    const double flops = (double)blocks * threads * kChains * (double)iters * flops_per_fma;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((st = cuda_check(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "probe stream")) != SL_OK) return st;
    st = cuda_check(cudaEventCreate(&e0), "probe event");
    if (st == SL_OK) st = cuda_check(cudaEventCreate(&e1), "probe event");
    float best = 0.f;
    for (int rep = 0; rep < 4 && st == SL_OK; ++rep) {
        cudaEventRecord(e0, s);
        if (kind == 0) k_peak_f64<<<blocks, threads, 0, s>>>(iters, 0, nullptr);
        else if (kind == 1) k_peak_f32<<<blocks, threads, 0, s>>>(iters, 0, nullptr);
        else k_peak_f32x2<<<blocks, threads, 0, s>>>(iters, 0, nullptr);
        cudaEventRecord(e1, s);
        st = cuda_check(cudaGetLastError(), "probe launch");
        if (st == SL_OK) st = cuda_check(cudaEventSynchronize(e1), "probe sync");
        float ms = 0.f;
        if (st == SL_OK) st = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "probe timing");
        if (st == SL_OK && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (st != SL_OK) return st;
    *flops_per_s = flops / (best * 1e-3);
    return SL_OK;
}
