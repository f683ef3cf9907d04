// pic_probe_fp64_rate: the FP64 fused multiply-add rate this device sustains, measured
// with many independent dependency chains per thread so that the FP64 pipes, not the
// instruction latency, bound it.  The benchmark divides the FP64 tile kernel's operation
// count by it (an ALU roofline from a measurement instead of a data-sheet figure).
#include "pic_internal.cuh"

namespace gbpic {

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_ITERS = 4096;

__device__ double g_probe_sink;   // keeps the chains live

__global__ void __launch_bounds__(256) k_probe_dfma(double b, double c) {
    double a[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = threadIdx.x * 1e-3 + k;
#pragma unroll 4
    for (int it = 0; it < PROBE_ITERS; ++it) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += a[k];
    if (s == 1.2345e300) g_probe_sink = s;   // never true for these inputs
}

}  // namespace gbpic

using namespace gbpic;

extern "C" pic_status pic_probe_fp64_rate(int32_t device, double* flops_per_s) {
    if (!flops_per_s || device < 0) return PIC_ERR_ARG;
    *flops_per_s = 0.0;
    DeviceScope dscope_(device);
    if (!dscope_.ok) return PIC_ERR_NO_DEVICE;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0)
        return PIC_ERR_NO_DEVICE;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return PIC_ERR_CUDA;
    const int blocks = sms * 8, threads = 256;
    k_probe_dfma<<<blocks, threads>>>(0.999999, 1e-7);   // warm-up
    cudaEventRecord(a);
    const int reps = 5;
    for (int r = 0; r < reps; ++r) k_probe_dfma<<<blocks, threads>>>(0.999999, 1e-7);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess || !(ms > 0.0f)) return PIC_ERR_CUDA;
    const double flops = 2.0 * PROBE_CHAINS * PROBE_ITERS * (double)blocks * threads * reps;
    *flops_per_s = flops / (ms * 1e-3);
    return PIC_OK;
}
