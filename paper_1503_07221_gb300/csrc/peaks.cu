// FMA throughput of the current device (not part of the paper's method): the
// denominators of the roofline fractions that bench.py reports. Each thread
// runs eight independent FMA chains (packed FP32 pairs, FP64) so the pipes,
// not the latency, bound the rate; the results land in a device sink that
// is never read, so nothing is allocated.
#include "tdbem_internal.h"

namespace tdbem {

static __device__ double g_peak_sink;

__global__ void __launch_bounds__(256) peak_f32x2_kernel(float s, int iters) {
    unsigned long long a[8], ss, h;
    asm("mov.b64 %0, {%1, %1};" : "=l"(ss) : "f"(s));
    asm("mov.b64 %0, {%1, %1};" : "=l"(h) : "f"(0.5f));
    for (int k = 0; k < 8; ++k) {
        const float v = threadIdx.x * 1e-3f + k;
        asm("mov.b64 %0, {%1, %1};" : "=l"(a[k]) : "f"(v));
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(ss), "l"(h));
    }
    float t = 0.f;
    for (int k = 0; k < 8; ++k) {
        float x, y;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a[k]));
        t += x + y;
    }
    if (t == 12345.f) g_peak_sink = t;
}

__global__ void __launch_bounds__(256) peak_f64_kernel(double s, int iters) {
    double a[8];
    for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 1e-3 + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], s, 0.5);
    }
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += a[k];
    if (t == 12345.0) g_peak_sink = t;
}

// FP32 (packed-pair FMA) and FP64 FMA throughput in TFLOP/s; FMA = 2 flops.
cudaError_t measure_fma_peaks(double *fp32, double *fp64, cudaStream_t st) {
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
    const int blocks = nsm * 8, threads = 256;
    const int it32 = 20000, it64 = 2000;
    float ms32 = 0.f, ms64 = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, st);
        peak_f32x2_kernel<<<blocks, threads, 0, st>>>(0.999f, it32);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms32, e0, e1);
        cudaEventRecord(e0, st);
        peak_f64_kernel<<<blocks, threads, 0, st>>>(0.999, it64);
        cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms64, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    const double n = (double)blocks * threads * 8;
    if (fp32) *fp32 = 2.0 * 2.0 * n * it32 / (ms32 * 1e-3) / 1e12;
    if (fp64) *fp64 = 2.0 * n * it64 / (ms64 * 1e-3) / 1e12;
    return cudaGetLastError();
}

}  // namespace tdbem
