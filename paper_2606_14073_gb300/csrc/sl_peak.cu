// sl_peak.cu -- FMA throughput microbenchmark (the ALU roofline of the descriptor kernels).
//
// Every thread runs 8 independent FMA chains; 4 blocks of 256 threads per SM keep
// every scheduler issuing.  FLOP count: 2 per FMA.
#include <cstring>

#include "sl_internal.h"

namespace sl {

template <typename R>
__global__ void __launch_bounds__(256) k_fma_peak(R *out, int iters, R b, R c) {
    R a[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) a[t] = R(threadIdx.x) * R(1e-3) + R(t);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int t = 0; t < 8; ++t) a[t] = a[t] * b + c;
        }
    }
    R s = R(0);
#pragma unroll
    for (int t = 0; t < 8; ++t) s += a[t];
    if (s == R(-12345.678)) out[blockIdx.x] = s;   // keeps the chains live, never true
}

template <typename R>
static int run_peak(int iters, double *flops, double *ms) {
    int dev, sms;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    R *out;
    if (cudaMalloc(&out, sizeof(R) * sms * 8) != cudaSuccess) return -1;
    const int blocks = sms * 4, threads = 256;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_peak<R><<<blocks, threads>>>(out, 16, R(0.999999), R(1e-7));   // warm-up
    cudaEventRecord(e0);
    k_fma_peak<R><<<blocks, threads>>>(out, iters, R(0.999999), R(1e-7));
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return -1;
    *ms = t;
    *flops = 2.0 * 8.0 * 16.0 * (double)iters * blocks * threads / (t * 1e-3);
    return 0;
}

// Self-test of the FP32 radial carrier (polynomial cutoff) against the FP64 one (library
// sincospi): f_k and df_k/dr at r = rc (i + 1/2)/n, i < n.  err[0], err[1]: largest
// |f32 - f64| and |df32 - df64|; err[2], err[3]: largest |f64| and |df64| (all >= 0, so
// the FP64 bit patterns order like the values).
__global__ void k_selftest_carrier(int n, double rc, unsigned long long *err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double r = rc * ((double)i + 0.5) / (double)n;
    double fd[NK], dfd[NK];
    float ff[NK], dff[NK];
    carrier_fd<double>(r, 1.0 / rc, fd, dfd);
    carrier_fd<float>((float)r, (float)(1.0 / rc), ff, dff);
    double e0 = 0, e1 = 0, m0 = 0, m1 = 0;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        e0 = fmax(e0, fabs((double)ff[k] - fd[k]));
        e1 = fmax(e1, fabs((double)dff[k] - dfd[k]));
        m0 = fmax(m0, fabs(fd[k]));
        m1 = fmax(m1, fabs(dfd[k]));
    }
    atomicMax(err + 0, (unsigned long long)__double_as_longlong(e0));
    atomicMax(err + 1, (unsigned long long)__double_as_longlong(e1));
    atomicMax(err + 2, (unsigned long long)__double_as_longlong(m0));
    atomicMax(err + 3, (unsigned long long)__double_as_longlong(m1));
}

int selftest_carrier(int n, double rc, double out[4]) {
    unsigned long long *d;
    if (cudaMalloc(&d, 4 * sizeof(unsigned long long)) != cudaSuccess) return -1;
    cudaMemset(d, 0, 4 * sizeof(unsigned long long));
    k_selftest_carrier<<<(n + 255) / 256, 256>>>(n, rc, d);
    unsigned long long h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return -1;
    for (int t = 0; t < 4; ++t) {
        double v;
        std::memcpy(&v, &h[t], sizeof v);
        out[t] = v;
    }
    return 0;
}

int measure_fma_peak(int precision, double *flops, double *ms) {
    // FP32: ~0.2 s at ~70 TFLOP/s; FP64 is expected far slower on this part, so
    // fewer iterations keep that run short as well.
    return precision == 0 ? run_peak<double>(512, flops, ms) : run_peak<float>(8192, flops, ms);
}

}  // namespace sl
