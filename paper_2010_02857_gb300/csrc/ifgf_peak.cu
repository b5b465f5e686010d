// Roofline probe: the FP64 and FP32 fused multiply-add throughput of the current device,
// measured by a kernel of independent FMA chains that touches no memory (one store per
// thread, taken only on an impossible value so that the chains are not removed).
//
// The evaluation kernels of the FP64 and mixed paths are bound by these pipes (their
// operands come from registers, shared memory and L1), so their roofline fractions are
// taken against the rates measured here rather than against nominal figures.
#include <algorithm>

#include "ifgf_internal.h"

namespace {

constexpr int kChains = 8;      // independent FMA chains per thread
constexpr int kPeakThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(T *sink, int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = T(threadIdx.x + 1) * T(1e-3) + T(i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    // the chains stay finite and positive (a < 1, b > 0), so this store never happens
    if (s == T(-1) && sink) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
cudaError_t time_peak(cudaStream_t st, int blocks, int iters, double *tflops)
{
    cudaEvent_t e0, e1;
    cudaError_t err = cudaEventCreate(&e0);
    if (err != cudaSuccess) return err;
    err = cudaEventCreate(&e1);
    if (err != cudaSuccess) {
        cudaEventDestroy(e0);
        return err;
    }
    const T a = T(0.999999), b = T(1e-6);
    double best = 0;
    for (int rep = 0; rep < 6 && err == cudaSuccess; ++rep) {  // the first run warms up
        cudaEventRecord(e0, st);
        k_fma_peak<T><<<blocks, kPeakThreads, 0, st>>>(nullptr, iters, a, b);
        cudaEventRecord(e1, st);
        err = cudaGetLastError();
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && rep > 0 && ms > 0) {
            const double flops = 2.0 * kChains * (double)iters * blocks * kPeakThreads;
            best = std::max(best, flops / (ms * 1e-3) / 1e12);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *tflops = best;
    return err;
}

}  // namespace

extern "C" ifgf_status ifgf_device_peak(int which, double *tflops, void *stream)
{
    if (!tflops || (which != 0 && which != 1)) return IFGF_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return IFGF_ECUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // enough resident warps per SM to cover the pipes' latency; a few ms per run
    cudaError_t e = which == 0 ? time_peak<double>(st, sms * 4, 4096, tflops)
                               : time_peak<float>(st, sms * 8, 16384, tflops);
    return e == cudaSuccess ? IFGF_OK : IFGF_ECUDA;
}
