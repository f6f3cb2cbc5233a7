// xm_peaks.cu -- measured ceilings for the roofline of the scan (no
// counterpart in the paper): float32 FMA rate, float64 FMA rate and
// read-only HBM bandwidth of the current device, each the best of several
// event-timed launches on the caller's stream.
//
// The FMA kernels run eight independent dependent chains per thread on every
// lane of a full grid (enough warps to cover the pipe latency), with the
// multiplier and addend passed at run time so nothing folds; the chains end
// in a store that no input makes true, so nothing is dead code. The read
// kernel streams a buffer larger than L2 with 16-byte loads, four in flight
// per thread, and folds them into one word per thread.

#include <stdint.h>

#include "xm_internal.cuh"

namespace xm {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_peak_fma(T m, T c, int iters, T* sink) {
    T x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = (T)(threadIdx.x + k);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
#pragma unroll
            for (int k = 0; k < kChains; k++) x[k] = fma(x[k], m, c);
        }
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += x[k];
    if (s == (T)-1.0) sink[blockIdx.x] = s;  // never true for the inputs used
}

__global__ void __launch_bounds__(512) k_peak_read(const int4* __restrict__ p, int64_t n4,
                                                   uint32_t* sink) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint32_t acc = 0;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n4; i += 4 * stride) {
        const int4 a = __ldcs(p + i), b = __ldcs(p + i + stride), c = __ldcs(p + i + 2 * stride),
                   d = __ldcs(p + i + 3 * stride);
        acc ^= (uint32_t)(a.x ^ a.y ^ a.z ^ a.w) ^ (uint32_t)(b.x ^ b.y ^ b.z ^ b.w) ^
               (uint32_t)(c.x ^ c.y ^ c.z ^ c.w) ^ (uint32_t)(d.x ^ d.y ^ d.z ^ d.w);
    }
    for (; i < n4; i += stride) {
        const int4 a = __ldcs(p + i);
        acc ^= (uint32_t)(a.x ^ a.y ^ a.z ^ a.w);
    }
    if (acc == 0x9E3779B9u) sink[0] = acc;  // the buffer is zero: never true
}

// Best device time (ms) of `reps` launches of f (after one untimed launch).
template <typename F>
cudaError_t best_ms(F f, cudaStream_t s, int reps, float* out) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    float best = 1e30f;
    for (int r = 0; r <= reps && e == cudaSuccess; r++) {
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) f();
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *out = best;
    return e;
}

}  // namespace
}  // namespace xm

extern "C" xm_status xm_measure_peak(int32_t what, double* value, void* stream) {
    using namespace xm;
    if (!value) return set_error(XM_EINVAL, "xm_measure_peak: value is NULL");
    *value = 0.0;
    if (what < XM_PEAK_FP32_FMA || what > XM_PEAK_HBM_READ)
        return set_error(XM_EINVAL, "xm_measure_peak: unknown quantity %d", what);
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "xm_measure_peak: device");
    const int reps = 5;
    float ms = 0.0f;
    if (what == XM_PEAK_FP32_FMA || what == XM_PEAK_FP64_FMA) {
        const bool f32 = what == XM_PEAK_FP32_FMA;
        // full occupancy: 8 blocks of 256 threads per SM; float64 runs at a
        // small fraction of the float32 rate, so it gets fewer iterations
        const int blocks = 8 * sms, iters = f32 ? 4096 : 64;
        void* sink = dev_alloc(blocks * sizeof(double), s);
        if (!sink) return set_error(XM_ENOMEM, "xm_measure_peak: sink");
        if (f32)
            e = best_ms([&] { k_peak_fma<float><<<blocks, kPeakThreads, 0, s>>>(0.99999994f, 1e-7f, iters, (float*)sink); },
                        s, reps, &ms);
        else
            e = best_ms([&] { k_peak_fma<double><<<blocks, kPeakThreads, 0, s>>>(0.9999999999999999, 1e-15, iters, (double*)sink); },
                        s, reps, &ms);
        dev_free(sink, s);
        if (e != cudaSuccess) return cuda_fail(e, "xm_measure_peak: fma");
        const double fmas = (double)blocks * kPeakThreads * iters * kUnroll * kChains;
        *value = 2.0 * fmas / (ms * 1e-3) / 1e12;  // TFLOP/s
        return XM_OK;
    }
    // read-only HBM: 4 GiB, far beyond the 129 MB L2
    const size_t bytes = (size_t)4 << 30;
    void* buf = dev_alloc(bytes, s);
    uint32_t* sink = (uint32_t*)dev_alloc(sizeof(uint32_t), s);
    if (!buf || !sink) {
        dev_free(buf, s);
        dev_free(sink, s);
        return set_error(XM_ENOMEM, "xm_measure_peak: %zu-byte buffer", bytes);
    }
    e = cudaMemsetAsync(buf, 0, bytes, s);
    const int64_t n4 = (int64_t)(bytes / sizeof(int4));
    if (e == cudaSuccess)
        e = best_ms([&] { k_peak_read<<<4 * sms, 512, 0, s>>>((const int4*)buf, n4, sink); }, s, reps, &ms);
    dev_free(buf, s);
    dev_free(sink, s);
    if (e != cudaSuccess) return cuda_fail(e, "xm_measure_peak: read");
    *value = (double)bytes / (ms * 1e-3) / 1e9;  // GB/s
    return XM_OK;
}
