// Arithmetic peaks of the current device, measured by short isolated kernels: the roofline
// denominators of the kernels that are bound by FP32 / FP64 FMAs or by tcgen05 kind::tf32
// products (the memory-bound kernels use the measured copy bandwidth instead).  No counterpart
// in the paper.
#include <stdint.h>
#include <stdio.h>

#include "tcgen05.cuh"
#include "arkcos_peaks.h"

namespace arkcos {

namespace {

using namespace tc;

constexpr int kChains = 16;  // independent FMA chains per thread (covers the FMA latency)

// FP32 FMAs: every thread runs kChains independent chains x = x a + b, `iters` times.
__global__ void __launch_bounds__(256) k_peak_ffma(float *out, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1e-3f * (float)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == -1.f) out[blockIdx.x] = s;  // never true; keeps the chains alive
}

// The same with packed two-lane FP32 FMAs (two FMAs per instruction).
__global__ void __launch_bounds__(256) k_peak_ffma2(float *out, int iters, float a, float b)
{
    float2 x[kChains / 2];
#pragma unroll
    for (int i = 0; i < kChains / 2; ++i) x[i] = make_float2(1e-3f * (float)(threadIdx.x + i), 2e-3f * (float)i);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains / 2; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains / 2; ++i) s += x[i].x + x[i].y;
    if (s == -1.f) out[blockIdx.x] = s;
}

// FP64 FMAs.
__global__ void __launch_bounds__(256) k_peak_dfma(float *out, int iters, double a, double b)
{
    double x[kChains / 2];
#pragma unroll
    for (int i = 0; i < kChains / 2; ++i) x[i] = 1e-3 * (double)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains / 2; ++i) x[i] = fma(x[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains / 2; ++i) s += x[i];
    if (s == -1.0) out[blockIdx.x] = (float)s;
}

// tcgen05.mma kind::tf32, M = 128, N = 256, K = 8 (the shape of the library's tensor-core
// kernels): one CTA per SM, one thread issues 4 `iters` MMAs from operands in shared memory
// (A 16 KiB, B 32 KiB in the no-swizzle K-major layout, filled with TF32 values) into one
// 256-column accumulator, then commits once; every thread waits for the completion (bounded),
// and the accumulator is released.  A wait that gives up sets *err.
constexpr uint32_t kPkA = 16384, kPkB = 32768;

__global__ void __launch_bounds__(128, 1) k_peak_tf32_mma(float *out, int *err, int iters)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *A = smem, *B = smem + kPkA;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kPkA + kPkB);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + kPkA + kPkB + 8);
    const int tid = threadIdx.x, warp = tid >> 5;
    // operands: TF32 values of a fixed hash of the byte offset
    for (uint32_t e = tid; e < (kPkA + kPkB) / 4; e += blockDim.x) {
        const uint32_t h = (e * 2654435761u) >> 9;
        reinterpret_cast<float *>(smem)[e] = tf32_round(1.0f + (float)(h & 1023) * (1.0f / 1024.0f));
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"((uint32_t)__cvta_generic_to_shared(tslot)), "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t bar_s = (uint32_t)__cvta_generic_to_shared(bar);
    if (tid == 0) {
        const uint32_t idesc = tf32_idesc(128, 256);
        const uint32_t sa = (uint32_t)__cvta_generic_to_shared(A), sb = (uint32_t)__cvta_generic_to_shared(B);
        for (int it = 0; it < iters; ++it)
            for (int ks = 0; ks < 4; ++ks) {
                const uint32_t o = (uint32_t)ks * 2 * kLBO;
                mma_tf32(tmem, smem_desc(sa + o), smem_desc(sb + o), idesc, (it | ks) ? 1 : 0);
            }
        mma_commit(bar_s);
    }
    bool ok = mbar_wait(bar_s, 0);
    if (!ok) ok = mbar_wait(bar_s, 0);  // the issued MMAs may still complete: wait once more
    ok = __syncthreads_and(ok);
    if (!ok && tid == 0) atomicOr(err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {  // CTA-uniform: every warp reads its lane quarter (warp-collective load)
        uint32_t v[8];
        tmem_ld_async(tmem + ((uint32_t)(warp * 32) << 16), v);
        tmem_wait_ld();
        if ((tid & 31) == 0 && __uint_as_float(v[0]) == -1.f) out[blockIdx.x] = 0.f;  // keeps the products observable
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

}  // namespace

// Times `reps` launches of a kernel (after one warm-up) with CUDA events; returns the best.
template <class F>
cudaError_t time_best(F launch, int reps, cudaStream_t st, float *best_ms)
{
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    float best = 1e30f;
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        float t = 0.f;
        if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
        if (r > 0 && t < best) best = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *best_ms = best;
    return e;
}

cudaError_t measure_peak(int unit, double *tflops, double *ms, cudaStream_t st)
{
    const int sms = device_sms();
    float *out = nullptr;
    int *err = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(float) * 8 * (size_t)sms);
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&err, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(out);
        return e;
    }
    cudaMemsetAsync(err, 0, sizeof(int), st);
    float best = 0.f;
    double flop = 0.0;
    if (unit == 0 || unit == 1 || unit == 2) {
        const int blocks = sms * 8, threads = 256;
        const int iters = unit == 2 ? 1 << 12 : 1 << 15;
        const double per_thread = unit == 2 ? 2.0 * (kChains / 2) * iters : 2.0 * kChains * iters;
        flop = per_thread * blocks * threads;
        auto launch = [&]() {
            if (unit == 0) k_peak_ffma<<<blocks, threads, 0, st>>>(out, iters, 0.9999999f, 1e-7f);
            else if (unit == 1) k_peak_ffma2<<<blocks, threads, 0, st>>>(out, iters, 0.9999999f, 1e-7f);
            else k_peak_dfma<<<blocks, threads, 0, st>>>(out, iters, 0.9999999, 1e-7);
        };
        e = time_best(launch, 5, st, &best);
    } else {
        const size_t smem = 200 * 1024;  // one CTA per SM
        e = cudaFuncSetAttribute((const void *)k_peak_tf32_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const int iters = 1 << 14;
        flop = 2.0 * 128 * 256 * 8 * 4.0 * iters * sms;
        auto launch = [&]() { k_peak_tf32_mma<<<sms, 128, smem, st>>>(out, err, iters); };
        if (e == cudaSuccess) e = time_best(launch, 5, st, &best);
        int herr = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && herr) e = cudaErrorLaunchTimeout;
    }
    cudaFree(out);
    cudaFree(err);
    if (e != cudaSuccess) return e;
    *ms = best;
    *tflops = flop / (best * 1e-3) / 1e12;
    return cudaSuccess;
}

}  // namespace arkcos

extern "C" arkcos_status arkcos_measure_peak(int unit, double *tflops, double *ms, void *stream)
{
    if (!tflops || !ms || unit < 0 || unit > 3) {
        arkcos::set_last_error("arkcos_measure_peak: unit must be 0..3 and tflops, ms non-NULL");
        return ARKCOS_EINVAL;
    }
    const cudaError_t e = arkcos::measure_peak(unit, tflops, ms, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof(msg), "arkcos_measure_peak: %s", cudaGetErrorString(e));
        arkcos::set_last_error(msg);
        return e == cudaErrorLaunchTimeout ? ARKCOS_ETIMEOUT : ARKCOS_ECUDA;
    }
    return ARKCOS_OK;
}
