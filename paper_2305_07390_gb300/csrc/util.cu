// util.cu -- reduction fold and device microbenchmarks.
//
// The microbenchmarks measure the throughputs the cost model of Section 5 and
// the roofline need (Section 6.1 measures latency and throughput to apply
// Little's law): FP64 and FP32 FMA rates, shared-memory load bandwidth and the
// cost of a device-wide barrier (the paper's T_Dsync, Section 5.2.2).
#include <cstdio>

#include "dispatch.h"
#include "stencil.cuh"

namespace ebisu {

// Fold the per-block partials (sum, sum of squares, max) in a fixed order.
__global__ void reduce_final_kernel(const double* part, int64_t n, double* out)
{
    __shared__ double s0[256], s1[256], s2[256];
    double a = 0.0, b = 0.0, c = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 256) {
        a += part[3 * i + 0];
        b += part[3 * i + 1];
        c = fmax(c, part[3 * i + 2]);
    }
    s0[threadIdx.x] = a;
    s1[threadIdx.x] = b;
    s2[threadIdx.x] = c;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s0[threadIdx.x] += s0[threadIdx.x + w];
            s1[threadIdx.x] += s1[threadIdx.x + w];
            s2[threadIdx.x] = fmax(s2[threadIdx.x], s2[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = s0[0];
        out[1] = sqrt(s1[0]);
        out[2] = s2[0];
    }
}

cudaError_t reduce_final(const double* part, int64_t nparts, double* out3_dev, cudaStream_t st)
{
    reduce_final_kernel<<<1, 256, 0, st>>>(part, nparts, out3_dev);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// microbenchmarks

template <int CH>
__global__ void probe_dfma(double* sink, int iters, double b, double c)
{
    double a[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) a[i] = threadIdx.x * 1e-3 + i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < CH; ++i) a[i] = fma(a[i], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += a[i];
    if (s == 1234.5678) sink[0] = s;
}

template <int CH>
__global__ void probe_ffma(float* sink, int iters, float b, float c)
{
    float a[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) a[i] = threadIdx.x * 1e-3f + i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < CH; ++i) a[i] = fmaf(a[i], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += a[i];
    if (s == 1234.5678f) sink[0] = s;
}

// 16-byte shared loads folded with integer XOR (no FP pipe in the way).
__global__ void probe_lds(unsigned* sink, int iters)
{
    __shared__ uint4 sm[2048];
    for (int i = threadIdx.x; i < 2048; i += blockDim.x) sm[i] = make_uint4(i, i + 1, i + 2, i + 3);
    __syncthreads();
    uint4 acc = make_uint4(0, 0, 0, 0);
    const int base = threadIdx.x;
    for (int it = 0; it < iters; ++it) {
        const int o = (it * 64) & 1023;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint4 v = sm[(base + o + u * 512) & 2047];
            acc.x ^= v.x; acc.y ^= v.y; acc.z ^= v.z; acc.w ^= v.w;
        }
    }
    if ((acc.x ^ acc.y ^ acc.z ^ acc.w) == 0x12345678u) sink[0] = acc.x;
}

// Device-wide barrier rounds with the same bounded-spin counter scheme the
// persistent kernels use between dependent items.
__global__ void probe_barrier(unsigned* counter, int* err, int rounds, int64_t timeout_ns)
{
    for (int r = 0; r < rounds; ++r) {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            red_release_add_u32(counter, 1u);
            const unsigned target = (unsigned)(r + 1) * gridDim.x;
            const uint64_t t0 = global_ns();
            while (ld_acquire_u32(counter) < target) {
                if (global_ns() - t0 > (uint64_t)timeout_ns) {
                    atomicExch(err, 1);
                    break;
                }
            }
        }
        __syncthreads();
        if (*(volatile int*)err) return;
    }
}

__global__ void probe_clock(long long* out)
{
    const long long c0 = clock64();
    const uint64_t t0 = global_ns();
    long long c1;
    uint64_t t1;
    do {
        c1 = clock64();
        t1 = global_ns();
    } while (t1 - t0 < 2000000ull);
    out[0] = c1 - c0;
    out[1] = (long long)(t1 - t0);
}

static float time_launch(cudaEvent_t e0, cudaEvent_t e1, void (*fn)(void*), void* ctx)
{
    fn(ctx);  // warm
    cudaEventRecord(e0);
    fn(ctx);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
}

cudaError_t probe_device(double* out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    void* buf = nullptr;
    e = cudaMalloc(&buf, 4096);
    if (e != cudaSuccess) return e;
    cudaMemset(buf, 0, 4096);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    struct Ctx { void* buf; int sms; } ctx{buf, sms};

    const int dit = 4000, fit = 100000, lit = 20000;
    float ms = time_launch(e0, e1, [](void* c) {
        auto* x = (Ctx*)c;
        probe_dfma<8><<<x->sms * 2, 512>>>((double*)x->buf, 4000, 0.999, 1e-3);
    }, &ctx);
    out[0] = 2.0 * 8 * dit * 512.0 * 2 * sms / (ms * 1e-3);
    ms = time_launch(e0, e1, [](void* c) {
        auto* x = (Ctx*)c;
        probe_ffma<8><<<x->sms * 2, 512>>>((float*)x->buf, 100000, 0.999f, 1e-3f);
    }, &ctx);
    out[1] = 2.0 * 8 * fit * 512.0 * 2 * sms / (ms * 1e-3);
    ms = time_launch(e0, e1, [](void* c) {
        auto* x = (Ctx*)c;
        probe_lds<<<x->sms * 2, 512>>>((unsigned*)x->buf, 20000);
    }, &ctx);
    out[2] = 16.0 * 4 * lit * 512.0 * 2 * sms / (ms * 1e-3);
    // barrier: one 256-thread CTA per SM, 2000 rounds
    {
        unsigned* counter = (unsigned*)((char*)buf + 1024);
        int* err = (int*)((char*)buf + 2048);
        cudaMemset((char*)buf + 1024, 0, 2048);
        probe_barrier<<<sms, 256>>>(counter, err, 10, 2000000000LL);
        cudaDeviceSynchronize();
        cudaMemset((char*)buf + 1024, 0, 2048);
        cudaEventRecord(e0);
        probe_barrier<<<sms, 256>>>(counter, err, 2000, 2000000000LL);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        out[3] = ms * 1e-3 / 2000.0;
    }
    out[4] = sms;
    {
        long long h[2] = {0, 0};
        probe_clock<<<1, 1>>>((long long*)buf);
        cudaMemcpy(h, buf, sizeof(h), cudaMemcpyDeviceToHost);
        out[5] = h[1] > 0 ? (double)h[0] / (double)h[1] * 1e9 : 0.0;
    }
    e = cudaDeviceSynchronize();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

}  // namespace ebisu
