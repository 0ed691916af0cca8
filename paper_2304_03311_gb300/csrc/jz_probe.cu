// jz_probe.cu -- integer-issue probes: the measured ceilings that the
// trajectory kernel's roofline is quoted against.
//
// kind 0: independent LOP3 (three-input logic) chains
// kind 1: independent IMAD (32-bit multiply-add) chains
// kind 2: the 1:1:1 IMAD / LOP3 / IADD3 mix of the Metropolis update
// kind 3: Philox4x32-10 blocks (the random-number share of an update alone)
// Each thread runs 8 independent chains so issue, not latency, limits the rate.
// Results: thread-instructions per second (kinds 0-2) or blocks per second (3).
#include <cuda_runtime.h>

#include <cstdint>

#include "jz_device.cuh"

namespace jz {

constexpr int kProbeChains = 8;

template <int KIND>
__global__ void __launch_bounds__(256) probe_kernel(uint32_t seed, int iters, uint32_t* sink,
                                                    const PhiloxKeys K)
{
    uint32_t v[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) v[c] = seed ^ (threadIdx.x * 0x9E3779B9u + c);
    const uint32_t a = seed | 1u, b = seed * 3u + 7u;
    if constexpr (KIND == 3) {
        uint32_t acc = 0;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const uint4 u = philox(v[c] + (uint32_t)i, (uint32_t)i, blockIdx.x, (uint32_t)c, K);
                acc ^= u.x ^ u.y ^ u.z ^ u.w;
            }
        }
        if (acc == 0x12345678u) sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
    } else {
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) {
            uint32_t x = v[c];
            if (KIND == 0) {
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x) : "r"(a), "r"(b));
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x) : "r"(b), "r"(a));
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x) : "r"(a), "r"(b));
            } else if (KIND == 1) {
                asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x) : "r"(a), "r"(b));
                asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x) : "r"(b), "r"(a));
                asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x) : "r"(a), "r"(b));
            } else {
                asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x) : "r"(a), "r"(b));
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x) : "r"(b), "r"(a));
                asm volatile("add.u32 %0, %0, %1;" : "+r"(x) : "r"(a));
            }
            v[c] = x;
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) acc ^= v[c];
    if (acc == 0x12345678u) sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
    }
}

// Returns the rate, or a negative value on a CUDA error.
double run_probe(int kind, int device)
{
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return -1.0;
    const int threads = 256;
    const int blocks = prop.multiProcessorCount * (prop.maxThreadsPerMultiProcessor / threads);
    const int iters = kind == 3 ? 2000 : 4000;
    uint32_t* sink = nullptr;
    if (cudaMalloc(&sink, (size_t)blocks * threads * sizeof(uint32_t)) != cudaSuccess) return -1.0;
    PhiloxKeys K;
    for (int i = 0; i < 10; ++i) {
        K.k0[i] = 0x1234u + i * kPhiloxW0;
        K.k1[i] = 0x5678u + i * kPhiloxW1;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&]() {
        switch (kind) {
        case 0: probe_kernel<0><<<blocks, threads>>>(7u, iters, sink, K); break;
        case 1: probe_kernel<1><<<blocks, threads>>>(7u, iters, sink, K); break;
        case 2: probe_kernel<2><<<blocks, threads>>>(7u, iters, sink, K); break;
        default: probe_kernel<3><<<blocks, threads>>>(7u, iters, sink, K); break;
        }
    };
    for (int w = 0; w < 3; ++w) launch();
    const int reps = 10;
    cudaEventRecord(e0);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1);
    double rate = -1.0;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaGetLastError() == cudaSuccess) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per_thread = kind == 3 ? 2.0 * iters : 3.0 * kProbeChains * iters;
        rate = per_thread * (double)blocks * threads * reps / (ms * 1e-3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    return rate;
}

}  // namespace jz
