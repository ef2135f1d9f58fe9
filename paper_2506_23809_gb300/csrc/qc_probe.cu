// qc_probe.cu -- measurement probes for the rooflines the benchmark reports beside the
// local-energy kernel (no counterpart in the paper).
//   alu probe:        every thread runs eight independent chains of the filter test's
//                     integer operations (a right shift, a funnel shift by it, a second
//                     shift and an XOR: 4 ALU-pipe operations per link); the achieved rate is
//                     the integer throughput a kernel of that mix can reach on this GPU
//   L2 gather probe:  random 16-byte loads from a table that fits in L2 (the bucket-probe
//                     pattern of the main kernel), eight loads in flight per thread
// Both are timed with CUDA events around one launch after a warm-up launch.
#include <cuda_runtime.h>

#include <cstdint>

#include "qc_eloc.h"
#include "qc_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kAluOpsPerLink = 4;

__global__ void __launch_bounds__(256) alu_probe_kernel(uint32_t* out, int iters, uint32_t seed) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed ^ (t * 0x9E3779B9u) ^ (0x85EBCA6Bu * (c + 1));
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            const uint32_t s = a[c] >> 27;
            a[c] = __funnelshift_r(a[c], a[c], s) ^ (a[c] >> 22);
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) r ^= a[c];
    if (r == seed) out[t & 1023u] = r;  // keeps the chains live; almost never taken
}

__global__ void __launch_bounds__(256) l2_fill_kernel(ulonglong2* tab, unsigned n) {
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        tab[i] = make_ulonglong2(i * 0x9E3779B97F4A7C15ULL, i);
}

__global__ void __launch_bounds__(256) l2_gather_kernel(const ulonglong2* __restrict__ tab, unsigned mask,
                                                        int iters, unsigned long long* out) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = t * 2654435761u + 0x632BE5ABu * (c + 1);
    unsigned long long acc = 0;
    for (int i = 0; i < iters; ++i) {
        ulonglong2 v[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            x[c] = x[c] * 1664525u + 1013904223u;
            v[c] = __ldcg(tab + ((x[c] >> 7) & mask));
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) acc ^= v[c].x + v[c].y;
    }
    if (acc == 0x1234567ULL) out[t & 1023u] = acc;
}

}  // namespace

extern "C" qc_status qc_probe_peaks(double* alu_ops_per_s, double* l2_gather_gbs, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    uint32_t* sink = nullptr;
    ulonglong2* tab = nullptr;
    const unsigned entries = 1u << 18;  // 4 MB: resident in L2 like the main kernel's bucket table
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMalloc(&sink, 1024 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&tab, entries * sizeof(ulonglong2));
    const unsigned blocks = static_cast<unsigned>(sms) * 8;  // 2,048 threads per SM
    if (e == cudaSuccess && alu_ops_per_s) {
        const int iters = 4096;
        alu_probe_kernel<<<blocks, 256, 0, s>>>(sink, iters / 8, 1u);  // warm-up
        e = cudaEventRecord(e0, s);
        alu_probe_kernel<<<blocks, 256, 0, s>>>(sink, iters, 1u);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess)
            *alu_ops_per_s = static_cast<double>(blocks) * 256.0 * iters * kChains * kAluOpsPerLink / (ms * 1e-3);
    }
    if (e == cudaSuccess && l2_gather_gbs) {
        l2_fill_kernel<<<blocks, 256, 0, s>>>(tab, entries);
        const int iters = 256;
        l2_gather_kernel<<<blocks, 256, 0, s>>>(tab, entries - 1, iters / 8,
                                                reinterpret_cast<unsigned long long*>(sink));
        e = cudaEventRecord(e0, s);
        l2_gather_kernel<<<blocks, 256, 0, s>>>(tab, entries - 1, iters, reinterpret_cast<unsigned long long*>(sink));
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess) *l2_gather_gbs = static_cast<double>(blocks) * 256.0 * iters * 8 * 16 / (ms * 1e-3) / 1e9;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (tab) cudaFree(tab);
    return e == cudaSuccess ? QC_OK : QC_ERR_CUDA;
}
