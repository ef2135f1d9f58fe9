// qc_main_kernel.cuh -- K2, the local-energy kernel of one molecule, as a template over its
// launch variants, with the launchers and kernel pointers of a variant set.  qc_kernels.cu
// instantiates the timed variants (DIAG = false); qc_kernels_diag.cu the same kernels with the
// pair-by-pair hit lists and work counters compiled in (DIAG = true), in a translation unit of
// their own so that the two sets compile in parallel.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "qc_device.cuh"

namespace qc {

template <int PREC, int U, bool FILTER, int LEAN, bool JOIN, bool DIAG, bool SEG = false>
__global__ void __launch_bounds__(32 * kFilteredMaxWarps) eloc_main_kernel(const __grid_constant__ SysParams sp,
                                                        const __grid_constant__ TableParams tp,
                                                        const __grid_constant__ EvalParams ep) {
    static_assert(31 + 32 * U <= kCandCap, "candidate queue too small for U");
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + kOffBar);
    uint32_t* filt = reinterpret_cast<uint32_t*>(smem + kOffVar);
    const unsigned fbytes = FILTER ? (4u << tp.fw) : 0u;
    if constexpr (FILTER) {
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            fence_barrier_init();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_expect_tx(bar, fbytes);
            constexpr unsigned kChunk = 32768;
            for (unsigned off = 0; off < fbytes; off += kChunk) {
                const unsigned n = (fbytes - off < kChunk) ? (fbytes - off) : kChunk;
                bulk_g2s(reinterpret_cast<unsigned char*>(filt) + off,
                         reinterpret_cast<const unsigned char*>(tp.filter) + off, n, bar);
            }
        }
    }
    fill_cta_tables(sp, ep.T, smem);
    if constexpr (FILTER) {
        bool ready = false;
        const unsigned limit = ep.wait_limit > 0 ? static_cast<unsigned>(ep.wait_limit - 1) : kWaitLimit;
        for (unsigned it = 0; it < limit; ++it) {
            if (mbar_try_wait(bar, 0)) {
                ready = true;
                break;
            }
        }
        if (!__syncthreads_and(ready ? 1 : 0)) {
            // the copy did not land in time: report, give it one more bounded wait, leave
            // (the whole CTA leaves together: the decision above is CTA-uniform)
            if (threadIdx.x == 0) atomicOr(&ep.ctr->flags, QC_FLAG_TIMEOUT);
            if (!ready)
                for (unsigned it = 0; it < kWaitLimit; ++it)
                    if (mbar_try_wait(bar, 0)) break;
            return;
        }
    } else {
        __syncthreads();
    }
    if (DIAG && ep.work != nullptr && threadIdx.x == 0) atomicAdd(&ep.work->ctas, 1ULL);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char* wl = smem + kOffVar + fbytes + static_cast<size_t>(warp) * main_warp_bytes(sp, FILTER, LEAN == 1, JOIN, SEG ? tp.alpha_cap : 0);
    // samples go to warps as they come free: one cursor for the grid, so a warp that drew
    // cheap samples takes more of them and the launch ends with little tail
    // with C excitation chunks per sample a work item is (sample, chunk): item = s * C + c
    const unsigned long long C = static_cast<unsigned long long>(ep.chunks > 1 ? ep.chunks : 1);
    const unsigned long long items = static_cast<unsigned long long>(ep.n_u) * C;
    while (true) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(&ep.ctr->next, 1ULL);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= items) break;
        const unsigned long long q = it / C;
        // heavy samples first when the host gave an order: the launch then ends on light ones
        const unsigned long long s =
            ep.order != nullptr ? static_cast<unsigned long long>(__ldg(ep.order + QC_IX(q, ep.n_u, sp.err))) : q;
        run_sample<PREC, U, FILTER, LEAN, JOIN, DIAG, SEG, SEG>(sp, tp, ep, static_cast<long long>(s), lane, smem, wl, filt,
                                                static_cast<int>(it - q * C), static_cast<int>(C));
    }
}

template <int PREC, int LEAN, bool DIAG>
static void launch_filtered(const SysParams& sp, const TableParams& tp, const EvalParams& ep, const LaunchCfg& c,
                            cudaStream_t s) {
    const dim3 grid(c.grid), block(32 * c.warps);
    if (c.join && c.acap > 0) eloc_main_kernel<PREC, 4, true, LEAN, true, DIAG, true><<<grid, block, c.smem, s>>>(sp, tp, ep);
    else if (c.join) eloc_main_kernel<PREC, 4, true, LEAN, true, DIAG><<<grid, block, c.smem, s>>>(sp, tp, ep);
    else if (c.unroll == 1) eloc_main_kernel<PREC, 1, true, LEAN, false, DIAG><<<grid, block, c.smem, s>>>(sp, tp, ep);
    else if (c.unroll == 2) eloc_main_kernel<PREC, 2, true, LEAN, false, DIAG><<<grid, block, c.smem, s>>>(sp, tp, ep);
    else eloc_main_kernel<PREC, 4, true, LEAN, false, DIAG><<<grid, block, c.smem, s>>>(sp, tp, ep);
}

template <int PREC, bool DIAG>
static cudaError_t launch_main_p(const SysParams& sp, const TableParams& tp, const EvalParams& ep,
                                 const LaunchCfg& c, cudaStream_t s) {
    if (c.kernel != 2) {
        eloc_main_kernel<PREC, 1, false, 0, false, DIAG><<<dim3(c.grid), dim3(32 * c.warps), c.smem, s>>>(sp, tp, ep);
    } else if (c.lean) {
        launch_filtered<PREC, 1, DIAG>(sp, tp, ep, c, s);
    } else {
        launch_filtered<PREC, 0, DIAG>(sp, tp, ep, c, s);
    }
    return cudaGetLastError();
}

// the join is built with U = 4 only; seg: its alpha list is capped (enumerated in segments)
template <int PREC, bool DIAG>
static const void* main_kernel_ptr(int kernel, int unroll, int lean, int join, int seg = 0) {
    if (kernel != 2) return (const void*)eloc_main_kernel<PREC, 1, false, 0, false, DIAG>;
    if (lean) {
        if (join && seg) return (const void*)eloc_main_kernel<PREC, 4, true, 1, true, DIAG, true>;
        if (join) return (const void*)eloc_main_kernel<PREC, 4, true, 1, true, DIAG>;
        if (unroll == 1) return (const void*)eloc_main_kernel<PREC, 1, true, 1, false, DIAG>;
        if (unroll == 2) return (const void*)eloc_main_kernel<PREC, 2, true, 1, false, DIAG>;
        return (const void*)eloc_main_kernel<PREC, 4, true, 1, false, DIAG>;
    }
    if (join && seg) return (const void*)eloc_main_kernel<PREC, 4, true, 0, true, DIAG, true>;
    if (join) return (const void*)eloc_main_kernel<PREC, 4, true, 0, true, DIAG>;
    if (unroll == 1) return (const void*)eloc_main_kernel<PREC, 1, true, 0, false, DIAG>;
    if (unroll == 2) return (const void*)eloc_main_kernel<PREC, 2, true, 0, false, DIAG>;
    return (const void*)eloc_main_kernel<PREC, 4, true, 0, false, DIAG>;
}

template <bool DIAG>
static cudaError_t launch_main_variant(const SysParams& sp, const TableParams& tp, const EvalParams& ep,
                                       const LaunchCfg& c, cudaStream_t s) {
    return sp.precision == QC_FP64 ? launch_main_p<QC_FP64, DIAG>(sp, tp, ep, c, s)
                                   : launch_main_p<QC_FP32_COMP, DIAG>(sp, tp, ep, c, s);
}

template <bool DIAG>
static cudaError_t prepare_variant(size_t max_smem) {
    const int v = static_cast<int>(max_smem);
    cudaError_t e = cudaSuccess;
    for (int prec = 0; prec < 2; ++prec)
        for (int kernel = 1; kernel <= 2; ++kernel)
            for (int unroll : {1, 2, 4})
                for (int lean = 0; lean < 2; ++lean)
                    for (int join = 0; join < 3; ++join) {
                        const void* f = prec == QC_FP64 ? main_kernel_ptr<QC_FP64, DIAG>(kernel, unroll, lean, join > 0, join == 2)
                                                        : main_kernel_ptr<QC_FP32_COMP, DIAG>(kernel, unroll, lean, join > 0, join == 2);
                        const cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
                        if (r != cudaSuccess) e = r;
                    }
    return e;
}

}  // namespace qc
