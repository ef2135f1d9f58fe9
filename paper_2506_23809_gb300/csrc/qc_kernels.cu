// qc_kernels.cu -- the single-molecule kernels of libqc_eloc (sm_103a) and their launchers:
// K0 table build, K2 local-energy kernel (filtered and unfiltered), K3 reduction.  The
// device code they share with the batch kernels is in qc_device.cuh.
#include <cstdint>
#include <cuda_runtime.h>

#include "qc_device.cuh"

namespace qc {

int reduce_blocks(long long n) {
    long long b = (n + kRedThreads * 8 - 1) / (kRedThreads * 8);
    if (b < 1) b = 1;
    if (b > 1024) b = 1024;
    return static_cast<int>(b);
}

size_t smem_fixed_bytes() { return kOffVar; }

size_t filtered_smem_bytes(const SysParams& sp, int warps, int fw, bool lean, bool join) {
    return kOffVar + (static_cast<size_t>(4) << fw) + static_cast<size_t>(warps) * main_warp_bytes(sp, true, lean, join);
}
size_t direct_smem_bytes(const SysParams& sp, int warps) {
    return kOffVar + static_cast<size_t>(warps) * main_warp_bytes(sp, false);
}

__global__ void __launch_bounds__(256) build_table_kernel(TableParams tp, int n_orb, int na, int nb,
                                                          const unsigned long long* __restrict__ T,
                                                          unsigned long long* slots,
                                                          uint32_t* filter, unsigned long long* aset,
                                                          unsigned long long* bset, Counters* ctr,
                                                          unsigned* jkey, unsigned* jlen) {
    const long long r = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r < tp.n) build_one(tp, n_orb, na, nb, T, slots, filter, aset, bset, ctr, r, jkey, jlen, 0u,
                            2u * (tp.set_mask + 1u));
}

template <int PREC, int U, bool FILTER, int LEAN, bool JOIN>
__global__ void __launch_bounds__(640) eloc_main_kernel(const __grid_constant__ SysParams sp,
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
        for (unsigned it = 0; it < kWaitLimit; ++it) {
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
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char* wl = smem + kOffVar + fbytes + static_cast<size_t>(warp) * main_warp_bytes(sp, FILTER, LEAN == 1, JOIN);
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
        const unsigned long long s = ep.order != nullptr ? static_cast<unsigned long long>(__ldg(ep.order + q)) : q;
        run_sample<PREC, U, FILTER, LEAN, JOIN>(sp, tp, ep, static_cast<long long>(s), lane, smem, wl, filt,
                                                static_cast<int>(it - q * C), static_cast<int>(C));
    }
}

__global__ void __launch_bounds__(kRedThreads) reduce_pass1(EvalParams ep, double* part) {
    reduce_pass1_body(ep, part, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kRedThreads) reduce_pass2(EvalParams ep, double* part,
                                                            qc_eloc_summary* out, long long pairs_per_sample) {
    reduce_pass2_body(ep, part, out, pairs_per_sample, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------------------------------
// host launchers
// ------------------------------------------------------------------------------------
cudaError_t launch_build_table(const TableParams& tp, int n_orb, int na, int nb,
                               const unsigned long long* T, unsigned long long* slots,
                               uint32_t* filter, unsigned long long* aset,
                               unsigned long long* bset, Counters* ctr, cudaStream_t s, unsigned* jkey,
                               unsigned* jlen) {
    if (tp.n <= 0) return cudaSuccess;
    const long long blocks = (tp.n + 255) / 256;
    build_table_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(tp, n_orb, na, nb, T, slots,
                                                                      filter, aset, bset, ctr, jkey, jlen);
    return cudaGetLastError();
}

template <int PREC, int LEAN>
static void launch_filtered(const SysParams& sp, const TableParams& tp, const EvalParams& ep, const LaunchCfg& c,
                            cudaStream_t s) {
    const dim3 grid(c.grid), block(32 * c.warps);
    if (c.join) eloc_main_kernel<PREC, 4, true, LEAN, true><<<grid, block, c.smem, s>>>(sp, tp, ep);
    else if (c.unroll == 1) eloc_main_kernel<PREC, 1, true, LEAN, false><<<grid, block, c.smem, s>>>(sp, tp, ep);
    else if (c.unroll == 2) eloc_main_kernel<PREC, 2, true, LEAN, false><<<grid, block, c.smem, s>>>(sp, tp, ep);
    else eloc_main_kernel<PREC, 4, true, LEAN, false><<<grid, block, c.smem, s>>>(sp, tp, ep);
}

template <int PREC>
static cudaError_t launch_main_p(const SysParams& sp, const TableParams& tp, const EvalParams& ep,
                                 const LaunchCfg& c, cudaStream_t s) {
    if (c.kernel != 2) {
        eloc_main_kernel<PREC, 1, false, 0, false><<<dim3(c.grid), dim3(32 * c.warps), c.smem, s>>>(sp, tp, ep);
    } else if (c.lean) {
        launch_filtered<PREC, 1>(sp, tp, ep, c, s);
    } else {
        launch_filtered<PREC, 0>(sp, tp, ep, c, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_eloc_main(const SysParams& sp, const TableParams& tp, const EvalParams& ep,
                             const LaunchCfg& c, cudaStream_t s) {
    if (ep.n_u <= 0) return cudaSuccess;
    return sp.precision == QC_FP64 ? launch_main_p<QC_FP64>(sp, tp, ep, c, s)
                                   : launch_main_p<QC_FP32_COMP>(sp, tp, ep, c, s);
}

cudaError_t launch_reduce(const EvalParams& ep, double* partials, int nblk, void* summary_dev,
                          long long pairs_per_sample, cudaStream_t s) {
    reduce_pass1<<<nblk, kRedThreads, 0, s>>>(ep, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_pass2<<<nblk, kRedThreads, 0, s>>>(ep, partials,
                                              static_cast<qc_eloc_summary*>(summary_dev), pairs_per_sample);
    return cudaGetLastError();
}

// the join is built with U = 4 only
template <int PREC>
static const void* main_kernel_ptr(int kernel, int unroll, int lean, int join) {
    if (kernel != 2) return (const void*)eloc_main_kernel<PREC, 1, false, 0, false>;
    if (lean) {
        if (join) return (const void*)eloc_main_kernel<PREC, 4, true, 1, true>;
        if (unroll == 1) return (const void*)eloc_main_kernel<PREC, 1, true, 1, false>;
        if (unroll == 2) return (const void*)eloc_main_kernel<PREC, 2, true, 1, false>;
        return (const void*)eloc_main_kernel<PREC, 4, true, 1, false>;
    }
    if (join) return (const void*)eloc_main_kernel<PREC, 4, true, 0, true>;
    if (unroll == 1) return (const void*)eloc_main_kernel<PREC, 1, true, 0, false>;
    if (unroll == 2) return (const void*)eloc_main_kernel<PREC, 2, true, 0, false>;
    return (const void*)eloc_main_kernel<PREC, 4, true, 0, false>;
}

int max_active_ctas(int kernel, int precision, int unroll, int threads, size_t smem, int lean, int join) {
    const void* f = precision == QC_FP64 ? main_kernel_ptr<QC_FP64>(kernel, unroll, lean, join)
                                         : main_kernel_ptr<QC_FP32_COMP>(kernel, unroll, lean, join);
    int n = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, threads, smem) == cudaSuccess ? n : 0;
}

cudaError_t prepare_kernels(size_t max_smem) {
    const int v = static_cast<int>(max_smem);
    cudaError_t e = cudaSuccess;
    for (int prec = 0; prec < 2; ++prec)
        for (int kernel = 1; kernel <= 2; ++kernel)
            for (int unroll : {1, 2, 4})
                for (int lean = 0; lean < 2; ++lean)
                    for (int join = 0; join < 2; ++join) {
                        const void* f = prec == QC_FP64 ? main_kernel_ptr<QC_FP64>(kernel, unroll, lean, join)
                                                        : main_kernel_ptr<QC_FP32_COMP>(kernel, unroll, lean, join);
                        const cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
                        if (r != cudaSuccess) e = r;
                    }
    return e;
}

}  // namespace qc
