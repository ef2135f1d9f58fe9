// qc_kernels.cu -- the single-molecule kernels of libqc_eloc (sm_103a) and their launchers:
// K0 table build, K2 local-energy kernel (filtered and unfiltered; the template is in
// qc_main_kernel.cuh, its diagnostic instantiations in qc_kernels_diag.cu), K3 reduction.  The
// device code they share with the batch kernels is in qc_device.cuh.
#include <cstdint>
#include <cuda_runtime.h>

#include "qc_main_kernel.cuh"

namespace qc {

int reduce_blocks(long long n) {
    // two rows per thread: enough blocks that every SM has a few (latency-bound loads)
    long long b = (n + kRedThreads * 2 - 1) / (kRedThreads * 2);
    if (b < 1) b = 1;
    if (b > 1024) b = 1024;
    return static_cast<int>(b);
}

size_t smem_fixed_bytes() { return kOffVar; }

size_t filtered_smem_bytes(const SysParams& sp, int warps, int fw, bool lean, bool join, int acap) {
    return kOffVar + (static_cast<size_t>(4) << fw) +
           static_cast<size_t>(warps) * main_warp_bytes(sp, true, lean, join, join ? acap : 0);
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

__global__ void __launch_bounds__(kRedThreads) reduce_pass1(EvalParams ep, double* part) {
    reduce_pass1_body(ep, part, blockIdx.x, gridDim.x, 0, ep.n_u);
}
__global__ void __launch_bounds__(kRedThreads) reduce_pass2(EvalParams ep, double* part,
                                                            qc_eloc_summary* out, long long pairs_per_sample) {
    reduce_pass2_body(ep, part, out, pairs_per_sample, blockIdx.x, gridDim.x, 0, ep.n_u);
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

cudaError_t launch_eloc_main(const SysParams& sp, const TableParams& tp, const EvalParams& ep,
                             const LaunchCfg& c, cudaStream_t s) {
    if (ep.n_u <= 0) return cudaSuccess;
    // per-sample digests, hit lists or work counters asked for: the diagnostic instantiations
    // (qc_kernels_diag.cu)
    if (ep.hit_count != nullptr || ep.hit_rowsum != nullptr || ep.hit_signsum != nullptr || ep.hit_list != nullptr ||
        ep.work != nullptr)
        return launch_eloc_main_diag(sp, tp, ep, c, s);
    return launch_main_variant<false>(sp, tp, ep, c, s);
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

int max_active_ctas(int kernel, int precision, int unroll, int threads, size_t smem, int lean, int join, int seg) {
    const void* f = precision == QC_FP64 ? main_kernel_ptr<QC_FP64, false>(kernel, unroll, lean, join, seg)
                                         : main_kernel_ptr<QC_FP32_COMP, false>(kernel, unroll, lean, join, seg);
    int n = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, threads, smem) == cudaSuccess ? n : 0;
}

cudaError_t prepare_kernels(size_t max_smem) {
    const cudaError_t e = prepare_variant<false>(max_smem);
    const cudaError_t d = prepare_kernels_diag(max_smem);
    return e != cudaSuccess ? e : d;
}

}  // namespace qc
