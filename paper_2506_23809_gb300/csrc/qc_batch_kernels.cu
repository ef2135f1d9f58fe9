// qc_batch_kernels.cu -- many molecules in one launch (sm_103a): batched table build,
// the persistent multi-molecule local-energy kernel, and the batched reduction.
#include <cstdint>
#include <cuda_runtime.h>

#include "qc_device.cuh"

namespace qc {

// Every molecule of a batch: thread -> (molecule, row) through the prefix of table sizes.
__global__ void __launch_bounds__(256) build_batch_kernel(const MolParams* __restrict__ mols,
                                                          const MolWork* __restrict__ work,
                                                          const long long* __restrict__ key_off,
                                                          int n_mol, long long n_keys) {
    const long long g = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= n_keys) return;
    int lo = 0, hi = n_mol;  // largest m with key_off[m] <= g
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (key_off[mid] <= g) lo = mid; else hi = mid;
    }
    const MolParams& P = mols[lo];
    const MolWork& W = work[lo];
    build_one(P.tp, P.sp.n_orb, P.sp.na, P.sp.nb, P.ep.T, W.slots, W.filter, W.aset, W.bset, W.ctr,
              g - key_off[lo], W.jkey, W.jlen, W.jbase, W.jsent, W.jval);
}

// batch: blockIdx.y is the molecule
__global__ void __launch_bounds__(kRedThreads) reduce_batch_pass1(const MolParams* __restrict__ mols,
                                                                  const MolWork* __restrict__ work) {
    const MolWork& W = work[blockIdx.y];
    if (blockIdx.x >= static_cast<unsigned>(W.nblk)) return;  // block-uniform
    const MolParams& P = mols[blockIdx.y];
    reduce_pass1_body(P.ep, W.part, blockIdx.x, W.nblk, P.red_lo, P.red_hi);
}
__global__ void __launch_bounds__(kRedThreads) reduce_batch_pass2(const MolParams* __restrict__ mols,
                                                                  const MolWork* __restrict__ work) {
    const MolParams& P = mols[blockIdx.y];
    const MolWork& W = work[blockIdx.y];
    if (blockIdx.x >= static_cast<unsigned>(W.nblk)) return;  // block-uniform
    reduce_pass2_body(P.ep, W.part, static_cast<qc_eloc_summary*>(W.sum), P.sp.pairs, blockIdx.x, W.nblk, P.red_lo,
                      P.red_hi);
}

// K4: many molecules in one persistent launch, one molecule after another.  Every CTA
// walks the molecules in the host's order (largest estimated cost first); for each one
// that still has samples it loads the molecule's parameters and Bloom filter into shared
// memory and rebuilds the CTA tables, then its warps take samples of that molecule from
// the molecule's global cursor until none are left.  All CTAs therefore work on one or two
// molecules at a time: their integral tables stay in L2 as in one plain launch, while
// CTAs that run out of a molecule's samples start the next molecule without waiting for
// the rest of the grid.
// MAXT: the launch bound.  The per-molecule parameters live in shared memory, not in the
// constant bank, so the sample code needs more registers than in the single-molecule
// kernel: 512 threads (16 warps, 128 registers) keep it free of spills, 640 threads (20
// warps, 96 registers) trade a few spills for more warps (768 threads would spill 80-170
// bytes a thread).
// JOIN: the molecules' tables carry the sample-space join index (built with U = 4 only).
template <int PREC, int U, int MAXT, bool JOIN>
__global__ void __launch_bounds__(MAXT) eloc_batch_kernel(const __grid_constant__ BatchParams bp) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ MolParams mp;
    __shared__ int skip;
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + kOffBar);
    uint32_t* filt = reinterpret_cast<uint32_t*>(smem + kOffVar);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_barrier_init();
    }
    unsigned phase = 0;
    for (int k = 0; k < bp.n_mol; ++k) {
        __syncthreads();  // every warp is done with the previous molecule's shared data
        const int m = bp.order[k];
        const unsigned* src = reinterpret_cast<const unsigned*>(bp.mols + m);
        unsigned* dst = reinterpret_cast<unsigned*>(&mp);
        for (int t = threadIdx.x; t < static_cast<int>(sizeof(MolParams) / 4); t += blockDim.x) dst[t] = src[t];
        if (threadIdx.x == 0)
            skip = *reinterpret_cast<volatile unsigned long long*>(bp.next + k) >=
                   static_cast<unsigned long long>(bp.mols[m].r1 - bp.mols[m].r0) *
                       static_cast<unsigned long long>(bp.mols[m].ep.chunks > 1 ? bp.mols[m].ep.chunks : 1);
        __syncthreads();
        if (skip) continue;  // other CTAs took all of this molecule's samples
        const unsigned fbytes = 4u << mp.tp.fw;
        if (threadIdx.x == 0) {
            mbar_expect_tx(bar, fbytes);
            constexpr unsigned kChunk = 32768;
            for (unsigned off = 0; off < fbytes; off += kChunk) {
                const unsigned n = (fbytes - off < kChunk) ? (fbytes - off) : kChunk;
                bulk_g2s(reinterpret_cast<unsigned char*>(filt) + off,
                         reinterpret_cast<const unsigned char*>(mp.tp.filter) + off, n, bar);
            }
        }
        fill_cta_tables(mp.sp, mp.ep.T, smem);
        bool ready = false;
        for (unsigned it = 0; it < kWaitLimit; ++it) {
            if (mbar_try_wait(bar, phase)) {
                ready = true;
                break;
            }
        }
        if (!__syncthreads_and(ready ? 1 : 0)) {
            // the copy did not land in time: report, one more bounded wait, leave together
            if (threadIdx.x == 0) atomicOr(&mp.ep.ctr->flags, QC_FLAG_TIMEOUT);
            if (!ready)
                for (unsigned it = 0; it < kWaitLimit; ++it)
                    if (mbar_try_wait(bar, phase)) break;
            return;
        }
        phase ^= 1u;
        // this molecule's layout: its own filter size and per-warp region; warps beyond
        // what fits in shared memory sit it out
        const int nw = mp.active_warps;
        if (warp < nw) {
            unsigned char* wl = smem + kOffVar + fbytes + static_cast<size_t>(warp) * mp.warp_stride;
            // rows [r0, r1) of this molecule: all of them, or one slice of a long request;
            // with C excitation chunks per sample a work item is (row, chunk)
            const unsigned long long C = static_cast<unsigned long long>(mp.ep.chunks > 1 ? mp.ep.chunks : 1);
            const unsigned long long n_run = static_cast<unsigned long long>(mp.r1 - mp.r0) * C;
            const long long r0 = mp.r0;
            while (true) {
                unsigned long long i0 = 0;
                if (lane == 0) i0 = atomicAdd(bp.next + k, static_cast<unsigned long long>(bp.chunk));
                i0 = __shfl_sync(0xffffffffu, i0, 0);
                if (i0 >= n_run) break;
                const unsigned long long i1 = i0 + bp.chunk < n_run ? i0 + bp.chunk : n_run;
                for (unsigned long long it = i0; it < i1; ++it) {
                    const unsigned long long q = it / C;
                    // a joining molecule's rows heavy first (slices cut the same order)
                    const long long s = mp.ep.order != nullptr
                                            ? static_cast<long long>(__ldg(mp.ep.order + r0 + static_cast<long long>(q)))
                                            : r0 + static_cast<long long>(q);
                    const int c = static_cast<int>(it - q * C);
                    // a joining molecule's alpha list may be capped (mp.tp.alpha_cap): segments.
                    // One copy of the sample code takes either list layout (ep.lean), so the
                    // kernel holds it once
                    run_sample<PREC, U, true, 2, JOIN, false, JOIN, JOIN>(mp.sp, mp.tp, mp.ep, s, lane, smem, wl, filt, c,
                                                                     static_cast<int>(C));
                }
            }
        }
    }
}

size_t batch_warp_bytes(const SysParams& sp, bool lean, bool join, int acap) {
    return main_warp_bytes(sp, true, lean, join, acap);
}

cudaError_t launch_build_batch(const MolParams* mols, const MolWork* work, const long long* key_off,
                               int n_mol, long long n_keys, cudaStream_t s) {
    if (n_keys <= 0) return cudaSuccess;
    build_batch_kernel<<<static_cast<unsigned>((n_keys + 255) / 256), 256, 0, s>>>(mols, work, key_off, n_mol,
                                                                                    n_keys);
    return cudaGetLastError();
}

cudaError_t launch_reduce_batch(const MolParams* mols, const MolWork* work, int n_mol, int max_blocks,
                                cudaStream_t s) {
    const dim3 grid(max_blocks, n_mol);
    reduce_batch_pass1<<<grid, kRedThreads, 0, s>>>(mols, work);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_batch_pass2<<<grid, kRedThreads, 0, s>>>(mols, work);
    return cudaGetLastError();
}

template <int PREC>
static const void* batch_kernel_ptr(int unroll, int warps, bool join) {
    if (join) return warps > 16 ? (const void*)eloc_batch_kernel<PREC, 4, 640, true> : (const void*)eloc_batch_kernel<PREC, 4, 512, true>;
    if (warps > 16) return unroll == 2 ? (const void*)eloc_batch_kernel<PREC, 2, 640, false> : (const void*)eloc_batch_kernel<PREC, 4, 640, false>;
    return unroll == 2 ? (const void*)eloc_batch_kernel<PREC, 2, 512, false> : (const void*)eloc_batch_kernel<PREC, 4, 512, false>;
}

template <int PREC, int U, bool JOIN>
static void launch_batch_u(const BatchParams& bp, int grid, int warps, size_t smem, cudaStream_t s) {
    const dim3 g(grid), b(32 * warps);
    if (warps > 16) eloc_batch_kernel<PREC, U, 640, JOIN><<<g, b, smem, s>>>(bp);
    else eloc_batch_kernel<PREC, U, 512, JOIN><<<g, b, smem, s>>>(bp);
}

cudaError_t launch_eloc_batch(const BatchParams& bp, int precision, int unroll, int grid, int warps,
                              size_t smem, cudaStream_t s, bool join) {
    if (precision == QC_FP64) {
        if (join) launch_batch_u<QC_FP64, 4, true>(bp, grid, warps, smem, s);
        else if (unroll == 2) launch_batch_u<QC_FP64, 2, false>(bp, grid, warps, smem, s);
        else launch_batch_u<QC_FP64, 4, false>(bp, grid, warps, smem, s);
    } else {
        if (join) launch_batch_u<QC_FP32_COMP, 4, true>(bp, grid, warps, smem, s);
        else if (unroll == 2) launch_batch_u<QC_FP32_COMP, 2, false>(bp, grid, warps, smem, s);
        else launch_batch_u<QC_FP32_COMP, 4, false>(bp, grid, warps, smem, s);
    }
    return cudaGetLastError();
}

int max_active_batch(int precision, int unroll, int threads, size_t smem, bool join) {
    const int w = threads / 32;
    const void* f = precision == QC_FP64 ? batch_kernel_ptr<QC_FP64>(unroll, w, join)
                                         : batch_kernel_ptr<QC_FP32_COMP>(unroll, w, join);
    int n = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, threads, smem) == cudaSuccess ? n : 0;
}

// Dynamic shared memory of the batch kernels: the opt-in limit less their static share.
cudaError_t prepare_batch_kernels(size_t max_smem, size_t* dyn_limit) {
    cudaError_t e = cudaSuccess;
    size_t lim = max_smem;
    for (int prec = 0; prec < 2; ++prec)
        for (int k = 0; k < 8; ++k) {
            const int unroll = (k & 1) ? 4 : 2, w = (k & 2) ? 20 : 16;
            const bool join = (k & 4) != 0;
            const void* f = prec == QC_FP64 ? batch_kernel_ptr<QC_FP64>(unroll, w, join)
                                            : batch_kernel_ptr<QC_FP32_COMP>(unroll, w, join);
            cudaFuncAttributes a{};
            cudaError_t r = cudaFuncGetAttributes(&a, f);
            if (r != cudaSuccess) { e = r; continue; }
            const size_t dyn = max_smem - a.sharedSizeBytes;
            if (dyn < lim) lim = dyn;
            r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(dyn));
            if (r != cudaSuccess) e = r;
        }
    if (dyn_limit) *dyn_limit = lim;
    return e;
}

}  // namespace qc
