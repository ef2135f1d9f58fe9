// qc_grad.cu -- Eq. 4 (Sec. II-A): the energy gradient
//   d<E>/d theta_p = 2 Re < d_theta_p ln Psi*(n) (E_loc(n) - <E>) >_n
// as a count-weighted average over the unique samples of one evaluation.  Two device steps:
//   K5 grad_weights_kernel   w_i = c_i (E_loc,i - Ebar) / W   (0 where E_loc is not finite)
//   K6 grad_contract_kernel  partial_rp = sum over rows of chunk r of Re(w_i D_ip)
//   K7 grad_finish_kernel    g_p = 2 sum_r partial_rp   (fixed order: deterministic)
// Ebar and W come from the evaluation's device summary (written by the Eq. 1 reduction on
// the same stream), so the call is asynchronous.  The contraction streams the n_u x P
// complex rows D = d ln Psi* once from HBM (16 B per element, 16-byte streaming loads,
// coalesced along a row) and spends two FP64 fused multiply-adds per element; at this GPU's
// FP64 rate the arithmetic, not HBM, bounds it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "qc_eloc.h"
#include "qc_handle.h"
#include "qc_internal.h"

namespace {

constexpr int kGradThreads = 256;  // columns per CTA of the contraction
constexpr int kGradRowsMax = 256;  // rows of a chunk staged in shared memory at a time

__device__ __forceinline__ double2 weight(const double2 e, const long long c, const qc_eloc_summary* sum) {
    const double W = sum->w;
    if (!(W > 0.0) || c < 0 || !isfinite(e.x) || !isfinite(e.y)) return make_double2(0.0, 0.0);
    const double s = static_cast<double>(c) / W;
    return make_double2(s * (e.x - sum->e_re), s * (e.y - sum->e_im));
}

__global__ void __launch_bounds__(256) grad_weights_kernel(const double2* __restrict__ eloc,
                                                           const long long* __restrict__ counts, long long n,
                                                           const qc_eloc_summary* __restrict__ sum,
                                                           double2* __restrict__ w) {
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        w[i] = weight(eloc[i], counts[i], sum);
}

// One CTA: kGradThreads consecutive columns of one chunk of rows.  The chunk's weights are
// staged in shared memory; every thread then walks the rows of its column, four loads in
// flight.
__global__ void __launch_bounds__(kGradThreads) grad_contract_kernel(const double2* __restrict__ eloc,
                                                                    const long long* __restrict__ counts,
                                                                    long long n, const qc_eloc_summary* __restrict__ sum,
                                                                    const double2* __restrict__ D, long long P,
                                                                    long long rows_per_chunk, double* __restrict__ part) {
    __shared__ double2 ws[kGradRowsMax];
    const long long p = static_cast<long long>(blockIdx.x) * kGradThreads + threadIdx.x;
    const long long r0 = static_cast<long long>(blockIdx.y) * rows_per_chunk;
    const long long r1 = r0 + rows_per_chunk < n ? r0 + rows_per_chunk : n;
    double acc = 0.0;
    for (long long b = r0; b < r1; b += kGradRowsMax) {
        const int nb = static_cast<int>(r1 - b < kGradRowsMax ? r1 - b : kGradRowsMax);
        __syncthreads();
        for (int t = threadIdx.x; t < nb; t += kGradThreads) ws[t] = weight(eloc[b + t], counts[b + t], sum);
        __syncthreads();
        if (p < P) {
            const double2* row = D + b * P + p;
            int t = 0;
            for (; t + 4 <= nb; t += 4) {
                const double2 d0 = __ldcs(row + (t + 0) * P);
                const double2 d1 = __ldcs(row + (t + 1) * P);
                const double2 d2 = __ldcs(row + (t + 2) * P);
                const double2 d3 = __ldcs(row + (t + 3) * P);
                // Re(w d) as two fused multiply-adds per element: the FP64 pipe, not HBM, is
                // the narrower resource on this GPU, so no third FP64 operation per element
                acc = fma(ws[t + 0].x, d0.x, acc);
                acc = fma(-ws[t + 0].y, d0.y, acc);
                acc = fma(ws[t + 1].x, d1.x, acc);
                acc = fma(-ws[t + 1].y, d1.y, acc);
                acc = fma(ws[t + 2].x, d2.x, acc);
                acc = fma(-ws[t + 2].y, d2.y, acc);
                acc = fma(ws[t + 3].x, d3.x, acc);
                acc = fma(-ws[t + 3].y, d3.y, acc);
            }
            for (; t < nb; ++t) {
                const double2 d = __ldcs(row + t * P);
                acc = fma(ws[t].x, d.x, acc);
                acc = fma(-ws[t].y, d.y, acc);
            }
        }
    }
    if (p < P) part[static_cast<long long>(blockIdx.y) * P + p] = acc;
}

__global__ void __launch_bounds__(256) grad_finish_kernel(const double* __restrict__ part, int chunks, long long P,
                                                          double* __restrict__ g) {
    for (long long p = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; p < P;
         p += static_cast<long long>(gridDim.x) * blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < chunks; ++r) s += part[static_cast<long long>(r) * P + p];
        g[p] = 2.0 * s;
    }
}

// Row chunks of the contraction: a function of n only (not of the GPU), so the summation
// order, and the result, are the same everywhere.
int grad_chunks(long long n) {
    const long long c = (n + 63) / 64;
    return static_cast<int>(std::max<long long>(1, std::min<long long>(c, 512)));
}

}  // namespace

extern "C" qc_status qc_eloc_grad(qc_eloc* H, const double* eloc, const int64_t* counts, int64_t n_u,
                                  const double* dconj, int64_t n_par, double* w_out, double* g_out,
                                  void* stream) {
    if (!H) return QC_ERR_ARG;
    auto fail = [&](qc_status st, const char* m) {
        H->err = m;
        return st;
    };
    if (n_u < 0 || n_par < 0) return fail(QC_ERR_ARG, "negative size");
    if (n_u > 0 && (!eloc || !counts)) return fail(QC_ERR_ARG, "eloc or counts is NULL");
    if (g_out && n_par > 0 && !dconj) return fail(QC_ERR_ARG, "g_out needs dconj");
    auto mis = [](const void* q, unsigned a) { return q && (reinterpret_cast<uintptr_t>(q) & (a - 1)) != 0; };
    if (mis(eloc, 16) || mis(dconj, 16) || mis(w_out, 16) || mis(counts, 8) || mis(g_out, 8))
        return fail(QC_ERR_ARG, "device arrays must be 16-byte aligned (counts, g_out: 8)");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != H->device) return fail(QC_ERR_ARG, "handle belongs to another device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double2* e2 = reinterpret_cast<const double2*>(eloc);
    const long long* c = reinterpret_cast<const long long*>(counts);
    cudaError_t e = cudaSuccess;
    if (w_out && n_u > 0) {
        const long long blocks = std::min<long long>((n_u + 255) / 256, 4096);
        grad_weights_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(e2, c, n_u, H->d_sum,
                                                                          reinterpret_cast<double2*>(w_out));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && g_out && n_par > 0) {
        if (n_u == 0) {
            e = cudaMemsetAsync(g_out, 0, static_cast<size_t>(n_par) * sizeof(double), s);
        } else {
            const int chunks = grad_chunks(n_u);
            const long long rows = (n_u + chunks - 1) / chunks;
            const size_t need = static_cast<size_t>(chunks) * static_cast<size_t>(n_par);
            if (need > H->gpart_cap) {
                if (H->d_gpart) cudaFree(H->d_gpart);
                H->d_gpart = nullptr;
                H->gpart_cap = 0;
                e = qc::dev_alloc(&H->d_gpart, need * sizeof(double));
                if (e == cudaSuccess) H->gpart_cap = need;
            }
            if (e == cudaSuccess) {
                const long long tiles = (n_par + kGradThreads - 1) / kGradThreads;
                if (tiles > 0x7fffffffLL) return fail(QC_ERR_CAPACITY, "n_par too large");
                grad_contract_kernel<<<dim3(static_cast<unsigned>(tiles), static_cast<unsigned>(chunks)), kGradThreads,
                                       0, s>>>(e2, c, n_u, H->d_sum, reinterpret_cast<const double2*>(dconj), n_par,
                                               rows, H->d_gpart);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) {
                const long long blocks = std::min<long long>((n_par + 255) / 256, 4096);
                grad_finish_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(H->d_gpart, chunks, n_par, g_out);
                e = cudaGetLastError();
            }
        }
    }
    if (e != cudaSuccess) {
        H->err = std::string("qc_eloc_grad: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? QC_ERR_OOM : QC_ERR_CUDA;
    }
    return QC_OK;
}
