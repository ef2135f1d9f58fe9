// qc_full.cu -- the "accurate energy" of Sec. IV-C-4 at scale: the full connected set of
// every sample is handed to the caller (whose network evaluates psi on it), and Eq. 5 is
// then reduced against those values.
//   K8 eloc_export_kernel  every single and double excitation x' of each sample, its signed
//                          Slater-Condon element <x|H|x'> (Eq. 2, Sec. III-B (ii)) and the
//                          diagonal <x|H|x>, written in a fixed order (below)
//   K9 eloc_apply_kernel   E_loc(x) = <x|H|x> + sum_j <x|H|x'_j> psi(x'_j) / psi(x)
// followed by the Eq. 1 reduction (K3) over the chunk.
//
// Order of the connected set of one sample (P = pairs per sample, position = class offset
// + u * n2 + w): alpha singles, beta singles (w = occupied index * empty count + empty
// index, both over the spin's ascending lists), alpha-alpha and beta-beta doubles (u an
// occupied pair, w an empty pair; the pair (p < q) has index q (q - 1) / 2 + p), then
// alpha-beta doubles (u an alpha single, w a beta single).
//
// Both kernels stream HBM: the export writes 24 B per pair (key and element), the apply
// reads 24 B per pair (element and psi) plus two FP64 fused multiply-adds.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "qc_device.cuh"
#include "qc_eloc.h"
#include "qc_handle.h"
#include "qc_internal.h"

namespace qc {
namespace {

constexpr int kExpWarps = 8;
constexpr int kPer = 2;  // double excitations per lane per step of the export (4 measured slower)

struct ExportOut {
    ulonglong2* keys;   // [n_u * P] or null
    double* elems;      // [n_u * P] or null
    double* diag;       // [n_u] or null
};

// Work item (sample s, part c of C): part c takes the singles when c = 0 and the outer
// entries c, c + C, ... of each double class; items are handed out from a device cursor so
// that the launch ends with little tail.
template <int PREC>
__global__ void __launch_bounds__(32 * kExpWarps, 4) eloc_export_kernel(const __grid_constant__ SysParams sp,
                                                                     const ulonglong2* __restrict__ samples,
                                                                     long long n_u,
                                                                     const unsigned long long* __restrict__ Tg,
                                                                     const ExportOut out, int C,
                                                                     unsigned long long* __restrict__ cursor) {
    extern __shared__ __align__(128) unsigned char smem[];
    fill_cta_tables(sp, Tg, smem);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char* wl = smem + kOffVar + 256 * warp;
    const unsigned long long* T64 = reinterpret_cast<const unsigned long long*>(smem + kOffT);
    const long long P = sp.pairs;
    const unsigned long long items = static_cast<unsigned long long>(n_u) * C;
    while (true) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(cursor, 1ULL);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= items) break;
        const long long s = static_cast<long long>(it / C);
        const int c = static_cast<int>(it - static_cast<unsigned long long>(s) * C);
        const ulonglong2 x = samples[s];
        unsigned long long hx, As, Bs, hxa;
        double ediag;
        const bool ok = sample_setup(sp, x, lane, wl, T64, hx, ediag, As, Bs, hxa);
        __syncwarp();
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
        if (lane == 0 && out.diag && c == 0) out.diag[s] = ok ? ediag : nan;
        const ulonglong2 px = prefix_parity(x);
        long long off = static_cast<long long>(s) * P;
        const unsigned char* occA = wl;
        const unsigned char* virA = wl + 64;
        const unsigned char* occB = wl + 128;
        const unsigned char* virB = wl + 192;
        const unsigned short* lut = reinterpret_cast<const unsigned short*>(smem + kOffLut);
        const unsigned char* divA = smem + kOffDiv;
        const unsigned char* divB = divA + 1024;
        const int K = sp.K;
        for (int cls = 0; cls < 5; ++cls) {
            const int n1 = cls < 2 ? 1 : cls == 2 ? sp.npoa : cls == 3 ? sp.npob : sp.nsa;
            const int n2 = cls == 0 ? sp.nsa : cls == 1 ? sp.nsb : cls == 2 ? sp.npva : cls == 3 ? sp.npvb : sp.nsb;
            // singles in part 0; the outer entries of the doubles interleaved over the parts
            for (int u = cls < 2 ? (c == 0 ? 0 : n1) : c; u < n1; u += cls < 2 ? 1 : C) {
                // the part of the excitation fixed by u (uniform across the warp): emptied
                // orbital(s), their bits and their share of the phase and of the integral index
                int i = 0, j = 0, a0 = 0;
                ulonglong2 xu = x;
                int paru = 0;
                const int sp_ = cls == 3 ? 1 : 0;
                if (ok && cls >= 2) {
                    if (cls == 4) {
                        const int io = divA[u];
                        i = 2 * occA[io];
                        a0 = 2 * virA[u - io * sp.va];
                        flip(xu, i);
                        flip(xu, a0);
                        paru = pbit(px, i) ^ pbit(px, a0);
                    } else {
                        const unsigned pu = lut[u];
                        const unsigned char* occ = cls == 2 ? occA : occB;
                        i = 2 * occ[pu & 255u] + sp_;
                        j = 2 * occ[pu >> 8] + sp_;
                        flip(xu, i);
                        flip(xu, j);
                        paru = pbit(px, i) ^ pbit(px, j);
                    }
                }
                if (!ok || cls < 2) {
                    for (int w0 = 0; w0 < n2; w0 += 32) {
                        const int w = w0 + lane;
                        if (w >= n2) continue;
                        const long long pos = off + static_cast<long long>(u) * n2 + w;
                        if (!ok) {  // not a determinant of this system: no connected set
                            if (out.keys) __stcs(out.keys + pos, make_ulonglong2(0ULL, 0ULL));
                            if (out.elems) __stcs(out.elems + pos, nan);
                            continue;
                        }
                        // singles: the general path (a small share of the pairs)
                        const unsigned code = (static_cast<unsigned>(cls) << 24) | static_cast<unsigned>(w);
                        const unsigned orbs = decode(code, sp, wl, smem, nullptr, nullptr);
                        if (out.keys) {
                            unsigned long long h;
                            __stcs(out.keys + pos, excite(orbs, x, hx, T64, h));
                        }
                        if (out.elems) {
                            double h64 = 0.0;
                            float h32 = 0.f;
                            bool sneg = false;
                            single_element<PREC>(orbs, px, sp, wl, nullptr, h64, h32, sneg);
                            __stcs(out.elems + pos, PREC == QC_FP64 ? h64 : static_cast<double>(h32));
                        }
                    }
                    continue;
                }
                // doubles: kPer excitations per lane per step (w, w + 32, ...), every integral
                // load issued before any is used
                for (int w0 = 0; w0 < n2; w0 += 32 * kPer) {
                    int aa[kPer], bb[kPer], jj[kPer];
                    bool v[kPer];
#pragma unroll
                    for (int h = 0; h < kPer; ++h) {
                        const int w = w0 + 32 * h + lane;
                        v[h] = w < n2;
                        const int ww = v[h] ? w : 0;
                        if (cls == 4) {
                            const int jo = divB[ww];
                            aa[h] = a0;
                            jj[h] = 2 * occB[jo] + 1;
                            bb[h] = 2 * virB[ww - jo * sp.vb] + 1;
                        } else {
                            const unsigned pw = lut[ww];
                            const unsigned char* vir = cls == 2 ? virA : virB;
                            jj[h] = j;
                            aa[h] = 2 * vir[pw & 255u] + sp_;
                            bb[h] = 2 * vir[pw >> 8] + sp_;
                        }
                    }
                    double e1[kPer], e2[kPer];
                    float f1[kPer], f2[kPer];
#pragma unroll
                    for (int h = 0; h < kPer; ++h) {
                        e1[h] = e2[h] = 0.0;
                        f1[h] = f2[h] = 0.f;
                    }
                    if (out.elems) {
#pragma unroll
                        for (int h = 0; h < kPer; ++h) {
                            if (!v[h]) continue;
                            const int ki = i >> 1, ka = aa[h] >> 1, kj = jj[h] >> 1, kb = bb[h] >> 1;
                            const size_t d = ((static_cast<size_t>(ka) * K + ki) * K + kb) * K + kj;  // (ai|bj)
                            const size_t d2 = ((static_cast<size_t>(ka) * K + kj) * K + kb) * K + ki;  // (aj|bi)
                            if (PREC == QC_FP64) {
                                e1[h] = __ldg(sp.eri + d);
                                if (cls != 4) e2[h] = __ldg(sp.eri + d2);
                            } else {
                                f1[h] = __ldg(sp.eri32 + d);
                                if (cls != 4) f2[h] = __ldg(sp.eri32 + d2);
                            }
                        }
                    }
#pragma unroll
                    for (int h = 0; h < kPer; ++h) {
                        if (!v[h]) continue;
                        const long long pos = off + static_cast<long long>(u) * n2 + w0 + 32 * h + lane;
                        ulonglong2 xp = xu;
                        if (cls == 4) {
                            flip(xp, jj[h]);
                            flip(xp, bb[h]);
                        } else {
                            flip(xp, aa[h]);
                            flip(xp, bb[h]);
                        }
                        if (out.keys) __stcs(out.keys + pos, xp);
                        if (out.elems) {
                            // <ab||ij> and its phase exactly as double_element forms them
                            const int ii = i, ja = jj[h], a = aa[h], b = bb[h];
                            const int par = (paru ^ (cls == 4 ? (pbit(px, ja) ^ pbit(px, b)) : (pbit(px, a) ^ pbit(px, b)))) +
                                            (ii < ja) + (ii < b) + (ja < b) + (ii < a) + (ja < a) + (b < a);
                            double val;
                            if (PREC == QC_FP64) {
                                double e = e1[h];
                                if (cls != 4) e -= e2[h];
                                val = (par & 1) ? -e : e;
                            } else {
                                float e = f1[h];
                                if (cls != 4) e -= f2[h];
                                val = static_cast<double>((par & 1) ? -e : e);
                            }
                            __stcs(out.elems + pos, val);
                        }
                    }
                }
            }
            off += static_cast<long long>(n1) * n2;
        }
        __syncwarp();
    }
}

// One warp per sample: the P products summed lane-wise in FP64 (fixed lanes, fixed shuffle
// tree: deterministic), then one complex division by psi(x).
__global__ void __launch_bounds__(256) eloc_apply_kernel(const double* __restrict__ elems,
                                                         const double* __restrict__ diag,
                                                         const double2* __restrict__ psi_conn,
                                                         const double2* __restrict__ psi, long long n_u,
                                                         long long P, double2* __restrict__ eloc,
                                                         Counters* __restrict__ ctr) {
    const int lane = threadIdx.x & 31;
    const long long warps = static_cast<long long>(gridDim.x) * (blockDim.x >> 5);
    for (long long s = static_cast<long long>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); s < n_u;
         s += warps) {
        const double* e = elems + s * P;
        const double2* q = psi_conn + s * P;
        // two independent partial sums per lane (j and j + 32 of each 64), added at the end
        double re = 0.0, im = 0.0, re2 = 0.0, im2 = 0.0;
        long long j = lane;
        for (; j + 32 < P; j += 64) {
            const double h0 = __ldcs(e + j), h1 = __ldcs(e + j + 32);
            const double2 v0 = __ldcs(q + j), v1 = __ldcs(q + j + 32);
            re = fma(h0, v0.x, re);
            im = fma(h0, v0.y, im);
            re2 = fma(h1, v1.x, re2);
            im2 = fma(h1, v1.y, im2);
        }
        if (j < P) {
            const double h0 = __ldcs(e + j);
            const double2 v0 = __ldcs(q + j);
            re = fma(h0, v0.x, re);
            im = fma(h0, v0.y, im);
        }
        re = warp_sum(re + re2);
        im = warp_sum(im + im2);
        if (lane == 0) {
            const double2 p = psi[s];
            const double n2 = p.x * p.x + p.y * p.y;
            const double d = diag[s];
            double2 out;
            if (n2 == 0.0 || !isfinite(d)) {
                out.x = out.y = __longlong_as_double(0x7ff8000000000000LL);
                atomicAdd(&ctr->bad, 1ULL);
                if (n2 == 0.0) atomicOr(&ctr->flags, QC_FLAG_ZERO_PSI);
                else {
                    atomicAdd(&ctr->invalid, 1ULL);
                    atomicOr(&ctr->flags, QC_FLAG_NELEC);
                }
            } else {
                const double inv = 1.0 / n2;
                out.x = d + (re * p.x + im * p.y) * inv;
                out.y = (im * p.x - re * p.y) * inv;
            }
            eloc[s] = out;
        }
    }
}

qc_status ffail(qc_eloc* H, qc_status st, const std::string& m) {
    H->err = m;
    return st;
}

}  // namespace
}  // namespace qc

extern "C" qc_status qc_eloc_export(qc_eloc* H, const uint64_t* samples, int64_t n_u, uint64_t* keys_out,
                                    double* elems_out, double* diag_out, void* stream) {
    if (!H) return QC_ERR_ARG;
    if (n_u < 0) return qc::ffail(H, QC_ERR_ARG, "negative n_u");
    if (n_u > 0 && !samples) return qc::ffail(H, QC_ERR_ARG, "samples is NULL");
    auto mis = [](const void* p, unsigned a) { return p && (reinterpret_cast<uintptr_t>(p) & (a - 1)) != 0; };
    if (mis(samples, 16) || mis(keys_out, 16) || mis(elems_out, 8) || mis(diag_out, 8))
        return qc::ffail(H, QC_ERR_ARG, "alignment: samples and keys 16 bytes, elements and diagonal 8");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != H->device) return qc::ffail(H, QC_ERR_ARG, "handle belongs to another device");
    if (n_u == 0 || (!keys_out && !elems_out && !diag_out)) return QC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    qc::ExportOut out{reinterpret_cast<ulonglong2*>(keys_out), elems_out, diag_out};
    const size_t smem = qc::kOffVar + 256 * qc::kExpWarps;
    // parts per sample: about 4,096 pairs each, at most 8
    const int C = static_cast<int>(std::max<long long>(1, std::min<long long>(8, H->sp.pairs / 4096)));
    const long long items = n_u * C;
    const long long blocks = std::min<long long>((items + qc::kExpWarps - 1) / qc::kExpWarps,
                                                 static_cast<long long>(H->sm_count) * 4);
    unsigned long long* cursor = &H->d_ctr->next;  // the handle's counters are free between evaluations
    cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return qc::ffail(H, QC_ERR_CUDA, std::string("export: ") + cudaGetErrorString(e));
    if (H->precision == QC_FP64)
        qc::eloc_export_kernel<QC_FP64><<<static_cast<unsigned>(blocks), 32 * qc::kExpWarps, smem, s>>>(
            H->sp, reinterpret_cast<const ulonglong2*>(samples), n_u, H->d_T, out, C, cursor);
    else
        qc::eloc_export_kernel<QC_FP32_COMP><<<static_cast<unsigned>(blocks), 32 * qc::kExpWarps, smem, s>>>(
            H->sp, reinterpret_cast<const ulonglong2*>(samples), n_u, H->d_T, out, C, cursor);
    e = cudaGetLastError();
    if (e != cudaSuccess) return qc::ffail(H, QC_ERR_CUDA, std::string("export launch: ") + cudaGetErrorString(e));
    return QC_OK;
}

extern "C" qc_status qc_eloc_apply(qc_eloc* H, const double* psi, const int64_t* counts, int64_t n_u,
                                   const double* elems, const double* diag, const double* psi_conn,
                                   double* eloc_out, qc_eloc_summary* summary, void* stream) {
    if (!H) return QC_ERR_ARG;
    if (n_u < 0) return qc::ffail(H, QC_ERR_ARG, "negative n_u");
    if (n_u > 0 && (!psi || !counts || !elems || !diag || !psi_conn || !eloc_out))
        return qc::ffail(H, QC_ERR_ARG, "NULL pointer");
    auto mis = [](const void* p, unsigned a) { return p && (reinterpret_cast<uintptr_t>(p) & (a - 1)) != 0; };
    if (mis(psi, 16) || mis(psi_conn, 16) || mis(eloc_out, 16) || mis(elems, 8) || mis(diag, 8) || mis(counts, 8))
        return qc::ffail(H, QC_ERR_ARG, "alignment: complex arrays 16 bytes, the others 8");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != H->device) return qc::ffail(H, QC_ERR_ARG, "handle belongs to another device");
    qc_status st = qc::ensure_workspace(H, std::max<int64_t>(n_u, 1), 1, 0);
    if (st != QC_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(H->d_ctr, 0, sizeof(qc::Counters), s);
    if (e == cudaSuccess && n_u > 0) {
        const long long blocks = std::min<long long>((n_u + 7) / 8, static_cast<long long>(H->sm_count) * 16);
        qc::eloc_apply_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(
            elems, diag, reinterpret_cast<const double2*>(psi_conn), reinterpret_cast<const double2*>(psi), n_u,
            H->sp.pairs, reinterpret_cast<double2*>(eloc_out), H->d_ctr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        qc::EvalParams ep{};
        ep.psi = reinterpret_cast<const double2*>(psi);
        ep.counts = reinterpret_cast<const long long*>(counts);
        ep.n_u = n_u;
        ep.eloc = reinterpret_cast<double2*>(eloc_out);
        ep.ctr = H->d_ctr;
        ep.T = H->d_T;
        ep.mode = QC_FULL;
        e = qc::launch_reduce(ep, H->d_part, qc::reduce_blocks(n_u), H->d_sum, H->sp.pairs, s);
    }
    if (e == cudaSuccess && summary)
        e = cudaMemcpyAsync(summary, H->d_sum, sizeof(qc_eloc_summary), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return qc::ffail(H, QC_ERR_CUDA, std::string("apply: ") + cudaGetErrorString(e));
    return QC_OK;
}
