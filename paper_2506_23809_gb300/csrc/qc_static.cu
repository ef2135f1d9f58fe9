// qc_static.cu -- qc_eloc_eval_static: the sample-space evaluation with its scratch memory
// in a file-scope device array, for callers that must not allocate device memory.
//
// Who needs it: code that runs where a device allocation is not allowed or not wanted --
// inside a CUDA stream capture in a capture mode that forbids unsafe API calls, inside a
// framework that owns all device memory through its own pool, or in a latency-bound
// request loop that must never block on the allocator.  Such a caller hands in device
// buffers for every input and output; the library supplies the rest from the array below.
//
// The array (kStaticBytes, about 8.4 MB) is created by the CUDA runtime on a GPU when the
// library's device code is loaded there -- with lazy module loading (the default since CUDA
// 12.2) at the first call on that device that needs it, which the set-up below forces -- and
// it stays there until the process exits.  Every call shares it, so
// two calls that overlap on the GPU (different streams, or different host threads) race
// on it; the array keeps whatever the last call left, and each call clears the parts that
// must start at zero.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "qc_eloc.h"
#include "qc_internal.h"

namespace qc {
namespace {

constexpr int kStaticMaxK = QC_STATIC_MAX_ORB / 2;
constexpr size_t kStaticBuckets = 2u * QC_STATIC_MAX_SAMPLES;  // next_pow2(2 n) at the maximum
constexpr int kStaticFilterLog2 = 15;

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffCtr = 0;
constexpr size_t kOffSum = align256(kOffCtr + sizeof(Counters));
constexpr size_t kOffPart = align256(kOffSum + sizeof(qc_eloc_summary));
constexpr size_t kOffTab = align256(kOffPart + 1024 * 4 * sizeof(double));
constexpr size_t kOffJ = align256(kOffTab + 128 * sizeof(unsigned long long));
constexpr size_t kOffX = align256(kOffJ + kStaticMaxK * kStaticMaxK * sizeof(double));
constexpr size_t kOffJt = align256(kOffX + kStaticMaxK * kStaticMaxK * sizeof(double));
constexpr size_t kOffXt = align256(kOffJt + static_cast<size_t>(kStaticMaxK) * kStaticMaxK * kStaticMaxK * sizeof(double));
constexpr size_t kOffFilter = align256(kOffXt + static_cast<size_t>(kStaticMaxK) * kStaticMaxK * kStaticMaxK * sizeof(double));
constexpr size_t kOffSlots = align256(kOffFilter + (static_cast<size_t>(4) << kStaticFilterLog2));
constexpr size_t kStaticBytes = align256(kOffSlots + 2 * kStaticBuckets * sizeof(unsigned long long));

// The scratch of qc_eloc_eval_static (see the file comment).
static __device__ __align__(256) unsigned char qc_static_scratch[kStaticBytes];

// per-device set-up: the address of the array as the device sees it
struct DeviceSlot {
    std::once_flag once;
    cudaError_t err = cudaSuccess;
    unsigned char* base = nullptr;
};
DeviceSlot g_slots[64];
qc_status static_fail(qc_status st, const std::string& m) {
    set_handleless_error(m);  // read back with qc_eloc_last_error(NULL)
    return st;
}

// J, X, Jt, Xt from (pq|rs) and the 128 entries of the linear key hash, on the device.
// The hash entries follow the same splitmix64 sequence (Vigna) as qc_eloc_create.
__global__ void static_prep_kernel(const double* __restrict__ eri, int K, double* J, double* X,
                                   double* Jt, double* Xt, unsigned long long* T) {
    const size_t n3 = static_cast<size_t>(K) * K * K;
    for (size_t t = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < n3;
         t += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int p = static_cast<int>(t / (static_cast<size_t>(K) * K));
        const int i = static_cast<int>((t / K) % K);
        const int k = static_cast<int>(t % K);
        Jt[t] = eri[((static_cast<size_t>(p) * K + i) * K + k) * K + k];  // (pi|kk)
        Xt[t] = eri[((static_cast<size_t>(p) * K + k) * K + k) * K + i];  // (pk|ki)
        if (p == 0) {
            J[i * K + k] = eri[((static_cast<size_t>(i) * K + i) * K + k) * K + k];  // (ii|kk)
            // same-spin pair term of the diagonal: (ii|kk) - (ik|ki)
            X[i * K + k] = J[i * K + k] - eri[((static_cast<size_t>(i) * K + k) * K + k) * K + i];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < 128) {
        unsigned long long z = 0x51c0de5eedULL + 0x9e3779b97f4a7c15ULL * (threadIdx.x + 1ULL);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
        T[threadIdx.x] = z ^ (z >> 31);
    }
}

unsigned long long next_pow2_u(unsigned long long v) {
    unsigned long long p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace
}  // namespace qc

extern "C" qc_status qc_eloc_eval_static(const double* h, const double* eri, double e_core, int n_orb,
                                         int n_elec, const uint64_t* samples, const int64_t* counts,
                                         const double* psi, int64_t n_u, double* eloc,
                                         qc_eloc_summary* summary, void* stream) {
    using namespace qc;
    if (n_orb < 2 || n_orb > QC_STATIC_MAX_ORB || (n_orb & 1))
        return static_fail(QC_ERR_ARG, "n_orb must be even, 2..128");
    if (n_elec <= 0 || n_elec >= n_orb || (n_elec & 1))
        return static_fail(QC_ERR_ARG, "n_elec must be even with 0 < n_elec < n_orb (S_z = 0)");
    if (n_u < 0) return static_fail(QC_ERR_ARG, "negative n_u");
    if (n_u > QC_STATIC_MAX_SAMPLES)
        return static_fail(QC_ERR_CAPACITY, "n_u exceeds QC_STATIC_MAX_SAMPLES (131072): the static "
                                            "scratch is sized for at most that many samples");
    if (!h || !eri || (n_u > 0 && (!samples || !counts || !psi || !eloc)))
        return static_fail(QC_ERR_ARG, "NULL pointer");
    auto mis = [](const void* p, unsigned a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) != 0; };
    if (n_u > 0 && (mis(samples, 16) || mis(psi, 16) || mis(eloc, 16) || mis(counts, 8)))
        return static_fail(QC_ERR_ARG, "device arrays must be 16-byte aligned (counts: 8)");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(QC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return static_fail(QC_ERR_ARG, "device ordinal above 63");
    DeviceSlot& slot = g_slots[dev];
    // first call on this device (device current): look the array up, set kernel attributes
    std::call_once(slot.once, [&]() {
        void* p = nullptr;
        slot.err = cudaGetSymbolAddress(&p, qc_static_scratch);
        if (slot.err == cudaSuccess) slot.base = static_cast<unsigned char*>(p);
        if (slot.err == cudaSuccess) {
            int optin = 0;
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            slot.err = prepare_kernels(static_cast<size_t>(optin));
        }
    });
    if (slot.err != cudaSuccess || !slot.base)
        return static_fail(QC_ERR_CUDA, std::string("static scratch set-up: ") + cudaGetErrorString(slot.err));
    unsigned char* S = slot.base;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // Hamiltonian parameters (FP64, sample-space mode)
    SysParams sp{};
    const int K = n_orb / 2;
    sp.n_orb = n_orb;
    sp.K = K;
    sp.na = sp.nb = n_elec / 2;
    sp.oa = sp.ob = n_elec / 2;
    sp.va = sp.vb = K - n_elec / 2;
    sp.nsa = sp.nsb = sp.oa * sp.va;
    sp.npoa = sp.npob = sp.oa * (sp.oa - 1) / 2;
    sp.npva = sp.npvb = sp.va * (sp.va - 1) / 2;
    sp.pairs = 2LL * sp.nsa + 2LL * sp.npoa * sp.npva + static_cast<long long>(sp.nsa) * sp.nsb;
    sp.e_core = e_core;
    sp.precision = QC_FP64;
    sp.h = h;
    sp.eri = eri;
    sp.J = reinterpret_cast<double*>(S + kOffJ);
    sp.X = reinterpret_cast<double*>(S + kOffX);
    sp.Jt = reinterpret_cast<double*>(S + kOffJt);
    sp.Xt = reinterpret_cast<double*>(S + kOffXt);
    unsigned long long* T = reinterpret_cast<unsigned long long*>(S + kOffTab);
    Counters* ctr = reinterpret_cast<Counters*>(S + kOffCtr);
    sp.err = &ctr->flags;
    double* part = reinterpret_cast<double*>(S + kOffPart);
    uint32_t* filter = reinterpret_cast<uint32_t*>(S + kOffFilter);
    unsigned long long* slots = reinterpret_cast<unsigned long long*>(S + kOffSlots);
    qc_eloc_summary* sum_dev = reinterpret_cast<qc_eloc_summary*>(S + kOffSum);

    // launch shape: the filtered kernel with the largest filter that leaves >= 8 warps
    int optin = 0, smc = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&smc, cudaDevAttrMultiProcessorCount, dev);
    const long long nt = n_u > 0 ? n_u : 1;
    int fw = 10;
    while (fw < kStaticFilterLog2 && (1LL << fw) < nt / 2 + 1) ++fw;
    const size_t wb = filtered_smem_bytes(sp, 1, fw) - filtered_smem_bytes(sp, 0, fw);
    int warps = 0;
    for (; fw >= 5; --fw) {
        const size_t base = filtered_smem_bytes(sp, 0, fw);
        if (base + wb > static_cast<size_t>(optin)) continue;
        warps = static_cast<int>((static_cast<size_t>(optin) - base) / wb);
        if (warps > kFilteredMaxWarps) warps = kFilteredMaxWarps;
        if (warps >= 8 || fw <= 10) break;
    }
    LaunchCfg cfg{};
    cfg.kernel = (fw >= 5 && warps >= 1) ? 2 : 1;
    cfg.unroll = 4;
    if (cfg.kernel == 2) {
        cfg.warps = warps;
        cfg.smem = filtered_smem_bytes(sp, warps, fw);
    } else {
        fw = 0;
        cfg.warps = 16;
        cfg.smem = direct_smem_bytes(sp, cfg.warps);
    }
    const int per_sm = max_active_ctas(cfg.kernel, QC_FP64, cfg.unroll, 32 * cfg.warps, cfg.smem);
    if (per_sm < 1) return static_fail(QC_ERR_CAPACITY, "main kernel cannot be resident with this shape");
    long long grid = static_cast<long long>(per_sm) * smc;
    const long long need = (n_u + cfg.warps - 1) / cfg.warps;
    cfg.grid = static_cast<int>(grid < need ? grid : (need > 0 ? need : 1));

    TableParams tp{};
    tp.keys = reinterpret_cast<const ulonglong2*>(samples);
    tp.psi = reinterpret_cast<const double2*>(psi);
    tp.n = n_u;
    tp.err = &ctr->flags;
    tp.slots = slots;
    tp.nb_mask = static_cast<unsigned>(next_pow2_u(2ULL * static_cast<unsigned long long>(nt)) - 1);
    tp.filter = cfg.kernel == 2 ? filter : nullptr;
    tp.fw = cfg.kernel == 2 ? fw : 0;

    EvalParams ep{};
    ep.samples = reinterpret_cast<const ulonglong2*>(samples);
    ep.psi = reinterpret_cast<const double2*>(psi);
    ep.counts = reinterpret_cast<const long long*>(counts);
    ep.n_u = n_u;
    ep.eloc = reinterpret_cast<double2*>(eloc);
    ep.ctr = ctr;
    ep.T = T;
    ep.mode = QC_SAMPLE;

#define QC_S(call, what)                                                                    \
    do {                                                                                    \
        e = (call);                                                                         \
        if (e != cudaSuccess) return static_fail(QC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e)); \
    } while (0)
    const size_t n3 = static_cast<size_t>(K) * K * K;
    static_prep_kernel<<<static_cast<unsigned>((n3 + 255) / 256), 256, 0, s>>>(
        eri, K, const_cast<double*>(sp.J), const_cast<double*>(sp.X), const_cast<double*>(sp.Jt),
        const_cast<double*>(sp.Xt), T);
    QC_S(cudaGetLastError(), "prep launch");
    QC_S(cudaMemsetAsync(ctr, 0, sizeof(Counters), s), "memset counters");
    QC_S(cudaMemsetAsync(slots, 0, 2 * (static_cast<size_t>(tp.nb_mask) + 1) * sizeof(unsigned long long), s),
         "memset table");
    if (cfg.kernel == 2) QC_S(cudaMemsetAsync(filter, 0, static_cast<size_t>(4) << fw, s), "memset filter");
    QC_S(launch_build_table(tp, n_orb, sp.na, sp.nb, T, slots, filter, nullptr, nullptr, ctr, s),
         "build_table launch");
    QC_S(launch_eloc_main(sp, tp, ep, cfg, s), "main kernel launch");
    QC_S(launch_reduce(ep, part, reduce_blocks(n_u), sum_dev, sp.pairs, s), "reduce launch");
    if (summary)
        QC_S(cudaMemcpyAsync(summary, sum_dev, sizeof(qc_eloc_summary), cudaMemcpyDefault, s), "summary copy");
#undef QC_S
    return QC_OK;
}
