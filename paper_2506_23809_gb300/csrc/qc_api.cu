// qc_api.cu -- host side of the libqc_eloc C ABI (declared in include/qc_eloc.h).
//
// A handle holds one Hamiltonian (Eq. 2: h_pq and (pq|rs)) on the device plus the
// workspace of an evaluation: the bucket hash index and Bloom filter over the lookup
// table (the sample-space lookup table of Sec. IV-C-4), the reduction partials of Eq. 1,
// counters and the device copy of the summary.  qc_eloc_eval only enqueues work on the
// caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "qc_eloc.h"
#include "qc_handle.h"
#include "qc_internal.h"


namespace {

thread_local std::string g_create_error;

qc_status fail(qc_eloc* h, qc_status st, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return st;
}

qc_status cuda_fail(qc_eloc* h, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(h, e == cudaErrorMemoryAllocation ? QC_ERR_OOM : QC_ERR_CUDA, m);
}

long long comb2(long long n) { return n < 2 ? 0 : n * (n - 1) / 2; }

// splitmix64 (Vigna): seeds the 128 entries of the linear key hash.
unsigned long long splitmix64(unsigned long long& s) {
    unsigned long long z = (s += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

unsigned long long next_pow2(unsigned long long v) {
    unsigned long long p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Buckets of two entries, at most a quarter of the slots filled: most probes of an
// absent key end at the first bucket.
unsigned long long table_buckets(long long n) {
    return next_pow2(2ULL * static_cast<unsigned long long>(std::max<long long>(n, 1)));
}

int ceil_log2(unsigned long long v) {
    int l = 0;
    while ((1ULL << l) < v) ++l;
    return l;
}

template <typename T>
void free_dev(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

bool prepared_devices[64] = {};

// qc_test_fail_alloc: allocations left before the injected failure (negative: none injected)
std::atomic<long long> g_fail_after{-1};

}  // namespace

void qc::set_handleless_error(const std::string& msg) { g_create_error = msg; }

cudaError_t qc::dev_alloc(void** p, size_t bytes) {
    if (g_fail_after.load(std::memory_order_relaxed) >= 0 && g_fail_after.fetch_sub(1) == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;  // injected: nothing was asked of the device
    }
    return cudaMalloc(p, bytes);
}

extern "C" {

const char* qc_eloc_last_error(const qc_eloc* h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

qc_status qc_eloc_create(const double* h, const double* eri, double e_core, int n_orb, int n_elec,
                         int precision, int mode, qc_eloc** out) {
    if (!out) return fail(nullptr, QC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!h || !eri) return fail(nullptr, QC_ERR_ARG, "h or eri is NULL");
    if (n_orb < 2 || n_orb > qc::kMaxOrb || (n_orb & 1))
        return fail(nullptr, QC_ERR_ARG, "n_orb must be even, 2..128");
    if (n_elec <= 0 || n_elec >= n_orb || (n_elec & 1))
        return fail(nullptr, QC_ERR_ARG, "n_elec must be even with 0 < n_elec < n_orb (S_z = 0)");
    if (precision != QC_FP64 && precision != QC_FP32_COMP)
        return fail(nullptr, QC_ERR_ARG, "precision must be QC_FP64 or QC_FP32_COMP");
    if (mode != QC_SAMPLE && mode != QC_FULL)
        return fail(nullptr, QC_ERR_ARG, "mode must be QC_SAMPLE or QC_FULL");

    qc_eloc* H = new (std::nothrow) qc_eloc();
    if (!H) return fail(nullptr, QC_ERR_OOM, "host allocation failed");
    H->n_orb = n_orb;
    H->n_elec = n_elec;
    H->K = n_orb / 2;
    H->na = H->nb = n_elec / 2;
    H->precision = precision;
    H->mode = mode;
    H->e_core = e_core;
    const int K = H->K;
    cudaError_t e = cudaGetDevice(&H->device);
    if (e != cudaSuccess) { qc_status s = cuda_fail(nullptr, e, "cudaGetDevice"); delete H; return s; }
    int smc = 0, optin = 0;
    cudaDeviceGetAttribute(&smc, cudaDevAttrMultiProcessorCount, H->device);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, H->device);
    H->sm_count = smc;
    H->smem_optin = static_cast<size_t>(optin);

    const size_t KK = static_cast<size_t>(K) * K, K4 = KK * KK;
    std::vector<double> J(KK), X(KK);
    for (int k = 0; k < K; ++k)
        for (int l = 0; l < K; ++l) {
            J[k * K + l] = eri[((static_cast<size_t>(k) * K + k) * K + l) * K + l];  // (kk|ll)
            // same-spin pair term of the diagonal: (kk|ll) - (kl|lk)
            X[k * K + l] = J[k * K + l] - eri[((static_cast<size_t>(k) * K + l) * K + l) * K + k];
        }
    const size_t K3 = KK * K;
    std::vector<double> Jt(K3), Xt(K3);
    for (int p = 0; p < K; ++p)
        for (int i = 0; i < K; ++i)
            for (int k = 0; k < K; ++k) {
                Jt[(static_cast<size_t>(p) * K + i) * K + k] = eri[((static_cast<size_t>(p) * K + i) * K + k) * K + k];  // (pi|kk)
                Xt[(static_cast<size_t>(p) * K + i) * K + k] = eri[((static_cast<size_t>(p) * K + k) * K + k) * K + i];  // (pk|ki)
            }
    // singles against the Aufbau reference (spatial orbitals below na / nb occupied)
    std::vector<double> Fref(2 * KK);
    for (int s = 0; s < 2; ++s)
        for (int a = 0; a < K; ++a)
            for (int i = 0; i < K; ++i) {
                double f = h[a * K + i];
                const size_t row = (static_cast<size_t>(a) * K + i) * K;
                for (int k = 0; k < H->na; ++k) f += Jt[row + k];
                for (int k = 0; k < H->nb; ++k) f += Jt[row + k];
                for (int k = 0; k < (s == 0 ? H->na : H->nb); ++k) f -= Xt[row + k];
                Fref[(static_cast<size_t>(s) * K + a) * K + i] = f;
            }
    std::vector<unsigned long long> T(128);
    unsigned long long seed = 0x51c0de5eedULL;
    for (auto& t : T) t = splitmix64(seed);

    auto cleanup = [&](qc_status s) { qc_eloc_destroy(H); return s; };
#define QC_TRY(call, what)                                          \
    do {                                                            \
        cudaError_t r_ = (call);                                    \
        if (r_ != cudaSuccess) return cleanup(cuda_fail(nullptr, r_, what)); \
    } while (0)
    QC_TRY(qc::dev_alloc(&H->d_h, KK * sizeof(double)), "cudaMalloc h");
    QC_TRY(cudaMemcpy(H->d_h, h, KK * sizeof(double), cudaMemcpyHostToDevice), "copy h");
    QC_TRY(qc::dev_alloc(&H->d_J, KK * sizeof(double)), "cudaMalloc J");
    QC_TRY(cudaMemcpy(H->d_J, J.data(), KK * sizeof(double), cudaMemcpyHostToDevice), "copy J");
    QC_TRY(qc::dev_alloc(&H->d_X, KK * sizeof(double)), "cudaMalloc X");
    QC_TRY(cudaMemcpy(H->d_X, X.data(), KK * sizeof(double), cudaMemcpyHostToDevice), "copy X");
    if (precision == QC_FP64) {
        QC_TRY(qc::dev_alloc(&H->d_Jt, K3 * sizeof(double)), "cudaMalloc Jt");
        QC_TRY(cudaMemcpy(H->d_Jt, Jt.data(), K3 * sizeof(double), cudaMemcpyHostToDevice), "copy Jt");
        QC_TRY(qc::dev_alloc(&H->d_Xt, K3 * sizeof(double)), "cudaMalloc Xt");
        QC_TRY(cudaMemcpy(H->d_Xt, Xt.data(), K3 * sizeof(double), cudaMemcpyHostToDevice), "copy Xt");
        QC_TRY(qc::dev_alloc(&H->d_Fref, 2 * KK * sizeof(double)), "cudaMalloc Fref");
        QC_TRY(cudaMemcpy(H->d_Fref, Fref.data(), 2 * KK * sizeof(double), cudaMemcpyHostToDevice), "copy Fref");
        QC_TRY(qc::dev_alloc(&H->d_eri, K4 * sizeof(double)), "cudaMalloc eri");
        QC_TRY(cudaMemcpy(H->d_eri, eri, K4 * sizeof(double), cudaMemcpyHostToDevice), "copy eri");
    } else {
        std::vector<float> h32(KK), e32(K4);
        for (size_t i = 0; i < KK; ++i) h32[i] = static_cast<float>(h[i]);
        for (size_t i = 0; i < K4; ++i) e32[i] = static_cast<float>(eri[i]);
        QC_TRY(qc::dev_alloc(&H->d_h32, KK * sizeof(float)), "cudaMalloc h32");
        QC_TRY(cudaMemcpy(H->d_h32, h32.data(), KK * sizeof(float), cudaMemcpyHostToDevice), "copy h32");
        std::vector<float> jt32(K3), xt32(K3);
        for (size_t i = 0; i < K3; ++i) {
            jt32[i] = static_cast<float>(Jt[i]);
            xt32[i] = static_cast<float>(Xt[i]);
        }
        QC_TRY(qc::dev_alloc(&H->d_Jt32, K3 * sizeof(float)), "cudaMalloc Jt32");
        QC_TRY(cudaMemcpy(H->d_Jt32, jt32.data(), K3 * sizeof(float), cudaMemcpyHostToDevice), "copy Jt32");
        QC_TRY(qc::dev_alloc(&H->d_Xt32, K3 * sizeof(float)), "cudaMalloc Xt32");
        QC_TRY(cudaMemcpy(H->d_Xt32, xt32.data(), K3 * sizeof(float), cudaMemcpyHostToDevice), "copy Xt32");
        QC_TRY(qc::dev_alloc(&H->d_eri32, K4 * sizeof(float)), "cudaMalloc eri32");
        QC_TRY(cudaMemcpy(H->d_eri32, e32.data(), K4 * sizeof(float), cudaMemcpyHostToDevice), "copy eri32");
    }
    QC_TRY(qc::dev_alloc(&H->d_T, 128 * sizeof(unsigned long long)), "cudaMalloc T");
    QC_TRY(cudaMemcpy(H->d_T, T.data(), 128 * sizeof(unsigned long long), cudaMemcpyHostToDevice), "copy T");
    QC_TRY(qc::dev_alloc(&H->d_ctr, sizeof(qc::Counters)), "cudaMalloc counters");
    QC_TRY(cudaMemset(H->d_ctr, 0, sizeof(qc::Counters)), "memset counters");
    QC_TRY(qc::dev_alloc(&H->d_sum, sizeof(qc_eloc_summary)), "cudaMalloc summary");
    if (H->device >= 0 && H->device < 64 && !prepared_devices[H->device]) {
        QC_TRY(qc::prepare_kernels(H->smem_optin), "cudaFuncSetAttribute");
        prepared_devices[H->device] = true;
    }
#undef QC_TRY

    qc::SysParams& sp = H->sp;
    sp.n_orb = n_orb;
    sp.K = K;
    sp.na = H->na;
    sp.nb = H->nb;
    sp.oa = H->na;
    sp.va = K - H->na;
    sp.ob = H->nb;
    sp.vb = K - H->nb;
    sp.nsa = sp.oa * sp.va;
    sp.nsb = sp.ob * sp.vb;
    sp.npoa = static_cast<int>(comb2(sp.oa));
    sp.npva = static_cast<int>(comb2(sp.va));
    sp.npob = static_cast<int>(comb2(sp.ob));
    sp.npvb = static_cast<int>(comb2(sp.vb));
    sp.pairs = static_cast<long long>(sp.nsa) + sp.nsb + static_cast<long long>(sp.npoa) * sp.npva +
               static_cast<long long>(sp.npob) * sp.npvb + static_cast<long long>(sp.nsa) * sp.nsb;
    sp.e_core = e_core;
    sp.precision = precision;
    sp.h = H->d_h;
    sp.eri = H->d_eri;
    sp.h32 = H->d_h32;
    sp.eri32 = H->d_eri32;
    sp.J = H->d_J;
    sp.X = H->d_X;
    sp.Jt = H->d_Jt;
    sp.Xt = H->d_Xt;
    sp.Fref = H->d_Fref;
    sp.err = &H->d_ctr->flags;
    sp.refA = H->na >= 64 ? ~0ULL : (1ULL << H->na) - 1ULL;
    sp.refB = H->nb >= 64 ? ~0ULL : (1ULL << H->nb) - 1ULL;
    sp.Jt32 = H->d_Jt32;
    sp.Xt32 = H->d_Xt32;
    *out = H;
    return QC_OK;
}

qc_status qc_eloc_destroy(qc_eloc* H) {
    if (!H) return QC_OK;
    free_dev(H->d_h);
    free_dev(H->d_eri);
    free_dev(H->d_J);
    free_dev(H->d_X);
    free_dev(H->d_Jt);
    free_dev(H->d_Xt);
    free_dev(H->d_Fref);
    free_dev(H->d_Jt32);
    free_dev(H->d_Xt32);
    free_dev(H->d_h32);
    free_dev(H->d_eri32);
    free_dev(H->d_T);
    free_dev(H->d_slots);
    free_dev(H->d_filter);
    free_dev(H->d_sets);
    free_dev(H->d_part);
    free_dev(H->d_ctr);
    free_dev(H->d_sum);
    free_dev(H->d_gpart);
    free_dev(H->d_cpart);
    free_dev(H->d_cticket);
    free_dev(H->d_join);
    free_dev(H->d_work);
    for (auto& ev : H->ev)
        if (ev) cudaEventDestroy(ev);
    delete H;
    return QC_OK;
}

int64_t qc_eloc_pairs_per_sample(const qc_eloc* H) { return H ? H->sp.pairs : -1; }

qc_status qc_eloc_set_option(qc_eloc* H, int option, int64_t value) {
    if (!H) return QC_ERR_ARG;
    switch (option) {
        case QC_OPT_TIMING: H->opt_timing = value ? 1 : 0; return QC_OK;
        case QC_OPT_KERNEL:
            if (value < 0 || value > 2) return fail(H, QC_ERR_ARG, "QC_OPT_KERNEL: 0, 1 or 2");
            H->opt_kernel = static_cast<int>(value);
            return QC_OK;
        case QC_OPT_FILTER_LOG2W:
            if (value != 0 && (value < 5 || value > 15)) return fail(H, QC_ERR_ARG, "QC_OPT_FILTER_LOG2W: 0 or 5..15");
            H->opt_fw = static_cast<int>(value);
            return QC_OK;
        case QC_OPT_WARPS:
            if (value < 0 || value > qc::kFilteredMaxWarps) return fail(H, QC_ERR_ARG, "QC_OPT_WARPS: 0..24");
            H->opt_warps = static_cast<int>(value);
            return QC_OK;
        case QC_OPT_UNROLL:
            if (!(value == 0 || value == 1 || value == 2 || value == 4))
                return fail(H, QC_ERR_ARG, "QC_OPT_UNROLL: 0, 1, 2 or 4");
            H->opt_unroll = static_cast<int>(value);
            return QC_OK;
        case QC_OPT_PREFILTER: H->opt_prefilter = value ? 1 : 0; return QC_OK;
        case QC_OPT_CHUNK_PAIRS:
            if (value < -1) return fail(H, QC_ERR_ARG, "QC_OPT_CHUNK_PAIRS: -1, 0 or pairs per chunk");
            H->opt_chunk_pairs = value;
            return QC_OK;
        case QC_OPT_LEAN:
            if (value < 0 || value > 2) return fail(H, QC_ERR_ARG, "QC_OPT_LEAN: 0, 1 or 2");
            H->opt_lean = static_cast<int>(value);
            return QC_OK;
        case QC_OPT_JOIN:
            if (value < 0 || value > 2) return fail(H, QC_ERR_ARG, "QC_OPT_JOIN: 0, 1 or 2");
            H->opt_join = static_cast<int>(value);
            return QC_OK;
        case QC_OPT_SCAN_COST:
            if (value < 0 || value > 1024) return fail(H, QC_ERR_ARG, "QC_OPT_SCAN_COST: 0..1024");
            H->opt_scan_cost = static_cast<int>(value);
            return QC_OK;
        case QC_OPT_BETA_COST:
            if (value < -1 || value > 1024) return fail(H, QC_ERR_ARG, "QC_OPT_BETA_COST: -1..1024");
            H->opt_beta_cost = static_cast<int>(value);
            return QC_OK;
        case QC_OPT_COUNT_WORK: H->opt_count_work = value ? 1 : 0; return QC_OK;
        case QC_OPT_ALPHA_SLOTS:
            if (value < 0 || value > 4096) return fail(H, QC_ERR_ARG, "QC_OPT_ALPHA_SLOTS: 0..4096");
            H->opt_alpha_slots = static_cast<int>(value);
            return QC_OK;
        case QC_OPT_WAIT_LIMIT:
            if (value >= 0x7fffffff) return fail(H, QC_ERR_ARG, "QC_OPT_WAIT_LIMIT: -1 or 0..2^31-2");
            H->opt_wait_limit = value < 0 ? 0 : static_cast<int>(value) + 1;
            return QC_OK;
        case QC_OPT_GRID:
            if (value < 0 || value > (1 << 20)) return fail(H, QC_ERR_ARG, "QC_OPT_GRID: 0..2^20");
            H->opt_grid = static_cast<int>(value);
            return QC_OK;
        default: return fail(H, QC_ERR_ARG, "unknown option");
    }
}

}  // extern "C"

namespace qc {

// The join index of an n_table-row table in one allocation: sort keys, group sizes and
// starts, entries, the sample order with its two scratch arrays, then the sort's workspace.
JoinLayout join_layout(long long n_table) {
    auto a256 = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t nt = static_cast<size_t>(std::max<long long>(n_table, 1));
    const size_t nb = static_cast<size_t>(table_buckets(n_table));
    JoinLayout L{};
    L.len = a256(2 * nt * 4);
    L.start = L.len + a256(2 * nb * 4);
    L.ent = L.start + a256(2 * nb * 4);
    L.ord = L.ent + a256(2 * nt * 16);
    L.ws = L.ord + 3 * a256(nt * 4);
    L.total = L.ws + join_workspace_bytes(static_cast<long long>(nt), static_cast<unsigned>(nb));
    return L;
}

qc_status ensure_join(qc_eloc* H, long long n_table) {
    const size_t need = join_layout(n_table).total;
    if (need > H->join_cap) {
        free_dev(H->d_join);
        H->join_cap = 0;
        cudaError_t e = qc::dev_alloc(&H->d_join, need);
        if (e != cudaSuccess) return cuda_fail(H, e, "cudaMalloc join index");
        H->join_cap = need;
    }
    return QC_OK;
}

// Workspace growth: bucket table for n_table keys, filter of 2^fw words, partials.
qc_status ensure_workspace(qc_eloc* H, long long n_u, long long n_table, int fw) {
    const size_t entries = 2 * static_cast<size_t>(table_buckets(n_table));
    if (entries > H->slots_cap) {
        free_dev(H->d_slots);
        H->slots_cap = 0;
        cudaError_t e = qc::dev_alloc(&H->d_slots, entries * sizeof(unsigned long long));
        if (e != cudaSuccess) return cuda_fail(H, e, "cudaMalloc hash table");
        H->slots_cap = entries;
    }
    if (fw > 0 && H->opt_prefilter) {
        const size_t se = static_cast<size_t>(table_buckets(n_table));
        if (se > H->sets_cap) {
            free_dev(H->d_sets);
            H->sets_cap = 0;
            cudaError_t e = qc::dev_alloc(&H->d_sets, 2 * se * sizeof(unsigned long long));
            if (e != cudaSuccess) return cuda_fail(H, e, "cudaMalloc spin-string sets");
            H->sets_cap = se;
        }
    }
    const size_t words = fw > 0 ? (static_cast<size_t>(1) << fw) : 0;
    if (words > H->filter_cap) {
        free_dev(H->d_filter);
        H->filter_cap = 0;
        cudaError_t e = qc::dev_alloc(&H->d_filter, words * sizeof(uint32_t));
        if (e != cudaSuccess) return cuda_fail(H, e, "cudaMalloc filter");
        H->filter_cap = words;
    }
    const int nblk = qc::reduce_blocks(n_u);
    if (nblk > H->part_cap) {
        free_dev(H->d_part);
        H->part_cap = 0;
        cudaError_t e = qc::dev_alloc(&H->d_part, static_cast<size_t>(nblk) * 4 * sizeof(double));
        if (e != cudaSuccess) return cuda_fail(H, e, "cudaMalloc partials");
        H->part_cap = nblk;
    }
    return QC_OK;
}

// Kernel choice and launch shape (the defaults the autotuner can override).
qc_status choose_config(qc_eloc* H, long long n_u, long long n_table, qc::LaunchCfg& c, int& fw) {
    const qc::SysParams& sp = H->sp;
    int kernel = H->opt_kernel;
    if (H->mode == QC_FULL) kernel = 1;  // every x' must be looked up: no filter
    if (kernel == 0) kernel = 2;
    fw = 0;
    int warps = 0;
    int lean = 0;
    // the join needs the spin-string sets and strings that are never empty (no spin without
    // electrons); by default taken when qc::join_by_default says so (below that its index
    // build, a few microseconds per launch, outweighs what it saves); built with U = 4
    // (its sort keys are 32-bit: both sets' slots and the sentinel below 2^32)
    const bool join = kernel == 2 && H->mode == QC_SAMPLE && H->opt_prefilter && H->na > 0 && H->nb > 0 &&
                      n_table > 0 && table_buckets(n_table) <= (1ULL << 30) &&
                      (H->opt_join == 2 || (H->opt_join == 0 && qc::join_by_default(n_table, sp.pairs)));
    if (kernel == 2) {
        // filter sized for ~16 bits per key, 2^10..2^15 words; then as many warps as fit,
        // shrinking the filter while that leaves fewer than 8.  With the join, which sends
        // fewer excitations through the filter, the most warps that fit with at least ~5
        // filter bits per key (measured: N=52, 10^5 keys, 20 warps at 2^14 words beat 18 at
        // 2^15; N=76, 2*10^5 keys, 16 warps at 2^15 beat 20 at 2^14).  Both list layouts are
        // tried (unless forced) and the one that fits more warps is taken (stored lists on a
        // tie; without the join, the larger filter first).
        int want = H->opt_fw;
        if (want == 0) {
            want = ceil_log2(static_cast<unsigned long long>(std::max<long long>(n_table, 1)) / 2 + 1);
            want = std::min(15, std::max(10, want));
        }
        int best_fw = 0, best_w = 0, best_lean = 0, best_acap = 0;
        // with the join the alpha list may get fewer slots than alpha singles (filled in
        // segments) when that fits more warps; the full list on a tie
        const int acaps[3] = {H->opt_alpha_slots, 64, 32};
        for (int ai = 0; ai < (join ? (H->opt_alpha_slots ? 1 : 3) : 1); ++ai)
        for (int ln = 0; ln < 2; ++ln) {
            if ((H->opt_lean == 1 && ln == 1) || (H->opt_lean == 2 && ln == 0)) continue;
            // a capacity of at least the alpha singles is the full list
            const int acap = acaps[ai] >= sp.nsa ? 0 : acaps[ai];
            if (ai > 0 && acap == 0) continue;  // an automatic candidate that caps nothing
            const size_t wb = qc::filtered_smem_bytes(sp, 1, want, ln, join, acap) -
                              qc::filtered_smem_bytes(sp, 0, want, ln, join, acap);
            int f = want, w = 0;
            if (join && H->opt_fw == 0) {
                const int min_f = std::min(want, std::max(10, ceil_log2(static_cast<unsigned long long>(
                                                                   std::max<long long>(n_table, 1)) * 5 / 32 + 1)));
                int bf = 0, bw = 0;
                for (int g = want; g >= min_f; --g) {
                    const size_t base = qc::filtered_smem_bytes(sp, 0, g, ln, join, acap);
                    if (base + wb > H->smem_optin) continue;
                    const int fit = static_cast<int>((H->smem_optin - base) / wb);
                    const int wg = std::min(qc::kFilteredMaxWarps, H->opt_warps ? H->opt_warps : fit);
                    if (wg <= fit && wg > bw) {
                        bw = wg;
                        bf = g;
                    }
                }
                f = bw > 0 ? bf : 4;
                w = bw;
            } else {
                for (; f >= 5; --f) {
                    const size_t base = qc::filtered_smem_bytes(sp, 0, f, ln, join, acap);
                    if (base + wb > H->smem_optin) continue;
                    const int fit = static_cast<int>((H->smem_optin - base) / wb);
                    w = std::min(qc::kFilteredMaxWarps, H->opt_warps ? H->opt_warps : fit);
                    if (w > fit) continue;
                    if (H->opt_fw == 0 && w < 8 && f > 10) continue;  // prefer occupancy
                    break;
                }
            }
            if (f < 5 || w < 1) continue;
            if (w > best_w || (w == best_w && !join && f > best_fw)) {
                best_fw = f;
                best_w = w;
                best_lean = ln;
                best_acap = acap;
            }
        }
        fw = best_fw;
        warps = best_w;
        lean = best_lean;
        c.acap = best_acap;
        if (warps < 1) {
            if (H->opt_kernel == 2) return fail(H, QC_ERR_CAPACITY, "filtered kernel does not fit shared memory");
            kernel = 1;
            fw = 0;
            lean = 0;
        }
    }
    c.kernel = kernel;
    c.lean = lean;
    c.join = kernel == 2 && join;
    c.unroll = c.join ? 4 : (H->opt_unroll ? H->opt_unroll : 4);
    if (!c.join) c.acap = 0;
    if (kernel == 2) {
        c.warps = warps;
        c.smem = qc::filtered_smem_bytes(sp, warps, fw, lean, c.join, c.acap);
    } else {
        c.warps = std::min(qc::kFilteredMaxWarps, H->opt_warps ? H->opt_warps : 16);
        c.smem = qc::direct_smem_bytes(sp, c.warps);
    }
    int per_sm = qc::max_active_ctas(c.kernel, H->precision, c.unroll, 32 * c.warps, c.smem, c.lean, c.join, c.acap > 0);
    if (per_sm < 1) return fail(H, QC_ERR_CAPACITY, "main kernel cannot be resident with this shape");
    long long grid = H->opt_grid ? H->opt_grid : static_cast<long long>(per_sm) * H->sm_count;
    const long long cp = H->opt_chunk_pairs == 0 ? qc::kDefaultChunkPairs : H->opt_chunk_pairs;
    c.chunks = qc::exc_chunks(sp.pairs, cp);
    const long long need = (n_u * c.chunks + c.warps - 1) / c.warps;
    grid = std::max<long long>(1, std::min(grid, need));
    c.grid = static_cast<int>(grid);
    return QC_OK;
}

}  // namespace qc

using qc::choose_config;
using qc::ensure_workspace;

extern "C" {

qc_status qc_eloc_reserve(qc_eloc* H, int64_t n_u_max, int64_t n_table_max) {
    if (!H) return QC_ERR_ARG;
    if (n_u_max < 0 || n_table_max < 0) return fail(H, QC_ERR_ARG, "negative size");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != H->device) return fail(H, QC_ERR_ARG, "handle belongs to another device");
    qc::LaunchCfg c{};
    int fw = 0;
    const long long nt = std::max<long long>(n_table_max, n_u_max);
    qc_status s = choose_config(H, std::max<long long>(n_u_max, 1), nt, c, fw);
    if (s != QC_OK) return s;
    s = ensure_workspace(H, n_u_max, nt, fw);
    if (s == QC_OK && c.join && nt > 0) s = qc::ensure_join(H, nt);  // the sample-space join's index
    return s;
}

qc_status qc_eloc_eval(qc_eloc* H, const uint64_t* samples, const int64_t* counts, const double* psi,
                       int64_t n_u, const uint64_t* table_keys, const double* table_psi,
                       int64_t n_table, qc_eloc_out* out, void* stream) {
    if (!H) return QC_ERR_ARG;
    if (!out || (!out->eloc && n_u > 0)) return fail(H, QC_ERR_ARG, "out or out->eloc is NULL");
    if (n_u < 0 || n_table < 0) return fail(H, QC_ERR_ARG, "negative size");
    if (n_u > 0 && (!samples || !counts || !psi)) return fail(H, QC_ERR_ARG, "samples, counts or psi is NULL");
    if (n_u >= (1LL << 31)) return fail(H, QC_ERR_CAPACITY, "n_u >= 2^31");
    const bool own_table = (table_keys == nullptr);
    if (H->mode == QC_FULL && own_table) return fail(H, QC_ERR_ARG, "QC_FULL needs table_keys/table_psi");
    if (!own_table && !table_psi) return fail(H, QC_ERR_ARG, "table_psi is NULL");
    const ulonglong2* tk = reinterpret_cast<const ulonglong2*>(own_table ? samples : table_keys);
    const double2* tpsi = reinterpret_cast<const double2*>(own_table ? psi : table_psi);
    const long long nt = own_table ? n_u : n_table;
    if (nt >= 0xfffffffeLL) return fail(H, QC_ERR_CAPACITY, "table larger than 2^32 - 2 rows");
    auto misaligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; };
    if ((n_u > 0 && (misaligned(samples) || misaligned(psi) || misaligned(out->eloc))) ||
        (nt > 0 && (misaligned(tk) || misaligned(tpsi))))
        return fail(H, QC_ERR_ARG, "device arrays must be 16-byte aligned");
    if (counts && (reinterpret_cast<uintptr_t>(counts) & 7u)) return fail(H, QC_ERR_ARG, "counts must be 8-byte aligned");
    if ((out->hit_cursor == nullptr) != (out->hit_list == nullptr))
        return fail(H, QC_ERR_ARG, "hit_cursor and hit_list go together");
    if (out->hit_list != nullptr &&
        (out->hit_list_cap < 0 || (reinterpret_cast<uintptr_t>(out->hit_list) & 7u) ||
         (reinterpret_cast<uintptr_t>(out->hit_cursor) & 7u)))
        return fail(H, QC_ERR_ARG, "hit_list / hit_cursor must be 8-byte aligned, hit_list_cap >= 0");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != H->device) return fail(H, QC_ERR_ARG, "handle belongs to another device");

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    qc::LaunchCfg cfg{};
    int fw = 0;
    qc_status st = choose_config(H, n_u, nt, cfg, fw);
    if (st != QC_OK) return st;
    st = ensure_workspace(H, n_u, nt, fw);
    if (st != QC_OK) return st;
    H->last_cfg = cfg;
    H->last_fw = fw;

    if (H->opt_timing) {
        for (auto& ev : H->ev)
            if (!ev) {
                cudaError_t e = cudaEventCreate(&ev);
                if (e != cudaSuccess) return cuda_fail(H, e, "cudaEventCreate");
            }
    }
    cudaError_t e;
#define QC_CHK(call, what)                              \
    do {                                                \
        e = (call);                                     \
        if (e != cudaSuccess) return cuda_fail(H, e, what); \
    } while (0)
    if (H->opt_timing) QC_CHK(cudaEventRecord(H->ev[0], s), "cudaEventRecord");
    QC_CHK(cudaMemsetAsync(H->d_ctr, 0, sizeof(qc::Counters), s), "memset counters");

    qc::TableParams tp{};
    tp.keys = tk;
    tp.psi = tpsi;
    tp.n = nt;
    tp.err = &H->d_ctr->flags;
    tp.slots = H->d_slots;
    tp.nb_mask = static_cast<unsigned>(table_buckets(nt) - 1);
    tp.filter = (cfg.kernel == 2) ? H->d_filter : nullptr;
    tp.fw = (cfg.kernel == 2) ? fw : 0;
    const size_t nbuckets = static_cast<size_t>(tp.nb_mask) + 1;
    unsigned long long* aset = nullptr;
    unsigned long long* bset = nullptr;
    if (cfg.kernel == 2 && H->opt_prefilter) {
        aset = H->d_sets;
        bset = H->d_sets + nbuckets;
        tp.aset = aset;
        tp.bset = bset;
        tp.set_mask = tp.nb_mask;
        QC_CHK(cudaMemsetAsync(H->d_sets, 0, 2 * nbuckets * sizeof(unsigned long long), s), "memset sets");
    }
    QC_CHK(cudaMemsetAsync(H->d_slots, 0, 2 * nbuckets * sizeof(unsigned long long), s), "memset table");
    if (cfg.kernel == 2) QC_CHK(cudaMemsetAsync(H->d_filter, 0, (static_cast<size_t>(4) << fw), s), "memset filter");
    // join index regions: slot keys, group sizes and starts, entries (strings, rows), sort space
    const bool join = cfg.join && nt > 0;
    auto a256 = [](size_t v) { return (v + 255) / 256 * 256; };
    const qc::JoinLayout JL = qc::join_layout(nt);
    const size_t jo_len = JL.len, jo_start = JL.start, jo_ent = JL.ent, jo_ord = JL.ord, jo_ws = JL.ws;
    unsigned* jkey = nullptr;
    unsigned* jlen = nullptr;
    const unsigned* join_order = nullptr;
    if (join) {
        st = qc::ensure_join(H, nt);
        if (st != QC_OK) return st;
        jkey = reinterpret_cast<unsigned*>(H->d_join);
        jlen = reinterpret_cast<unsigned*>(H->d_join + jo_len);
        QC_CHK(cudaMemsetAsync(jlen, 0, 2 * nbuckets * sizeof(unsigned), s), "memset join sizes");
    }
    QC_CHK(qc::launch_build_table(tp, H->n_orb, H->na, H->nb, H->d_T, H->d_slots, H->d_filter, aset, bset,
                                  H->d_ctr, s, jkey, jlen),
           "build_table launch");
    if (join) {
        unsigned* jstart = reinterpret_cast<unsigned*>(H->d_join + jo_start);
        ulonglong2* gent = reinterpret_cast<ulonglong2*>(H->d_join + jo_ent);
        // samples heavy first by the sizes of their own groups: the table's rows, or a caller's
        // samples no more numerous than its rows (the order's buffers hold one entry per row)
        unsigned* order = nullptr;
        unsigned* pa = nullptr;
        unsigned* pb = nullptr;
        if (own_table || n_u <= nt) {
            order = reinterpret_cast<unsigned*>(H->d_join + jo_ord);
            pa = reinterpret_cast<unsigned*>(H->d_join + jo_ord + a256(static_cast<size_t>(nt) * 4));
            pb = reinterpret_cast<unsigned*>(H->d_join + jo_ord + 2 * a256(static_cast<size_t>(nt) * 4));
            QC_CHK(cudaMemsetAsync(pa, 0, 2 * a256(static_cast<size_t>(nt) * 4), s), "memset sample order sizes");
        }
        QC_CHK(qc::launch_join_index(tp, static_cast<unsigned>(nbuckets), H->d_join + jo_ws, jkey, jlen, jstart,
                                     gent, s, order, pa, pb,
                                     own_table ? nullptr : reinterpret_cast<const ulonglong2*>(samples), n_u, H->d_T),
               "join index launch");
        join_order = order;
        tp.jstart = jstart;
        tp.jlen = jlen;
        tp.gent = gent;
        tp.scan_cost = H->opt_scan_cost ? H->opt_scan_cost : qc::kDefaultScanCost;
        tp.beta_cost = qc::beta_cost_of(H->opt_beta_cost);
        tp.alpha_cap = cfg.acap;
    }
    if (H->opt_timing) QC_CHK(cudaEventRecord(H->ev[1], s), "cudaEventRecord");

    qc::EvalParams ep{};
    ep.samples = reinterpret_cast<const ulonglong2*>(samples);
    ep.psi = reinterpret_cast<const double2*>(psi);
    ep.counts = reinterpret_cast<const long long*>(counts);
    ep.n_u = n_u;
    ep.eloc = reinterpret_cast<double2*>(out->eloc);
    ep.hit_count = out->hit_count;
    ep.hit_rowsum = reinterpret_cast<unsigned long long*>(out->hit_rowsum);
    ep.hit_signsum = reinterpret_cast<long long*>(out->hit_signsum);
    ep.hit_cursor = reinterpret_cast<long long*>(out->hit_cursor);
    ep.hit_list = reinterpret_cast<long long*>(out->hit_list);
    ep.hit_list_cap = out->hit_list != nullptr ? out->hit_list_cap : 0;
    if (H->opt_count_work) {
        if (!H->d_work) QC_CHK(qc::dev_alloc(&H->d_work, sizeof(qc::WorkCounters)), "cudaMalloc work counters");
        QC_CHK(cudaMemsetAsync(H->d_work, 0, sizeof(qc::WorkCounters), s), "memset work counters");
        ep.work = H->d_work;
        H->work_stream = s;
        H->work_recorded = true;
    }
    ep.ctr = H->d_ctr;
    ep.wait_limit = H->opt_wait_limit;
    ep.T = H->d_T;
    ep.mode = H->mode;
    ep.lean = cfg.lean;
    ep.chunks = cfg.chunks;
    ep.order = join_order;
    if (cfg.chunks > 1 && n_u > 0) {
        const size_t recs = static_cast<size_t>(n_u) * cfg.chunks;
        if (recs > H->cpart_cap) {
            free_dev(H->d_cpart);
            H->cpart_cap = 0;
            QC_CHK(qc::dev_alloc(&H->d_cpart, recs * sizeof(qc::ChunkRec)), "cudaMalloc chunk records");
            H->cpart_cap = recs;
        }
        if (static_cast<size_t>(n_u) > H->cticket_cap) {
            free_dev(H->d_cticket);
            H->cticket_cap = 0;
            QC_CHK(qc::dev_alloc(&H->d_cticket, static_cast<size_t>(n_u) * sizeof(unsigned)), "cudaMalloc chunk tickets");
            H->cticket_cap = static_cast<size_t>(n_u);
        }
        QC_CHK(cudaMemsetAsync(H->d_cticket, 0, static_cast<size_t>(n_u) * sizeof(unsigned), s), "memset tickets");
        ep.cpart = H->d_cpart;
        ep.cticket = H->d_cticket;
    }
    QC_CHK(qc::launch_eloc_main(H->sp, tp, ep, cfg, s), "main kernel launch");
    if (H->opt_timing) QC_CHK(cudaEventRecord(H->ev[2], s), "cudaEventRecord");
    QC_CHK(qc::launch_reduce(ep, H->d_part, qc::reduce_blocks(n_u), H->d_sum, H->sp.pairs, s),
           "reduce launch");
    if (H->opt_timing) QC_CHK(cudaEventRecord(H->ev[3], s), "cudaEventRecord");
    if (out->summary)
        QC_CHK(cudaMemcpyAsync(out->summary, H->d_sum, sizeof(qc_eloc_summary), cudaMemcpyDeviceToHost, s),
               "summary copy");
#undef QC_CHK
    H->ev_recorded = H->opt_timing != 0;
    return QC_OK;
}

qc_status qc_eloc_timings(qc_eloc* H, float* ms3) {
    if (!H || !ms3) return QC_ERR_ARG;
    if (!H->ev_recorded) return fail(H, QC_ERR_ARG, "no timed evaluation (set QC_OPT_TIMING first)");
    cudaError_t e = cudaEventSynchronize(H->ev[3]);
    if (e != cudaSuccess) return cuda_fail(H, e, "cudaEventSynchronize");
    for (int i = 0; i < 3; ++i) {
        e = cudaEventElapsedTime(&ms3[i], H->ev[i], H->ev[i + 1]);
        if (e != cudaSuccess) return cuda_fail(H, e, "cudaEventElapsedTime");
    }
    return QC_OK;
}

qc_status qc_test_fail_alloc(int64_t after) {
    g_fail_after.store(after < 0 ? -1 : static_cast<long long>(after));
    return QC_OK;
}

qc_status qc_eloc_work(qc_eloc* H, uint64_t* work, int n_fields) {
    if (!H || !work || n_fields < 1) return QC_ERR_ARG;
    if (!H->work_recorded) return fail(H, QC_ERR_ARG, "no evaluation counted its work (set QC_OPT_COUNT_WORK first)");
    qc::WorkCounters w{};
    cudaError_t e = cudaMemcpyAsync(&w, H->d_work, sizeof(w), cudaMemcpyDeviceToHost, H->work_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(H->work_stream);
    if (e != cudaSuccess) return cuda_fail(H, e, "work counters copy");
    const unsigned long long v[QC_WORK_FIELDS] = {w.samples, w.scan_rows, w.tests, w.probes, w.hits_single,
                                                  w.hits_same, w.hits_ab, w.ctas, w.hits_scanned,
                                                  w.beta_looked, w.beta_groups};
    for (int i = 0; i < n_fields && i < QC_WORK_FIELDS; ++i) work[i] = v[i];
    return QC_OK;
}

// Launch shape of the last evaluation: {kernel, grid, warps, unroll, smem bytes, filter log2 words,
// excitation chunks}.
qc_status qc_eloc_last_config(const qc_eloc* H, int64_t* cfg7) {
    if (!H || !cfg7) return QC_ERR_ARG;
    // 1 direct, 2 filtered, 3 filtered with lean lists, 4 / 5 the same two with the join
    cfg7[0] = H->last_cfg.kernel == 2 ? 2 + (H->last_cfg.lean ? 1 : 0) + (H->last_cfg.join ? 2 : 0)
                                      : H->last_cfg.kernel;
    cfg7[1] = H->last_cfg.grid;
    cfg7[2] = H->last_cfg.warps;
    cfg7[3] = H->last_cfg.unroll;
    cfg7[4] = static_cast<int64_t>(H->last_cfg.smem);
    cfg7[5] = H->last_fw;
    cfg7[6] = H->last_cfg.chunks > 1 ? H->last_cfg.chunks : 1;
    return QC_OK;
}

}  // extern "C"
