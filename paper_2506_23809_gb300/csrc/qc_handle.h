// qc_handle.h -- the handle of the C ABI (opaque to callers) and host helpers shared by
// the handle API (qc_api.cu) and the many-molecule batch (qc_batch.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "qc_eloc.h"
#include "qc_internal.h"

struct qc_eloc {
    int device = 0;
    int n_orb = 0, n_elec = 0, K = 0, na = 0, nb = 0, precision = 0, mode = 0;
    double e_core = 0.0;
    qc::SysParams sp{};
    double* d_h = nullptr;
    double* d_eri = nullptr;
    double* d_J = nullptr;
    double* d_X = nullptr;
    double* d_Jt = nullptr;
    double* d_Xt = nullptr;
    double* d_Fref = nullptr;
    float* d_Jt32 = nullptr;
    float* d_Xt32 = nullptr;
    float* d_h32 = nullptr;
    float* d_eri32 = nullptr;
    unsigned long long* d_T = nullptr;
    unsigned long long* d_slots = nullptr;
    size_t slots_cap = 0;  // 64-bit entries
    uint32_t* d_filter = nullptr;
    size_t filter_cap = 0;  // 32-bit words
    unsigned long long* d_sets = nullptr;  // alpha set | beta set
    size_t sets_cap = 0;                   // entries per set
    double* d_part = nullptr;
    int part_cap = 0;  // reduction blocks
    qc::Counters* d_ctr = nullptr;
    qc_eloc_summary* d_sum = nullptr;
    double* d_gpart = nullptr;  // Eq. 4 contraction partials
    size_t gpart_cap = 0;       // doubles
    void* d_cpart = nullptr;    // excitation-chunk records
    size_t cpart_cap = 0;       // records
    unsigned* d_cticket = nullptr;
    size_t cticket_cap = 0;     // samples
    unsigned char* d_join = nullptr;  // sample-space join index and its sort workspace
    size_t join_cap = 0;              // bytes
    long long opt_chunk_pairs = 0;  // 0 default, < 0 one chunk per sample, else pairs per chunk
    int opt_timing = 0, opt_kernel = 0, opt_fw = 0, opt_warps = 0, opt_unroll = 0, opt_grid = 0;
    int opt_prefilter = 1;
    int opt_lean = 0;  // 0 auto, 1 stored pair lists, 2 formed on the fly
    int opt_join = 0;  // 0 auto, 1 off, 2 on (sample-space mode, filtered kernel)
    int opt_scan_cost = 0;  // 0 default, else 4 x the cost of a scanned row in enumerated pairs
    int opt_beta_cost = 0;  // QC_OPT_BETA_COST: 0 default, -1 never, else its factor
    int opt_count_work = 0;  // QC_OPT_COUNT_WORK
    int opt_wait_limit = 0;  // QC_OPT_WAIT_LIMIT + 1 (0: the kernel's default)
    int opt_alpha_slots = 0;  // QC_OPT_ALPHA_SLOTS (0: auto)
    qc::WorkCounters* d_work = nullptr;
    cudaStream_t work_stream = nullptr;  // stream of the last evaluation that counted work
    bool work_recorded = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool ev_recorded = false;
    int sm_count = 0;
    size_t smem_optin = 0;
    qc::LaunchCfg last_cfg{};
    int last_fw = 0;
    std::string err;
};

namespace qc {
// grow the handle's workspace for n_u samples, an n_table-row table and 2^fw filter words
qc_status ensure_workspace(qc_eloc* H, long long n_u, long long n_table, int fw);
// the sample-space join's index for an n_table-row table: layout and growth
struct JoinLayout {
    size_t len, start, ent, ord, ws, total;
};
JoinLayout join_layout(long long n_table);
qc_status ensure_join(qc_eloc* H, long long n_table);
// kernel choice and launch shape for n_u samples against an n_table-row table
qc_status choose_config(qc_eloc* H, long long n_u, long long n_table, LaunchCfg& c, int& fw);
// point a batch at another set of handles, reusing its device allocations
qc_status batch_retarget(qc_batch* B, qc_eloc* const* handles, int n_mol);
// one slice of a molecule's rows per step (the serving form's long requests)
qc_status batch_set_slice(qc_batch* B, int mol, long long r0, long long r1, bool reduce, Counters* ctr);
// grow the batch's device buffers stream-ordered on s and copy its parameter blocks there
qc_status batch_set_alloc_stream(qc_batch* B, cudaStream_t s);
}  // namespace qc
