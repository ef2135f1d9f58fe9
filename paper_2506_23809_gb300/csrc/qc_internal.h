// qc_internal.h -- device-side parameter blocks shared by the host API and the kernels
// of libqc_eloc (not part of the public ABI; see include/qc_eloc.h for that).
#pragma once

#include <cstdint>
#include <string>
#include <cuda_runtime.h>

namespace qc {

constexpr int kMaxOrb = 128;     // spin orbitals (two 64-bit words)
constexpr int kMaxSpatial = 64;  // spatial orbitals per spin
constexpr int kPairLut = 2016;   // C(64, 2): colex pair index -> (i, j), i < j < 64
// Warps per CTA of the main kernel at most: its launch bound (768 threads) caps it at 80
// registers a thread, which it fits without spills since the sample's constants moved to
// shared memory; 24 warps beat 20 (96 registers) by 6% at N=52 (measured: 2.81 / 3.00 ms)
constexpr int kFilteredMaxWarps = 24;
// Warps per CTA of the batch kernel at most (its launch bounds: 512 or 640 threads)
constexpr int kBatchMaxWarps = 20;

// One Hamiltonian (Eq. 2) resident on the device.
struct SysParams {
    int n_orb, K;        // spin / spatial orbitals
    int na, nb;          // electrons per spin
    int oa, va, ob, vb;  // occupied / empty spatial orbitals per spin
    int nsa, nsb;        // singles per spin: o*v
    int npoa, npva, npob, npvb;  // C(o,2), C(v,2) per spin
    long long pairs;     // structural connected pairs per sample
    double e_core;
    int precision;       // 0 FP64, 1 FP32 compensated
    const double* h;     // K*K  FP64
    const double* eri;   // K^4  FP64 (FP64 precision)
    const float* h32;    // K*K  FP32 (FP32 precision)
    const float* eri32;  // K^4  FP32 (FP32 precision)
    const double* J;     // K*K  (kk|ll)  FP64
    const double* X;     // K*K  (kk|ll) - (kl|lk)  FP64 (the diagonal's same-spin pair term)
    const double* Jt;    // K^3  [a][i][k] = (ai|kk)  FP64 (single excitations)
    const double* Xt;    // K^3  [a][i][k] = (ak|ki)  FP64
    const float* Jt32;   // K^3  FP32 copies (FP32 precision)
    const float* Xt32;
    // single excitations relative to a reference determinant (FP64 precision; NULL: none):
    // Fref[s][a][i] = h_ai + sum_{k in ref, both spins} (ai|kk) - sum_{k in ref, spin s} (ak|ki)
    // for the Aufbau strings refA, refB (spatial orbitals 0 .. na - 1, 0 .. nb - 1)
    const double* Fref;  // 2*K*K
    unsigned long long refA, refB;
    unsigned* err;       // QC_CHECKED builds: flags word a failed bounds check sets (QC_FLAG_BOUNDS)
};

// The lookup table: sorted unique keys, their psi, and the device hash index over them.
struct TableParams {
    const ulonglong2* keys;
    const double2* psi;
    long long n;
    const unsigned long long* slots;  // 2 entries per 16-byte bucket
    unsigned nb_mask;                 // buckets - 1 (power of two)
    const uint32_t* filter;           // blocked Bloom filter, (1 << fw) 32-bit words
    int fw;
    // exact sets of the alpha and beta spatial strings of the table keys (open addressing,
    // 0 = empty); NULL disables the spin-string prefilter
    const unsigned long long* aset;
    const unsigned long long* bset;
    unsigned set_mask;
    // sample-space join index (NULL: not built).  Set slot s of the alpha set (s + set size of
    // the beta set) owns the group of table rows whose alpha (beta) string sits in it:
    // entries jstart[s] .. jstart[s] + jlen[s] - 1 of gent, in row order.  An entry holds the
    // row's string of the other spin (beta strings in alpha groups, alpha strings in beta
    // groups) and the row.
    const unsigned* jstart;
    const unsigned* jlen;
    const ulonglong2* gent;
    int scan_cost;  // a group is scanned when len * scan_cost <= 4 * (pairs it replaces)
    int beta_cost;  // a beta' group is scanned when len * beta_cost <= 4 * (long alpha' groups); 0 never
    int alpha_cap;  // join: slots of the per-warp alpha single list (0: all alpha singles)
    unsigned* err;  // QC_CHECKED builds: flags word a failed bounds check sets (QC_FLAG_BOUNDS)
};

// Counters and flags of one evaluation (device memory, zeroed at the start of a call).
struct Counters {
    unsigned long long hits;
    unsigned long long missing;
    unsigned long long bad;
    unsigned long long invalid;   // samples with a wrong electron count (not evaluated)
    unsigned int flags;
    unsigned int ticket;     // last-block ticket of the reduction passes
    double mean_re, mean_im;  // Ebar from pass 1
    long long w;              // sum of counts (pass 1)
    double sce_re, sce_im;
    unsigned long long used;
    unsigned long long next;  // next sample a warp of the local-energy kernel takes
};

// Work the local-energy kernel did in one launch (QC_OPT_COUNT_WORK; diagnostics, off in
// timed runs): the units the roofline's algorithmic bytes and operations are counted in.
struct WorkCounters {
    unsigned long long samples;      // samples set up (valid electron counts)
    unsigned long long scan_rows;    // join: table rows scanned (one 16-byte entry each)
    unsigned long long tests;        // excitations tested against the shared-memory filter
    unsigned long long probes;       // candidates probed in the bucket table
    unsigned long long hits_single;  // hits resolved: single excitations
    unsigned long long hits_same;    //   same-spin doubles
    unsigned long long hits_ab;      //   opposite-spin doubles
    unsigned long long ctas;         // CTAs that copied the filter into shared memory
    unsigned long long hits_scanned; // hits found by the join's scans (any kind; exact, no key load)
    unsigned long long beta_looked;  // join: beta' looked up in the beta set for the beta' phase
    unsigned long long beta_groups;  // join: beta' groups the beta' phase scans
};

struct EvalParams {
    const ulonglong2* samples;
    const double2* psi;
    const long long* counts;
    long long n_u;
    double2* eloc;
    uint32_t* hit_count;
    unsigned long long* hit_rowsum;
    long long* hit_signsum;
    long long* hit_cursor;        // pair-by-pair diagnostics (NULL: off): per-sample list cursor
    long long* hit_list;          //   phase * (row + 1) of every hit
    long long hit_list_cap;
    WorkCounters* work;           // QC_OPT_COUNT_WORK (NULL: off)
    int wait_limit;               // QC_OPT_WAIT_LIMIT + 1 for the first filter-copy wait (0: the default)
    int pad2_;
    Counters* ctr;
    const unsigned long long* T;  // 128 entries of the linear key hash
    int mode;                     // 0 SAMPLE, 1 FULL
    int lean;                     // pair hash lists formed on the fly (batch kernel)
    int chunks;                   // excitation chunks per sample (1: a warp owns a sample)
    int pad_;
    void* cpart;                  // chunks > 1: ChunkRec[n_u * chunks]
    unsigned* cticket;            // chunks > 1: per-sample count of finished chunks (zeroed)
    const unsigned* order;        // the order warps take samples in (NULL: index order)
};

// One excitation chunk's share of a sample (chunks > 1): the warp sums of its hits.
struct ChunkRec {
    double re, im;
    unsigned long long hits, rowsum;
    long long signsum;
    unsigned long long missing;
};

// Excitation chunks of a sample with `pairs` connected pairs: ceil(pairs / chunk_pairs),
// 1..8; chunk_pairs <= 0 means one chunk (a warp owns the whole sample).  Off by default:
// every chunk repeats the sample's set-up, which on the measured workloads costs more than
// the shorter tails save; the batch autotuner tries sizes around kChunkPairsProbe.
constexpr long long kDefaultChunkPairs = 0;
// Sample-space join: a group of table rows is scanned when len * kDefaultScanCost / 4 is at
// most the number of excitations that scanning it replaces.
constexpr int kDefaultScanCost = 4;
// The join's beta' phase: a beta' group is scanned for the rows of long alpha' groups when
// len * kDefaultBetaCost / 4 is at most their number (a scanned row costs about twice a
// filter test and its share of false-positive probes).
constexpr int kDefaultBetaCost = 8;
inline int beta_cost_of(int opt) { return opt == 0 ? kDefaultBetaCost : opt < 0 ? 0 : opt; }
constexpr long long kJoinMinRows = 16384;  // the join's default: tables from this many rows, or
// from kJoinMinPairRows table rows x connected pairs per sample, or from kJoinBigRows rows when
// a sample has at least kJoinBigPairs connected pairs (measured break-even: about 2e8 pair-rows
// at N=52; at N=76 and above the join wins from 1,000 rows, at N=124 6x faster at 8,000 rows)
constexpr long long kJoinMinPairRows = 200000000LL;
constexpr long long kJoinBigPairs = 50000, kJoinBigRows = 512;
inline bool join_by_default(long long n_table, long long pairs_per_sample) {
    return n_table >= kJoinMinRows || n_table * pairs_per_sample >= kJoinMinPairRows ||
           (pairs_per_sample >= kJoinBigPairs && n_table >= kJoinBigRows);
}
constexpr long long kChunkPairsProbe = 262144;
inline int exc_chunks(long long pairs, long long chunk_pairs) {
    if (chunk_pairs <= 0) return 1;
    const long long c = (pairs + chunk_pairs - 1) / chunk_pairs;
    return static_cast<int>(c < 1 ? 1 : (c > 8 ? 8 : c));
}

// A batch of molecules evaluated in one persistent launch.
struct MolWork {  // writable workspace of one molecule of a batch
    unsigned long long* slots;
    uint32_t* filter;
    unsigned long long* aset;
    unsigned long long* bset;
    Counters* ctr;
    double* part;  // nblk x 4 doubles
    void* sum;     // qc_eloc_summary (device)
    // sample-space join (null jkey: none): this molecule's 2n sort keys and values, the
    // batch's group sizes, the molecule's first slot key and the batch's sentinel key
    unsigned* jkey;
    unsigned* jval;
    unsigned* jlen;
    unsigned jbase, jsent;
    int nblk;      // reduction blocks: the single-molecule path's count, so results match it bitwise
    int pad;
};
struct MolParams {
    SysParams sp;
    TableParams tp;
    EvalParams ep;
    int active_warps;    // warps of a CTA that work on this molecule's samples (the rest idle)
    unsigned warp_stride;  // this molecule's per-warp shared-memory region
    long long r0, r1;      // rows evaluated by this launch (the table holds all n_u rows)
    long long red_lo, red_hi;  // rows the Eq. 1 reduction runs over
};
struct BatchParams {
    const MolParams* mols;
    const int* order;          // molecules in the order they are run (largest estimated cost first)
    unsigned long long* next;  // per position in `order`: next sample to hand out (zeroed before the launch)
    int n_mol;
    int chunk;                 // samples a warp takes per fetch
};

struct LaunchCfg {
    int kernel;   // 1 direct, 2 filtered
    int grid;
    int warps;
    int unroll;
    size_t smem;
    int lean;     // filtered kernel: pair hash lists formed on the fly
    int chunks;   // excitation chunks per sample
    int join;     // filtered kernel: sample-space join (short row groups scanned)
    int acap;     // join: slots of the per-warp alpha single list (0: all)
};

// host-side launchers (qc_kernels.cu)
cudaError_t launch_build_table(const TableParams& tp, int n_orb, int na, int nb,
                               const unsigned long long* T, unsigned long long* slots,
                               uint32_t* filter, unsigned long long* aset,
                               unsigned long long* bset, Counters* ctr, cudaStream_t s,
                               unsigned* jkey = nullptr, unsigned* jlen = nullptr);
cudaError_t launch_eloc_main(const SysParams& sp, const TableParams& tp, const EvalParams& ep,
                             const LaunchCfg& cfg, cudaStream_t s);
// the same kernels with the hit lists and work counters compiled in (qc_kernels_diag.cu)
cudaError_t launch_eloc_main_diag(const SysParams& sp, const TableParams& tp, const EvalParams& ep,
                                  const LaunchCfg& cfg, cudaStream_t s);
cudaError_t prepare_kernels_diag(size_t max_smem);
cudaError_t launch_reduce(const EvalParams& ep, double* partials, int nblk,
                          void* summary_dev, long long pairs_per_sample, cudaStream_t s);
int max_active_ctas(int kernel, int precision, int unroll, int threads, size_t smem, int lean = 0, int join = 0,
                    int seg = 0);
// batch: build every molecule's table in one launch (key_off: prefix of table sizes, device)
cudaError_t launch_build_batch(const MolParams* mols, const MolWork* work, const long long* key_off,
                               int n_mol, long long n_keys, cudaStream_t s);
cudaError_t launch_eloc_batch(const BatchParams& bp, int precision, int unroll, int grid, int warps,
                              size_t smem, cudaStream_t s, bool join = false);
cudaError_t launch_reduce_batch(const MolParams* mols, const MolWork* work, int n_mol, int max_blocks,
                                cudaStream_t s);
int max_active_batch(int precision, int unroll, int threads, size_t smem, bool join = false);
// join: the batch kernel has the join's queues; acap: the molecule's alpha list slots (0: all)
size_t batch_warp_bytes(const SysParams& sp, bool lean, bool join, int acap);
cudaError_t prepare_batch_kernels(size_t max_smem, size_t* dyn_limit);
cudaError_t prepare_kernels(size_t max_smem);
size_t filtered_smem_bytes(const SysParams& sp, int warps, int fw, bool lean = false, bool join = false, int acap = 0);
size_t direct_smem_bytes(const SysParams& sp, int warps);
size_t smem_fixed_bytes();  // CTA tables at the head of the main kernels' dynamic shared memory
int reduce_blocks(long long n);
// sample-space join index over an n-row table whose slot keys K0 wrote (qc_join.cu):
// jkey[0, 2n) slot keys (alpha rows, then beta rows offset by the set size), jlen counts
size_t join_workspace_bytes(long long n, unsigned set_size);
// with order (the table is the sample set): also the heavy-first order of the samples (pa, pb:
// n entries each of scratch)
// with order and samples (not the table's rows; n_samples <= tp.n, T the key hash's table): the
// heavy-first order of those samples, their groups looked up in the table's sets
cudaError_t launch_join_index(const TableParams& tp, unsigned set_size, void* ws, unsigned* jkey,
                              unsigned* jlen, unsigned* jstart, ulonglong2* gent, cudaStream_t s,
                              unsigned* order = nullptr, unsigned* pa = nullptr, unsigned* pb = nullptr,
                              const ulonglong2* samples = nullptr, long long n_samples = 0,
                              const unsigned long long* T = nullptr);
// a batch's join index: m sort items (every molecule's 2n keys, values written by K0),
// n_slots group sizes (slot_base[M] = n_slots, the sentinel key); entries in one gent array
size_t join_batch_workspace_bytes(long long m, unsigned long long n_slots);
// with order: also each joining molecule's rows heavy first (row_base: the molecules' first
// rows in order / pa / pb, m / 2 rows in all)
cudaError_t launch_join_batch(const MolParams* mols, const unsigned* slot_base, int n_mol, long long m,
                              unsigned long long n_slots, void* ws, unsigned* jkey, unsigned* jval,
                              unsigned* jlen, unsigned* jstart, ulonglong2* gent, cudaStream_t s,
                              const unsigned* row_base = nullptr, unsigned* order = nullptr,
                              unsigned* pa = nullptr, unsigned* pb = nullptr);
// in-place exclusive prefix sum of n u32 (qc_dedup.cu); sums: (n / 4096 + 2) u32 of scratch
cudaError_t exclusive_scan_u32(unsigned* a, long long n, unsigned* sums, cudaStream_t s);
// message returned by qc_eloc_last_error(NULL) on this thread (qc_api.cu)
void set_handleless_error(const std::string& msg);
// Device allocations of the handle, batch and gradient paths go through here, so that a test
// can make one of them fail on the host (qc_test_fail_alloc) and check the error paths.
cudaError_t dev_alloc(void** p, size_t bytes);
template <typename T>
inline cudaError_t dev_alloc(T** p, size_t bytes) {
    return dev_alloc(reinterpret_cast<void**>(p), bytes);
}

}  // namespace qc
