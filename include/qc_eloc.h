/*
 * qc_eloc.h -- C ABI of libqc_eloc: sample-batched local energies on one GB300 GPU.
 *
 * The operation (arxiv 2506.23809, Sec. III-B, Eq. 5):
 *
 *     E_loc(x) = sum_x' <x|H|x'> psi(x') / psi(x)
 *
 * for every unique sampled occupation bitstring x, with H the second-quantized
 * Hamiltonian of Eq. 2 (Sec. II-A) built from real one-electron integrals h_pq and
 * two-electron integrals (pq|rs), and x' running over x itself and every single and
 * double excitation of x that conserves S_z.  Then (Eq. 1) the count-weighted mean
 *
 *     Ebar = sum_i c_i E_loc(x_i) / W,   W = sum_i c_i,
 *
 * and the weighted variance  var = sum_i c_i |E_loc(x_i) - Ebar|^2 / W  (two-pass).
 *
 * Two modes, after the two energies of Sec. IV-C-4:
 *   QC_SAMPLE  "sample-space energy": x' contributes only if it is in the table of
 *              unique samples (the lookup table of Sec. IV-C-4); others contribute 0.
 *   QC_FULL    "accurate energy": the caller supplies psi for every connected x' in a
 *              table; an x' missing from it is an error for that sample.
 *
 * Bitstrings (the occupation-number vector of Sec. II-A, interleaved spin orbitals
 * n_1a, n_1b, ..., n_Ka, n_Kb): spin orbital i is spatial orbital i/2 with spin alpha
 * when i is even; it is bit (i % 64) of 64-bit word i/64.  A key is two uint64 words
 * {w0, w1}; a table is sorted ascending as the unsigned 128-bit number w1*2^64 + w0,
 * with no duplicates.  n_orb <= 128.
 *
 * Fermionic sign convention: |x> = a+_{i1} a+_{i2} ... |0> with i1 < i2 < ...
 *
 * Integrals: h is K x K row-major FP64 (K = n_orb/2), symmetric; eri is K^4 row-major
 * FP64 in chemist notation, eri[((p*K+q)*K+r)*K+s] = (pq|rs), with the 8-fold symmetry
 * of real orbitals.  <pq|rs> = (pr|qs) between spin orbitals of matching spins.
 *
 * Memory ownership: pointers passed to qc_eloc_create are read during the call only
 * (the library copies the integrals to the device).  Array pointers passed to
 * qc_eloc_eval are caller-owned DEVICE memory, 16-byte aligned, and must stay valid
 * until the stream has passed the call.  The handle owns its device workspace.
 *
 * Errors: no C++ exception crosses this ABI.  Functions return QC_OK (0) or a negative
 * qc_status; qc_eloc_last_error() gives a message.  Conditions found on the device
 * (unsorted or duplicate keys, wrong electron counts, psi(x) = 0, a missing x' in FULL
 * mode, a bounded wait that ran out) are reported in qc_eloc_summary.status / .flags
 * once the stream reaches the end of the call; the affected samples get E_loc = NaN
 * and are left out of the reduction.
 *
 * Threads and streams: a handle may be used from one host thread at a time, and its
 * evaluations must not overlap on the device (they share the handle's workspace).
 * Different handles are independent.
 */
#ifndef QC_ELOC_H
#define QC_ELOC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int qc_status;

#define QC_OK              0
#define QC_PENDING         1   /* qc_eloc_poll: job not finished within the timeout */
#define QC_ERR_ARG        -1   /* bad argument (null pointer, size, alignment, n_orb) */
#define QC_ERR_UNSORTED   -2   /* table keys not ascending */
#define QC_ERR_DUP        -3   /* duplicate key */
#define QC_ERR_NELEC      -4   /* key with wrong alpha/beta electron count or bits >= n_orb */
#define QC_ERR_OOM        -5   /* device allocation failed */
#define QC_ERR_BUDGET     -6   /* serving: job can never fit the memory budget */
#define QC_ERR_CUDA       -7   /* CUDA runtime error (message in qc_eloc_last_error) */
#define QC_ERR_ZERO_PSI   -8   /* psi(x) == 0 for some sample */
#define QC_ERR_MISSING    -9   /* FULL mode: a connected x' is absent from the table */
#define QC_ERR_TIMEOUT   -10   /* a bounded device wait ran out */
#define QC_ERR_CAPACITY  -11   /* size beyond a compiled or reserved limit */
#define QC_ERR_COUNTS    -12   /* negative count */
#define QC_ERR_BOUNDS    -13   /* an index failed its bounds check (QC_CHECKED builds only) */

/* device-detected condition bits in qc_eloc_summary.flags */
#define QC_FLAG_UNSORTED   0x01u
#define QC_FLAG_DUP        0x02u
#define QC_FLAG_NELEC      0x04u
#define QC_FLAG_ZERO_PSI   0x08u
#define QC_FLAG_MISSING    0x10u
#define QC_FLAG_NEG_COUNT  0x20u
#define QC_FLAG_TABLE_FULL 0x40u
#define QC_FLAG_TIMEOUT    0x80u
#define QC_FLAG_LIST_FULL  0x100u  /* a hit list position fell outside hit_list_cap */
#define QC_FLAG_BOUNDS     0x200u  /* QC_CHECKED builds: an integral, table or list index was
                                      out of range (the access was skipped) */

/* precision */
#define QC_FP64        0   /* every floating-point step in FP64 */
#define QC_FP32_COMP   1   /* matrix elements x psi ratios in FP32 with compensated
                              (TwoSum) accumulation per sample; diagonal energy,
                              1/psi(x) and the reduction over samples in FP64 */
/* mode */
#define QC_SAMPLE      0
#define QC_FULL        1

/* options for qc_eloc_set_option */
#define QC_OPT_TIMING        1  /* 1: record per-phase CUDA events (qc_eloc_timings) */
#define QC_OPT_KERNEL        2  /* 0 auto, 1 direct probe of every x', 2 filtered */
#define QC_OPT_FILTER_LOG2W  3  /* 0 auto, else log2 of filter 32-bit words (5..15) */
#define QC_OPT_WARPS         4  /* 0 auto, else warps per CTA of the main kernel, 1..24 */
#define QC_OPT_UNROLL        5  /* 0 auto, else outer entries per inner pass (1, 2, 4) */
#define QC_OPT_GRID          6  /* 0 auto, else CTAs of the main kernel */
#define QC_OPT_PREFILTER     7  /* 1 (default): drop single excitations whose new spin string no
                                   table key has, and the doubles built on them; 0: off */
#define QC_OPT_CHUNK_PAIRS   9  /* excitation chunks: a sample's doubles are split over
                                   ceil(pairs / value) warps (at most 8), each adding its share
                                   and the last to finish combining them in chunk order; 0 or -1
                                   (the default) one warp per sample */
#define QC_OPT_LEAN          8  /* filtered kernel's per-warp lists: 0 auto (the layout that fits
                                   more warps), 1 stored pair lists, 2 pair lists formed on the
                                   fly from per-orbital values (same results, less shared memory) */
#define QC_OPT_JOIN         10  /* sample-space mode, filtered kernel: 0 auto (on from 16384
                                   table rows, from 2e8 table rows x connected pairs per sample,
                                   or from 512 rows when a sample has 50000 pairs), 1 off, 2 on.  On,
                                   the table rows are also grouped by alpha string and by beta
                                   string (a per-evaluation index); a short group that can hold
                                   connected keys is scanned row by row, the excitations into a
                                   long one enumerated.  Same connected set, so the same results
                                   up to the order of accumulation */
#define QC_OPT_SCAN_COST    11  /* join: a group is scanned when its rows x this / 4 are at most
                                   the excitations it replaces; 0 the default */
#define QC_OPT_BETA_COST    15  /* join, launches whose alpha list is capped (QC_OPT_ALPHA_SLOTS,
                                   or the automatic choice at large orbital counts): for a sample
                                   with at least 8 alpha' groups too long to scan in the list's
                                   first segment, the group of a beta' (a single excitation of its
                                   beta string in the table) is scanned for the rows of long alpha'
                                   groups when its rows x this / 4 are at most that number, instead
                                   of enumerating the beta' against each of them; 0 the default
                                   (8), -1 never, else 1..1024.  Same connected set either way */
#define QC_OPT_COUNT_WORK   12  /* 1: the local-energy kernel counts the work it does (read with
                                   qc_eloc_work); costs global atomics, so off (0) in timed runs */
#define QC_OPT_ALPHA_SLOTS  14  /* join: slots of the per-warp alpha single list (the alpha' groups
                                   too long to scan); 0 auto (all alpha singles, or fewer when that
                                   fits more warps), else that many (at least 1; the full list from
                                   the number of alpha singles up): a sample with more long alpha'
                                   groups enumerates them in segments */
#define QC_OPT_WAIT_LIMIT   13  /* test hook: iteration limit of each CTA's first wait for its copy
                                   of the Bloom filter (-1, the default: 2^24).  When it runs out
                                   the CTA sets QC_FLAG_TIMEOUT, waits for the copy with the
                                   default limit (so nothing is left in flight) and leaves without
                                   evaluating samples; the summary's status is QC_ERR_TIMEOUT */

typedef struct qc_eloc qc_eloc;

/* Result summary (written to host memory at the end of an evaluation). */
typedef struct {
    double   e_re, e_im;        /* Ebar (Eq. 1) over samples with finite E_loc */
    double   var;               /* sum c |E - Ebar|^2 / W */
    double   w;                 /* W = sum c over those samples */
    double   sum_ce_re, sum_ce_im; /* sum c E (for combining shards) */
    uint64_t n_used;            /* samples entering the reduction */
    uint64_t n_pairs;           /* connected (x, x') pairs enumerated, diagonal excluded */
    uint64_t n_hits;            /* pairs whose x' was found in the table */
    uint64_t n_missing;         /* FULL mode: pairs whose x' was absent */
    uint64_t n_bad;             /* samples with E_loc = NaN */
    uint32_t flags;             /* QC_FLAG_* */
    int32_t  status;            /* QC_OK or the most severe device-detected error */
} qc_eloc_summary;

/* Outputs of one evaluation.  eloc is required; the rest may be NULL.
 *   eloc        device complex128[n_u] (re, im interleaved)
 *   summary     host memory; page-locked memory keeps qc_eloc_eval asynchronous
 *   hit_count   device uint32[n_u]: table hits per sample (diagnostics)
 *   hit_rowsum  device uint64[n_u]: sum over hits of (table row + 1)
 *   hit_signsum device int64[n_u]:  sum over hits of phase * (table row + 1), where the
 *               phase is <x'| a+_i a+_j a_b a_a |x> with a < b the spin orbitals emptied
 *               and i < j those filled (+-1; for a single, <x'| a+_i a_a |x>).
 * Pair-by-pair diagnostics (the connected set of Eq. 5 restricted to the table, with the
 * phase of every element), written where each hit is resolved; both NULL or both given:
 *   hit_cursor  device int64[n_u], read and written: on entry, the position in hit_list of
 *               sample i's first hit (e.g. the exclusive prefix sum of the hit_count of an
 *               earlier evaluation of the same inputs); on exit, one past its last
 *   hit_list    device int64[hit_list_cap]: phase * (table row + 1) of each hit of sample i
 *               at positions entry cursor .. exit cursor - 1, in no particular order
 *   hit_list_cap entries of hit_list; a hit whose position falls outside it is not written
 *               and sets QC_FLAG_LIST_FULL (status QC_ERR_CAPACITY)
 * The lists cost an atomic add per 32 hits and a store per hit: for tests and debugging,
 * not for timed runs. */
typedef struct {
    double*          eloc;
    qc_eloc_summary* summary;
    uint32_t*        hit_count;
    uint64_t*        hit_rowsum;
    int64_t*         hit_signsum;
    int64_t*         hit_cursor;
    int64_t*         hit_list;
    int64_t          hit_list_cap;
} qc_eloc_out;

/* Create a handle for one Hamiltonian, the second-quantized H of Eq. 2 (Sec. II-A) given by
 * its one- and two-electron integrals h_pq and (pq|rs).  n_orb: even, 2..128.  n_elec: even, S_z = 0
 * (n_elec/2 electrons of each spin), 0 < n_elec < n_orb.  h, eri: host FP64 (layout
 * above), copied to the device.  e_core: constant added to every diagonal element.
 * precision: QC_FP64 | QC_FP32_COMP.  mode: QC_SAMPLE | QC_FULL.  Uses the current CUDA
 * device.  Returns QC_ERR_ARG on bad sizes, QC_ERR_OOM / QC_ERR_CUDA on device errors. */
qc_status qc_eloc_create(const double* h, const double* eri, double e_core, int n_orb,
                         int n_elec, int precision, int mode, qc_eloc** out);

qc_status qc_eloc_destroy(qc_eloc* handle);

/* Message for the last error on this handle; with NULL, of the last handle-less call
 * (qc_eloc_create, qc_eloc_eval_static) on the calling thread. */
const char* qc_eloc_last_error(const qc_eloc* handle);

/* Pre-size the workspace for up to n_u_max samples and n_table_max table rows, so that
 * later evaluations within those sizes allocate nothing (and can be graph-captured). */
qc_status qc_eloc_reserve(qc_eloc* handle, int64_t n_u_max, int64_t n_table_max);

qc_status qc_eloc_set_option(qc_eloc* handle, int option, int64_t value);

/* Structural pair count per sample: sum over spins of o v + C(o,2) C(v,2), plus
 * o_a v_a o_b v_b (o occupied, v empty spatial orbitals per spin). */
int64_t qc_eloc_pairs_per_sample(const qc_eloc* handle);

/* Evaluate E_loc(x) = sum_x' <x|H|x'> psi(x') / psi(x) (Eq. 5, Sec. III-B) for n_u samples,
 * x' running over x and every single and double excitation of x: QC_SAMPLE keeps the x'
 * present in the table (the "sample space" energy of Sec. IV-C-4), QC_FULL needs them all;
 * then the count-weighted energy and variance of Eq. 1 (Sec. II-A) into out->summary.
 * Runs on `stream` (a cudaStream_t, NULL = legacy default).
 *   samples  device uint64[n_u][2]   bitstrings to evaluate
 *   counts   device int64[n_u]       sample counts (>= 0)
 *   psi      device complex128[n_u]  psi(x), (re, im) interleaved
 *   table_keys, table_psi, n_table   the lookup table: sorted unique keys and their psi.
 *            QC_SAMPLE with table_keys == NULL: the table is the sample set itself
 *            (samples must then be sorted and unique).  A separate table lets one
 *            evaluate a shard of the samples against the whole sample set.
 *            QC_FULL: required; must hold every connected x' of every sample.
 * Asynchronous: returns after enqueueing.  Host-detectable argument errors return
 * synchronously.  May allocate device workspace on first use or growth (see
 * qc_eloc_reserve). */
qc_status qc_eloc_eval(qc_eloc* handle, const uint64_t* samples, const int64_t* counts,
                       const double* psi, int64_t n_u, const uint64_t* table_keys,
                       const double* table_psi, int64_t n_table, qc_eloc_out* out,
                       void* stream);

/* Per-phase device times of the last evaluation in ms: {table build, main kernel,
 * reduction}.  Needs QC_OPT_TIMING = 1; synchronizes on the recorded events. */
qc_status qc_eloc_timings(qc_eloc* handle, float* ms3);

/* ---- the accurate energy at scale: export the connected set, apply psi --------------
 * Sec. IV-C-4's "accurate energy" sums Eq. 5 over every x' connected to a sample, with psi
 * from the network.  For large systems the connected set is far larger than any table, so
 * it is exported in chunks of samples, the caller evaluates psi on it, and Eq. 5 is then
 * reduced against those values.  Every sample has exactly P = qc_eloc_pairs_per_sample()
 * connected x', written in a fixed order (position = class offset + u * n2 + w): alpha
 * singles, beta singles (w = occupied index * empty count + empty index over the spin's
 * ascending occupied / empty lists), alpha-alpha then beta-beta doubles (u an occupied
 * pair, w an empty pair; pair (p < q) has index q (q - 1) / 2 + p), alpha-beta doubles
 * (u an alpha single, w a beta single).
 *   qc_eloc_export: samples device uint64[n_u][2] (sorted order not required); outputs
 *     (device, any may be NULL) keys_out uint64[n_u * P][2], elems_out double[n_u * P]
 *     (the signed elements <x|H|x'> of Eq. 2 by the Slater-Condon rules, in the handle's
 *     precision), diag_out double[n_u] (<x|H|x> with e_core).  A sample with a wrong
 *     electron count gets NaN diagonal and elements and zero keys.
 *   qc_eloc_apply: E_loc(x_i) = diag_i + sum_j elems_ij psi_conn_ij / psi_i (FP64, fixed
 *     order), then the Eq. 1 reduction over the chunk into the handle's device summary and,
 *     if `summary` is given (host memory, page-locked keeps it asynchronous), a copy.
 *     psi device complex128[n_u], counts int64[n_u], elems / diag as exported, psi_conn
 *     complex128[n_u * P] in the export order, eloc_out complex128[n_u].  psi(x) = 0 gives
 *     NaN and QC_ERR_ZERO_PSI in the summary; n_hits is 0 (nothing is looked up).
 * Both are asynchronous on `stream`; errors as for qc_eloc_eval. */
qc_status qc_eloc_export(qc_eloc* handle, const uint64_t* samples, int64_t n_u, uint64_t* keys_out,
                         double* elems_out, double* diag_out, void* stream);
qc_status qc_eloc_apply(qc_eloc* handle, const double* psi, const int64_t* counts, int64_t n_u,
                        const double* elems, const double* diag, const double* psi_conn, double* eloc_out,
                        qc_eloc_summary* summary, void* stream);

/* ---- the sample table from a raw sample stream --------------------------------------
 * Sec. IV-C-4 builds a lookup table over the unique samples and names its construction as
 * what limits scaling.  qc_dedup turns a raw stream of sampled bitstrings (any order,
 * repeats) into the table qc_eloc_eval takes: ascending unique keys (unsigned 128-bit order,
 * word 1 most significant) and their multiplicities, on the device, asynchronously.
 *   raw        device uint64[n_raw][2], read only, 16-byte aligned; n_raw < 2^31
 *   n_orb      significant bits (1..128); every bit >= n_orb must be 0
 *   keys_out   device uint64[n_raw][2]: the first *n_unique rows are written
 *   counts_out device int64[n_raw]: the first *n_unique entries are written
 *   n_unique   device int64: the number of unique keys, or -1 if a key had a bit >= n_orb
 *              set (keys_out and counts_out are then not a table)
 *   work       device scratch of qc_dedup_workspace_bytes(n_raw) bytes, 256-byte aligned,
 *              not shared with a concurrent call
 * A stable radix sort over ceil(n_orb / 8) 8-bit digits, then run lengths; exact (integer
 * work), so the result is bit-identical to any correct sort.  Errors (QC_ERR_ARG,
 * QC_ERR_CAPACITY for a short workspace, QC_ERR_CUDA) return synchronously; the message
 * is qc_eloc_last_error(NULL). */
int64_t qc_dedup_workspace_bytes(int64_t n_raw);
qc_status qc_dedup(const uint64_t* raw, int64_t n_raw, int n_orb, uint64_t* keys_out, int64_t* counts_out,
                   int64_t* n_unique, void* work, size_t work_bytes, void* stream);

/* ---- Eq. 4: the energy gradient ----------------------------------------------------
 * d<E>/d theta_p = 2 Re < d_theta_p ln Psi*(n) (E_loc(n) - <E>) >_n (Sec. II-A, Eq. 4), the
 * average taken over the unique samples of the last qc_eloc_eval on this handle with their
 * counts: with W and Ebar that evaluation's Eq. 1 sums (read on the device, so this call
 * is asynchronous on the same stream after it),
 *   w_i = c_i (E_loc,i - Ebar) / W       (0 for a sample whose E_loc is not finite)
 *   g_p = 2 Re sum_i w_i dconj_ip
 * Arguments (device memory, caller-owned):
 *   eloc    complex128[n_u]: the E_loc written by that evaluation (same order, same n_u)
 *   counts  int64[n_u]
 *   dconj   complex128[n_u][n_par], row-major: d/d theta_p ln Psi*(n_i); NULL if g_out is
 *   w_out   complex128[n_u] or NULL
 *   g_out   double[n_par] or NULL
 * The contraction reads dconj once (HBM-bound) in a fixed summation order (deterministic).
 * Errors: QC_ERR_ARG (sizes, NULL, alignment: 16 bytes, counts and g_out 8), QC_ERR_OOM
 * for the handle's n_par x (<= 512) partials buffer. */
qc_status qc_eloc_grad(qc_eloc* handle, const double* eloc, const int64_t* counts, int64_t n_u,
                       const double* dconj, int64_t n_par, double* w_out, double* g_out, void* stream);

/* ---- allocation-free evaluation ---------------------------------------------------
 * qc_eloc_eval_static: the sample-space, FP64 evaluation of qc_eloc_eval (the table is
 * the sample set itself) for callers that cannot allocate device memory when they call
 * -- code inside a CUDA stream capture whose capture mode forbids unsafe calls, a
 * framework that owns all device memory through its own pool, or a serving loop that
 * must never wait on the allocator.  The paper has no counterpart; it is an interface
 * convenience of this library.
 *
 * It takes no handle and allocates nothing: no cudaMalloc, cudaFree or allocating
 * library routine.  The caller passes every input and output as device memory: h (K*K)
 * and eri (K^4) in the layouts above, samples / counts / psi as for qc_eloc_eval, and
 * eloc (complex128[n_u]).  summary may be host or device memory, or NULL.  The library's
 * own working memory (hash index, filter, integral tables, counters, reduction partials)
 * lives in one file-scope device array of QC_STATIC_SCRATCH_MB (about 8.4 MB): a GPU holds
 * it from the moment the library's device code is loaded there (with lazy module loading,
 * the first call on that device) until the process exits.
 *
 * Limits: n_u <= QC_STATIC_MAX_SAMPLES and n_orb <= QC_STATIC_MAX_ORB; larger sizes
 * return QC_ERR_CAPACITY without touching the GPU.  Errors of this call are read with
 * qc_eloc_last_error(NULL) on the calling thread.
 *
 * The first call on each device (with that device current) looks up the device address
 * of the array and sets kernel attributes; make that first call before any stream
 * capture.  All calls share the one array and each clears what must start at zero, so
 * calls that overlap on the GPU (other streams, other host threads) race and must be
 * serialized by the caller.  Asynchronous on `stream` like qc_eloc_eval. */
#define QC_STATIC_MAX_SAMPLES 131072
#define QC_STATIC_MAX_ORB     128
#define QC_STATIC_SCRATCH_MB  8.4
qc_status qc_eloc_eval_static(const double* h, const double* eri, double e_core, int n_orb,
                              int n_elec, const uint64_t* samples, const int64_t* counts,
                              const double* psi, int64_t n_u, double* eloc,
                              qc_eloc_summary* summary, void* stream);

/* ---- the batched form: many molecules, one persistent launch ---------------------
 * A batch groups sample-space handles (same precision, same device); each keeps its
 * Hamiltonian resident.  One batched step is: a memset of the batch's workspace, one table
 * build over every molecule's keys, one persistent local-energy launch that runs the
 * molecules one after another (longest estimated time first; every CTA takes samples of
 * the current molecule from a cursor and moves on when none are left), and the two reduction
 * passes -- five device operations for any number of molecules.  The per-sample
 * arithmetic is the single-molecule kernel's, so a molecule's results are bitwise the
 * same alone and in a batch.  Inputs are caller-owned device arrays, as for qc_eloc_eval.
 * `summaries` receives one qc_eloc_summary per molecule (host memory, page-locked for an
 * asynchronous copy).  qc_batch_graph_launch captures the step once as a CUDA graph on a
 * non-default stream and replays it; changing inputs or the shape drops the graph. */
typedef struct qc_batch qc_batch;
qc_status qc_batch_create(qc_eloc* const* handles, int n_mol, qc_batch** out);
qc_status qc_batch_destroy(qc_batch* batch);
const char* qc_batch_last_error(const qc_batch* batch);
qc_status qc_batch_set_inputs(qc_batch* batch, int mol, const uint64_t* samples, const int64_t* counts,
                              const double* psi, int64_t n_u, double* eloc);
/* One piece of a molecule for replicas that share its work (Alg. 2's cost-weighted split of
 * the unique samples): the next steps evaluate only rows [r0, r1) of the molecule's samples
 * (by row index, against its whole sample table; r1 < 0: to the end) and reduce Eq. 1 over
 * those rows only, so its summary holds the piece's partials -- W, sum c E (sum_ce_re/im)
 * and var -- which combine across pieces into the molecule's energy.  E_loc of each row is
 * bitwise the same as in a whole-molecule step.  (0, n_u) restores the whole molecule.
 * Call after qc_batch_set_inputs; QC_ERR_ARG on a bad range. */
qc_status qc_batch_set_rows(qc_batch* batch, int mol, int64_t r0, int64_t r1);
/* launch shape: unroll 0|2|4 (0 = 4), warps 0..20 (0 = 16, the widest CTA without register spills), samples a warp
 * takes per fetch 0..1024 (0 = 1) */
qc_status qc_batch_set_config(qc_batch* batch, int unroll, int warps, int chunk);
/* {unroll, warps, chunk, grid, molecules with samples, dynamic shared memory bytes} */
qc_status qc_batch_config(const qc_batch* batch, int64_t* cfg6);
qc_status qc_batch_eval(qc_batch* batch, qc_eloc_summary* summaries, void* stream);
qc_status qc_batch_graph_launch(qc_batch* batch, qc_eloc_summary* summaries, void* stream);
/* device ms of the last eager step: {table build, local-energy kernel, reduction} */
qc_status qc_batch_timings(qc_batch* batch, float* ms3);
/* excitation chunks of the batch's molecules (as QC_OPT_CHUNK_PAIRS of a handle: pairs
 * per chunk, 0 or -1 one warp per sample, the default) */
qc_status qc_batch_set_chunk_pairs(qc_batch* batch, int64_t chunk_pairs);
/* autotuner: times every candidate shape on this batch (best of `iters`), keeps the
 * fastest, then the excitation-chunk size at that shape; best4 (may be NULL) receives
 * {unroll, warps, samples per fetch, pairs per chunk (-1: one warp per sample)} */
qc_status qc_batch_autotune(qc_batch* batch, void* stream, int iters, int64_t* best4);

/* ---- the serving form: asynchronous requests, continuous batching -----------------
 * qc_server_create starts a scheduler thread on `device`.  qc_eloc_submit queues one
 * sample-space request and returns a ticket at once; the scheduler admits requests in
 * arrival order while their device footprint fits `budget_bytes` and fewer than
 * `max_slots` are in flight, keeps each molecule's Hamiltonian resident for later requests
 * with the same nonzero mol_key (least-recently-used eviction when the budget needs
 * room), and launches admitted requests whose inputs are on the device as batches
 * ("waves") on `n_streams` streams.  A wave holds about `quantum` enumerated pairs
 * (QC_SRV_OPT_QUANTUM, default 1e12): the oldest request with a guaranteed share of it
 * (QC_SRV_OPT_OLDEST_PCT, default half), the
 * others least remaining work first (none with more than 4x the oldest's remaining work,
 * which waits for a wave of its own), and the wave's sample rows stay within
 * QC_SRV_OPT_WAVE_ROWS unless it holds one request; a request that does not fit whole runs a slice of its
 * rows (against its whole sample table) and joins the next wave, and after a wave that ran
 * a slice the ready short requests (at most half a quantum) get a wave of their own, so
 * requests that arrive while a long one runs are served between its slices.  A request that can never fit the
 * budget is refused with QC_ERR_BUDGET at submit.  qc_eloc_poll waits up to timeout_us for
 * a ticket and returns QC_PENDING if it is not done; a finished ticket is released by the
 * poll that returns it.  A request's E_loc and energy are bitwise the same alone and in
 * any mix: the batch runs the single-molecule per-sample code, and a sliced request's
 * Eq. 1 reduction runs once, over all of its rows, with its last slice. */
typedef struct qc_server qc_server;
#define QC_JOB_BORROW_INTEGRALS 1  /* qc_eloc_job.flags: h and eri stay valid until the ticket
                                      is polled done, so submit does not copy them */
typedef struct {
    const double* h;       /* host FP64 integrals as for qc_eloc_create: copied at submit   */
    const double* eri;     /* unless the molecule (mol_key) is resident or flags borrows them */
    double e_core;
    int n_orb, n_elec, precision;  /* QC_FP64 | QC_FP32_COMP; sample-space mode             */
    int flags;             /* QC_JOB_BORROW_INTEGRALS or 0                                  */
    uint64_t mol_key;      /* nonzero: keep this Hamiltonian resident under this key        */
    const uint64_t* samples;  /* host uint64[n_u][2], sorted unique; with counts and psi,   */
    const int64_t* counts;    /* valid until the ticket is polled done                      */
    const double* psi;
    int64_t n_u;
    double* eloc_out;      /* host complex128[n_u] written when done, or NULL               */
} qc_eloc_job;
typedef struct {
    qc_eloc_summary summary;
    int32_t status, pad;
    double t_submit, t_admit, t_start, t_done;  /* seconds on the steady clock              */
} qc_eloc_result;
qc_status qc_server_create(int device, uint64_t budget_bytes, int max_slots, int n_streams,
                           qc_server** out);
qc_status qc_eloc_submit(qc_server* server, const qc_eloc_job* job, uint64_t* ticket);
qc_status qc_eloc_poll(qc_server* server, uint64_t ticket, qc_eloc_result* result, int timeout_us);
/* {device bytes in use, requests in flight, requests waiting, resident molecules} */
qc_status qc_server_stats(qc_server* server, uint64_t* stats4);
#define QC_SRV_OPT_QUANTUM    1  /* enumerated pairs per wave, >= 0 (0: no slicing, one wave takes all) */
#define QC_SRV_OPT_OLDEST_PCT 2  /* percent of a wave guaranteed to the oldest request, 1..100 (50) */
#define QC_SRV_OPT_WAVE_ROWS  3  /* sample rows a wave of several requests may hold, >= 0 (65536; 0:
                                    no limit): a longer request runs in a wave of its own, as the
                                    plain launch would, instead of delaying the requests batched
                                    with it until all of them are done */
qc_status qc_server_set_option(qc_server* server, int option, int64_t value);
qc_status qc_server_destroy(qc_server* server);  /* finishes queued work first */

/* Measurement probes (no counterpart in the paper; used by the benchmark to report measured
 * ceilings beside the derived ones).  On the current device, synchronously:
 *   alu_ops_per_s  integer throughput of the filter test's operation mix (shift, funnel
 *                  shift, shift, XOR; independent chains, 2,048 threads per SM), or NULL
 *   l2_gather_gbs  random 16-byte loads from a 4 MB table resident in L2, GB/s, or NULL
 * Allocates and frees about 4 MB of device memory. */
qc_status qc_probe_peaks(double* alu_ops_per_s, double* l2_gather_gbs, void* stream);

/* Work counts of the last evaluation with QC_OPT_COUNT_WORK = 1 (the units of the local-energy
 * kernel's roofline; no counterpart in the paper).  Waits for that evaluation's stream.
 * Writes the first min(n_fields, QC_WORK_FIELDS) of {samples set up, join table rows scanned
 * (16-byte entries), excitations tested against the shared-memory Bloom filter, candidates
 * probed in the bucket table (16-byte buckets), hits that are single excitations, same-spin
 * doubles, opposite-spin doubles, CTAs that copied the filter, hits found by the join's scans
 * (of all kinds; their keys are not loaded again), beta' = beta single excitations looked up
 * in the table's beta set by the join's beta' phase (8-byte slots), beta' groups that phase
 * scans} to work.  QC_ERR_ARG if n_fields < 1. */
#define QC_WORK_FIELDS 11
qc_status qc_eloc_work(qc_eloc* handle, uint64_t* work, int n_fields);

/* Test hook (no counterpart in the paper): the library's next `after` device allocations
 * (handles, their workspaces, batches, gradient partials) succeed and the one after them
 * fails as if the device were out of memory, so that error paths can be tested on the host
 * without exhausting a shared GPU.  A negative value turns it off (the default).  Process-wide. */
qc_status qc_test_fail_alloc(int64_t after);

/* Launch shape of the last evaluation on this handle: {kernel (1 direct, 2 filtered,
 * 3 filtered with pair lists formed on the fly), grid CTAs, warps per CTA, unroll, dynamic
 * shared memory bytes, log2 filter words, excitation chunks per sample}. */
qc_status qc_eloc_last_config(const qc_eloc* handle, int64_t* cfg7);

#ifdef __cplusplus
}
#endif

#endif /* QC_ELOC_H */
