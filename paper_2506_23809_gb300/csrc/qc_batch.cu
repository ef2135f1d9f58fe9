// qc_batch.cu -- the batched form: many molecules (each a qc_eloc handle, its integrals
// already resident on the device) evaluated together.  One step is five device
// operations whatever the number of molecules -- a memset of the batch arena, one table
// build over every molecule's keys, one persistent local-energy launch that runs the
// molecules one after another (largest first, every CTA taking samples of the current
// molecule from its cursor), and the two reduction passes -- and it can be captured once
// as a CUDA graph.  The launch shape (unroll, warps per CTA, samples per fetch) is picked
// by an autotuner that times candidates on the batch itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "qc_eloc.h"
#include "qc_handle.h"
#include "qc_internal.h"

namespace {

struct BatchInput {
    const uint64_t* samples = nullptr;
    const int64_t* counts = nullptr;
    const double* psi = nullptr;
    int64_t n_u = 0;
    double* eloc = nullptr;
    // a slice of a long request (serving): rows [r0, r1) are evaluated against the whole
    // table, counters accumulate in caller memory across slices, and the Eq. 1 reduction
    // runs over all rows only with the last slice
    int64_t r0 = 0, r1 = -1;  // r1 < 0: all rows
    bool reduce = true;
    qc::Counters* ctr = nullptr;  // null: the batch's own counters, zeroed every step
    // a replica's piece (qc_batch_set_rows): rows [r0, r1) by row index, in row order, with
    // the Eq. 1 reduction over those rows only (the summary holds the piece's partials)
    bool piece = false;
};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

unsigned long long next_pow2(unsigned long long v) {
    unsigned long long p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

struct qc_batch {
    int device = 0;
    int precision = 0;
    int n_mol = 0;
    int mol_cap = 0;
    int sm_count = 0;
    size_t dyn_limit = 0;
    std::vector<qc_eloc*> handles;
    std::vector<BatchInput> in;
    qc::MolParams* d_mols = nullptr;
    qc::MolWork* d_work = nullptr;
    long long* d_key_off = nullptr;
    int* d_order = nullptr;  // molecules in run order
    unsigned char* d_arena = nullptr;
    size_t arena_cap = 0, arena_bytes = 0;
    qc_eloc_summary* d_sums = nullptr;
    // sample-space join over every molecule (one index for the batch): sort keys and values,
    // group starts, entries, sort space and the molecules' first slot keys, outside the
    // zeroed arena (the group sizes are inside it)
    bool join = false;
    unsigned char* d_join = nullptr;
    size_t join_cap = 0;
    long long j_items = 0;
    unsigned long long j_slots = 0;
    size_t jo_val = 0, jo_start = 0, jo_ent = 0, jo_ws = 0, jo_base = 0, ja_len = 0;
    size_t jo_rbase = 0, jo_order = 0, jo_pab = 0;  // rows heavy first per molecule, and their scratch
    // launch shape
    int unroll = 4, warps = 0, chunk = 1;
    long long chunk_pairs = qc::kDefaultChunkPairs;  // excitation chunks (<= 0: one warp per sample)
    int warps_used = 0, grid = 0, n_run = 0, red_blocks = 1;
    long long n_keys = 0;
    size_t smem = 0;
    bool dirty = true;
    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    qc_eloc_summary* graph_sums = nullptr;
    // timing of the last eager evaluation
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool timed = false;
    // non-null (the serving form's lanes): the arena and the join index grow stream-ordered on
    // this stream and the parameter blocks are copied on it, so a wave's set-up never waits for
    // work on other streams (a plain cudaFree waits for the whole device)
    cudaStream_t alloc_stream = nullptr;
    std::string err;
};

namespace {

qc_status bfail(qc_batch* b, qc_status st, const std::string& m) {
    if (b) b->err = m;
    return st;
}
qc_status bcuda(qc_batch* b, cudaError_t e, const char* what) {
    return bfail(b, e == cudaErrorMemoryAllocation ? QC_ERR_OOM : QC_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

int filter_log2(long long n) {
    int fw = 10;
    while (fw < 15 && (1LL << fw) < n / 2 + 1) ++fw;
    return fw;
}

// Lay out every molecule's workspace in one arena (after the per-molecule sample cursors),
// fill the parameter blocks and order the molecules by estimated running time, longest
// first, so that the small ones fill the tail of the launch.
qc_status prepare(qc_batch* B) {
    // host-to-device copies of the parameter blocks: on the allocation stream when the batch
    // has one (ordered after its stream-ordered allocations; pageable sources are staged
    // before the call returns), else synchronous
    auto h2d = [B](void* dst, const void* src, size_t bytes) {
        return B->alloc_stream ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, B->alloc_stream)
                               : cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    };
    const int M = B->n_mol;
    B->red_blocks = 1;
    std::vector<qc::MolParams> mp(M);
    std::vector<qc::MolWork> mw(M);
    std::vector<long long> key_off(M + 1, 0);
    size_t off = align256(static_cast<size_t>(M) * sizeof(unsigned long long));  // sample cursors
    struct Lay { size_t slots, filter, sets, ctr, part, sum, cpart, ctick; unsigned long long nb; int fw, chunks; };
    std::vector<Lay> lay(M);
    const size_t fixed0 = qc::smem_fixed_bytes();
    const int wcap = B->warps > 0 ? std::min(B->warps, qc::kBatchMaxWarps) : 16;  // 16: 128 registers
    // the join, per molecule as its handle would decide (so that a molecule's results are
    // the same in a batch as alone); the batch shares one index build over those molecules
    std::vector<char> jm(M, 0);
    bool join = false;
    for (int m = 0; m < M; ++m) {
        const qc_eloc* H = B->handles[m];
        jm[m] = H->opt_prefilter && H->na > 0 && H->nb > 0 &&
                (H->opt_join == 2 || (H->opt_join == 0 && qc::join_by_default(B->in[m].n_u, H->sp.pairs)));
        join = join || jm[m];
    }
    B->join = join;
    std::vector<int> act(M), lean(M), acap(M);
    std::vector<unsigned> stride(M);
    for (int m = 0; m < M; ++m) {
        const long long n = std::max<long long>(B->in[m].n_u, 1);
        Lay& L = lay[m];
        L.nb = next_pow2(2ULL * static_cast<unsigned long long>(n));
        // the single path's policy: the filter for ~16 bits per key, shrunk while that
        // leaves fewer than 8 warps, in the list layout that fits more warps
        int fw = 0, w = 0;
        lean[m] = 0;
        acap[m] = 0;
        // a joining molecule's alpha list may get fewer slots (enumerated in segments) when
        // that fits more warps; the full list on a tie
        const int nsa = B->handles[m]->sp.nsa;
        const int caps[3] = {0, 64, 32};
        for (int ci = 0; ci < (jm[m] ? 3 : 1); ++ci)
        for (int ln = 0; ln < 2; ++ln) {
            const int cap = caps[ci];
            if (cap > 0 && cap >= nsa) continue;
            const unsigned st =
                static_cast<unsigned>((qc::batch_warp_bytes(B->handles[m]->sp, ln, join, cap) + 15) / 16 * 16);
            int f = filter_log2(n), ww = 0;
            for (; f >= 5; --f) {
                const size_t base = fixed0 + (static_cast<size_t>(4) << f);
                if (base + st > B->dyn_limit) continue;
                ww = std::min(wcap, static_cast<int>((B->dyn_limit - base) / st));
                if (ww >= 8 || f <= 10 || ww >= wcap) break;
            }
            if (f < 5 || ww < 1) continue;
            if (ww > w || (ww == w && f > fw)) {
                fw = f;
                w = ww;
                lean[m] = ln;
                stride[m] = st;
                acap[m] = cap;
            }
        }
        if (w < 1) return bfail(B, QC_ERR_CAPACITY, "a molecule of the batch does not fit shared memory");
        L.fw = fw;
        act[m] = w;
        L.slots = off; off = align256(off + 2 * L.nb * 8);
        L.sets = off; off = align256(off + 2 * L.nb * 8);
        L.filter = off; off = align256(off + (static_cast<size_t>(4) << L.fw));
        L.ctr = off; off = align256(off + sizeof(qc::Counters));
        L.chunks = qc::exc_chunks(B->handles[m]->sp.pairs, B->chunk_pairs);
        L.cpart = L.ctick = 0;
        if (L.chunks > 1 && B->in[m].n_u > 0) {
            const size_t nu = static_cast<size_t>(B->in[m].n_u);
            L.cpart = off; off = align256(off + nu * L.chunks * sizeof(qc::ChunkRec));
            L.ctick = off; off = align256(off + nu * sizeof(unsigned));  // zeroed with the arena
        }
        L.part = off; off = align256(off + static_cast<size_t>(qc::reduce_blocks(B->in[m].n_u)) * 4 * sizeof(double));
        L.sum = 0;
        key_off[m + 1] = key_off[m] + B->in[m].n_u;
    }
    // join: molecule m's slot keys start at slot_base[m] (two sets of nb slots each)
    // (molecules without the join take no slots and no items)
    unsigned long long total_slots = 0;
    long long total_items = 0;
    std::vector<long long> item_off(M + 1, 0);
    for (int m = 0; m < M; ++m) {
        total_slots += jm[m] ? 2 * lay[m].nb : 0;
        item_off[m + 1] = item_off[m] + (jm[m] ? 2 * B->in[m].n_u : 0);
    }
    total_items = item_off[M];
    if (join && (total_items >= 0xffffffffLL || total_slots >= 0xffffffffULL)) {
        join = B->join = false;  // sort keys, values and entry positions are 32-bit
        std::fill(jm.begin(), jm.end(), 0);
    }
    std::vector<unsigned> slot_base(M + 1, 0u), row_base(M + 1, 0u);
    if (join)
        for (int m = 0; m < M; ++m) {
            slot_base[m + 1] = slot_base[m] + static_cast<unsigned>(jm[m] ? 2 * lay[m].nb : 0);
            row_base[m + 1] = row_base[m] + static_cast<unsigned>(jm[m] ? B->in[m].n_u : 0);
        }
    if (join) {
        B->ja_len = off;
        off = align256(off + static_cast<size_t>(slot_base[M]) * 4);
    }
    if (off > B->arena_cap) {
        // grow with headroom: a reallocation (cudaFree) waits for the whole device, unless
        // the batch allocates stream-ordered
        if (B->d_arena) {
            if (B->alloc_stream) cudaFreeAsync(B->d_arena, B->alloc_stream);
            else cudaFree(B->d_arena);
        }
        B->d_arena = nullptr;
        B->arena_cap = 0;
        const size_t cap = align256(off + off / 2);
        cudaError_t e = B->alloc_stream ? cudaMallocAsync(reinterpret_cast<void**>(&B->d_arena), cap, B->alloc_stream)
                                        : qc::dev_alloc(&B->d_arena, cap);
        if (e != cudaSuccess) return bcuda(B, e, "cudaMalloc batch arena");
        B->arena_cap = cap;
    }
    B->arena_bytes = off;
    unsigned char* A = B->d_arena;
    if (join) {
        const long long mi = total_items;
        const unsigned long long ns = slot_base[M];
        size_t jo = align256(static_cast<size_t>(std::max<long long>(mi, 1)) * 4);  // keys
        B->jo_val = jo; jo = align256(jo + static_cast<size_t>(std::max<long long>(mi, 1)) * 4);
        B->jo_start = jo; jo = align256(jo + static_cast<size_t>(ns) * 4);
        B->jo_ent = jo; jo = align256(jo + static_cast<size_t>(std::max<long long>(mi, 1)) * 16);
        B->jo_base = jo; jo = align256(jo + static_cast<size_t>(M + 1) * 4);
        B->jo_rbase = jo; jo = align256(jo + static_cast<size_t>(M + 1) * 4);
        const size_t rows = static_cast<size_t>(std::max<long long>(mi / 2, 1));
        B->jo_order = jo; jo = align256(jo + rows * 4);
        B->jo_pab = jo; jo = align256(jo + 2 * align256(rows * 4));
        B->jo_ws = jo; jo = align256(jo + qc::join_batch_workspace_bytes(mi, ns));
        if (jo > B->join_cap) {
            if (B->d_join) {
                if (B->alloc_stream) cudaFreeAsync(B->d_join, B->alloc_stream);
                else cudaFree(B->d_join);
            }
            B->d_join = nullptr;
            B->join_cap = 0;
            const size_t cap = align256(jo + jo / 2);
            cudaError_t e = B->alloc_stream ? cudaMallocAsync(reinterpret_cast<void**>(&B->d_join), cap, B->alloc_stream)
                                            : qc::dev_alloc(&B->d_join, cap);
            if (e != cudaSuccess) return bcuda(B, e, "cudaMalloc batch join index");
            B->join_cap = cap;
        }
        B->j_items = mi;
        B->j_slots = ns;
        cudaError_t e = h2d(B->d_join + B->jo_base, slot_base.data(), (M + 1) * sizeof(unsigned));
        if (e == cudaSuccess) e = h2d(B->d_join + B->jo_rbase, row_base.data(), (M + 1) * sizeof(unsigned));
        if (e != cudaSuccess) return bcuda(B, e, "copy join slot and row bases");
    }
    for (int m = 0; m < M; ++m) {
        const Lay& L = lay[m];
        const BatchInput& I = B->in[m];
        qc_eloc* H = B->handles[m];
        qc::MolWork& W = mw[m];
        W.slots = reinterpret_cast<unsigned long long*>(A + L.slots);
        W.aset = reinterpret_cast<unsigned long long*>(A + L.sets);
        W.bset = W.aset + L.nb;
        W.filter = reinterpret_cast<uint32_t*>(A + L.filter);
        W.ctr = I.ctr ? I.ctr : reinterpret_cast<qc::Counters*>(A + L.ctr);
        W.part = reinterpret_cast<double*>(A + L.part);
        W.sum = B->d_sums + m;
        const long long red_rows = I.piece ? (I.r1 < 0 ? I.n_u : I.r1) - I.r0 : I.n_u;
        W.nblk = I.reduce ? qc::reduce_blocks(red_rows) : 0;
        W.jkey = W.jval = W.jlen = nullptr;
        W.jbase = W.jsent = 0u;
        if (jm[m]) {
            W.jkey = reinterpret_cast<unsigned*>(B->d_join) + item_off[m];
            W.jval = reinterpret_cast<unsigned*>(B->d_join + B->jo_val) + item_off[m];
            W.jlen = reinterpret_cast<unsigned*>(A + B->ja_len);
            W.jbase = slot_base[m];
            W.jsent = slot_base[M];
        }
        B->red_blocks = std::max(B->red_blocks, W.nblk);
        qc::MolParams& P = mp[m];
        P.sp = H->sp;
        P.sp.err = &W.ctr->flags;
        P.tp = qc::TableParams{};
        P.tp.keys = reinterpret_cast<const ulonglong2*>(I.samples);
        P.tp.psi = reinterpret_cast<const double2*>(I.psi);
        P.tp.n = I.n_u;
        P.tp.err = &W.ctr->flags;
        P.tp.slots = W.slots;
        P.tp.nb_mask = static_cast<unsigned>(L.nb - 1);
        P.tp.filter = W.filter;
        P.tp.fw = L.fw;
        P.tp.aset = W.aset;
        P.tp.bset = W.bset;
        P.tp.set_mask = static_cast<unsigned>(L.nb - 1);
        if (jm[m]) {
            P.tp.jstart = reinterpret_cast<const unsigned*>(B->d_join + B->jo_start) + slot_base[m];
            P.tp.jlen = reinterpret_cast<const unsigned*>(A + B->ja_len) + slot_base[m];
            P.tp.gent = reinterpret_cast<const ulonglong2*>(B->d_join + B->jo_ent);
            P.tp.scan_cost = H->opt_scan_cost ? H->opt_scan_cost : qc::kDefaultScanCost;
            P.tp.beta_cost = qc::beta_cost_of(H->opt_beta_cost);
            P.tp.alpha_cap = acap[m];
        }
        P.ep = qc::EvalParams{};
        P.ep.samples = reinterpret_cast<const ulonglong2*>(I.samples);
        P.ep.psi = reinterpret_cast<const double2*>(I.psi);
        P.ep.counts = reinterpret_cast<const long long*>(I.counts);
        P.ep.n_u = I.n_u;
        P.ep.eloc = reinterpret_cast<double2*>(I.eloc);
        P.ep.ctr = W.ctr;
        P.ep.T = H->d_T;
        P.ep.mode = QC_SAMPLE;
        P.ep.lean = lean[m];
        P.ep.chunks = L.chunks;
        P.ep.cpart = L.cpart ? static_cast<void*>(A + L.cpart) : nullptr;
        P.ep.cticket = L.ctick ? reinterpret_cast<unsigned*>(A + L.ctick) : nullptr;
        // a joining molecule's rows are handed out heavy first (the order the batch's join
        // index builds each step)
        P.ep.order = jm[m] && !I.piece ? reinterpret_cast<const unsigned*>(B->d_join + B->jo_order) + row_base[m]
                                         : nullptr;
        if (P.ep.chunks > 1 && !P.ep.cpart) P.ep.chunks = 1;
        P.active_warps = act[m];
        P.warp_stride = stride[m];
        P.r0 = I.r0;
        P.r1 = I.r1 < 0 ? I.n_u : I.r1;
        P.red_lo = I.piece ? P.r0 : 0;
        P.red_hi = I.piece ? P.r1 : I.n_u;
    }
    // launch shape: the widest CTA any molecule uses, all the dynamic shared memory
    int warps = 1;
    for (int m = 0; m < M; ++m) warps = std::max(warps, act[m]);
    B->smem = B->dyn_limit;
    const int per_sm = qc::max_active_batch(B->precision, B->unroll, 32 * warps, B->smem, join);
    if (per_sm < 1) return bfail(B, QC_ERR_CAPACITY, "batch kernel cannot be resident with this shape");
    B->grid = per_sm * B->sm_count;
    // run order: estimated time n_u * pairs / active warps, longest first
    std::vector<int> order;
    std::vector<double> cost(M, 0.0);
    for (int m = 0; m < M; ++m) {
        const long long rows = mp[m].r1 - mp[m].r0;
        if (rows <= 0) continue;
        order.push_back(m);
        cost[m] = static_cast<double>(rows) * static_cast<double>(mp[m].sp.pairs) / act[m];
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    B->n_run = static_cast<int>(order.size());
    B->n_keys = key_off[M];
    cudaError_t e;
    if (!order.empty()) {
        e = h2d(B->d_order, order.data(), order.size() * sizeof(int));
        if (e != cudaSuccess) return bcuda(B, e, "copy run order");
    }
    e = h2d(B->d_mols, mp.data(), M * sizeof(qc::MolParams));
    if (e != cudaSuccess) return bcuda(B, e, "copy molecule parameters");
    e = h2d(B->d_work, mw.data(), M * sizeof(qc::MolWork));
    if (e != cudaSuccess) return bcuda(B, e, "copy molecule workspaces");
    e = h2d(B->d_key_off, key_off.data(), (M + 1) * sizeof(long long));
    if (e != cudaSuccess) return bcuda(B, e, "copy key offsets");
    B->dirty = false;
    B->warps_used = warps;
    return QC_OK;
}

}  // namespace

namespace {

// One batched step on stream s (eager or under capture).
qc_status enqueue(qc_batch* B, qc_eloc_summary* sums_host, cudaStream_t s, bool timed) {
    cudaError_t e;
#define QB(call, what)                                   \
    do {                                                 \
        e = (call);                                      \
        if (e != cudaSuccess) return bcuda(B, e, what);  \
    } while (0)
    if (timed) QB(cudaEventRecord(B->ev[0], s), "cudaEventRecord");
    QB(cudaMemsetAsync(B->d_arena, 0, B->arena_bytes, s), "memset arena");
    QB(qc::launch_build_batch(B->d_mols, B->d_work, B->d_key_off, B->n_mol, B->n_keys, s), "batch build");
    if (B->join) {
        const size_t rows = static_cast<size_t>(std::max<long long>(B->j_items / 2, 1));
        unsigned* pa = reinterpret_cast<unsigned*>(B->d_join + B->jo_pab);
        unsigned* pb = reinterpret_cast<unsigned*>(B->d_join + B->jo_pab + align256(rows * 4));
        QB(cudaMemsetAsync(pa, 0, 2 * align256(rows * 4), s), "memset join order sizes");
        QB(qc::launch_join_batch(B->d_mols, reinterpret_cast<const unsigned*>(B->d_join + B->jo_base), B->n_mol,
                                 B->j_items, B->j_slots, B->d_join + B->jo_ws, reinterpret_cast<unsigned*>(B->d_join),
                                 reinterpret_cast<unsigned*>(B->d_join + B->jo_val),
                                 reinterpret_cast<unsigned*>(B->d_arena + B->ja_len),
                                 reinterpret_cast<unsigned*>(B->d_join + B->jo_start),
                                 reinterpret_cast<ulonglong2*>(B->d_join + B->jo_ent), s,
                                 reinterpret_cast<const unsigned*>(B->d_join + B->jo_rbase),
                                 reinterpret_cast<unsigned*>(B->d_join + B->jo_order), pa, pb),
           "batch join index");
    }
    if (timed) QB(cudaEventRecord(B->ev[1], s), "cudaEventRecord");
    if (B->n_run > 0) {
        qc::BatchParams bp{};
        bp.mols = B->d_mols;
        bp.order = B->d_order;
        bp.next = reinterpret_cast<unsigned long long*>(B->d_arena);  // cursors lead the arena
        bp.n_mol = B->n_run;
        bp.chunk = B->chunk;
        QB(qc::launch_eloc_batch(bp, B->precision, B->unroll, B->grid, B->warps_used, B->smem, s, B->join),
           "batch kernel");
    }
    if (timed) QB(cudaEventRecord(B->ev[2], s), "cudaEventRecord");
    QB(qc::launch_reduce_batch(B->d_mols, B->d_work, B->n_mol, B->red_blocks, s), "batch reduce");
    if (timed) QB(cudaEventRecord(B->ev[3], s), "cudaEventRecord");
    if (sums_host)
        QB(cudaMemcpyAsync(sums_host, B->d_sums, B->n_mol * sizeof(qc_eloc_summary), cudaMemcpyDeviceToHost, s),
           "summary copy");
#undef QB
    return QC_OK;
}

void drop_graph(qc_batch* B) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    B->exec = nullptr;
    B->graph = nullptr;
    B->graph_sums = nullptr;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {
// (Re)size the per-molecule device arrays for n_mol molecules.
cudaError_t batch_alloc(qc_batch* B, int n_mol) {
    if (n_mol <= B->mol_cap) return cudaSuccess;
    n_mol = std::max(n_mol, 64);  // room for a typical batch without reallocating
    for (void* p : {static_cast<void*>(B->d_mols), static_cast<void*>(B->d_work), static_cast<void*>(B->d_key_off),
                    static_cast<void*>(B->d_sums), static_cast<void*>(B->d_order)})
        if (p) cudaFree(p);
    B->d_order = nullptr;
    B->d_mols = nullptr;
    B->d_work = nullptr;
    B->d_key_off = nullptr;
    B->d_sums = nullptr;
    B->mol_cap = 0;
    cudaError_t e = qc::dev_alloc(&B->d_mols, n_mol * sizeof(qc::MolParams));
    if (e == cudaSuccess) e = qc::dev_alloc(&B->d_work, n_mol * sizeof(qc::MolWork));
    if (e == cudaSuccess) e = qc::dev_alloc(&B->d_key_off, (n_mol + 1) * sizeof(long long));
    if (e == cudaSuccess) e = qc::dev_alloc(&B->d_sums, n_mol * sizeof(qc_eloc_summary));
    if (e == cudaSuccess) e = qc::dev_alloc(&B->d_order, n_mol * sizeof(int));
    if (e == cudaSuccess) B->mol_cap = n_mol;
    return e;
}
}  // namespace

// Point an existing batch at another set of handles (same precision and device), keeping
// its device allocations when they are large enough; inputs must be set again.
qc_status qc::batch_retarget(qc_batch* B, qc_eloc* const* handles, int n_mol) {
    if (!B || !handles || n_mol <= 0 || n_mol > 65535) return QC_ERR_ARG;
    for (int m = 0; m < n_mol; ++m)
        if (!handles[m] || handles[m]->mode != QC_SAMPLE || handles[m]->precision != B->precision ||
            handles[m]->device != B->device)
            return QC_ERR_ARG;
    cudaError_t e = batch_alloc(B, n_mol);
    if (e != cudaSuccess) return bcuda(B, e, "cudaMalloc batch arrays");
    B->n_mol = n_mol;
    B->handles.assign(handles, handles + n_mol);
    B->in.assign(n_mol, BatchInput{});
    B->dirty = true;
    drop_graph(B);
    return QC_OK;
}

// Evaluate only rows [r0, r1) of molecule `mol` (set after its inputs), accumulate its
// counters in `ctr` (device memory that the caller zeroes before the first slice), and run
// its Eq. 1 reduction over all rows only when `reduce` is set.
qc_status qc::batch_set_slice(qc_batch* B, int mol, long long r0, long long r1, bool reduce, qc::Counters* ctr) {
    if (!B || mol < 0 || mol >= B->n_mol) return QC_ERR_ARG;
    BatchInput& I = B->in[mol];
    if (r0 < 0 || r1 < r0 || r1 > I.n_u) return bfail(B, QC_ERR_ARG, "bad row slice");
    I.r0 = r0;
    I.r1 = r1;
    I.reduce = reduce;
    I.ctr = ctr;
    I.piece = false;
    B->dirty = true;
    drop_graph(B);
    return QC_OK;
}

// The serving form's lanes: grow the batch's device buffers stream-ordered on `s` (the lane
// stream its waves run on) and copy the parameter blocks there.
qc_status qc::batch_set_alloc_stream(qc_batch* B, cudaStream_t s) {
    if (!B) return QC_ERR_ARG;
    B->alloc_stream = s;
    return QC_OK;
}

extern "C" {

qc_status qc_batch_create(qc_eloc* const* handles, int n_mol, qc_batch** out) {
    if (!out) return QC_ERR_ARG;
    *out = nullptr;
    if (!handles || n_mol <= 0 || n_mol > 65535) return QC_ERR_ARG;
    qc_batch* B = new (std::nothrow) qc_batch();
    if (!B) return QC_ERR_OOM;
    B->n_mol = n_mol;
    B->handles.assign(handles, handles + n_mol);
    B->in.resize(n_mol);
    for (int m = 0; m < n_mol; ++m) {
        qc_eloc* H = handles[m];
        if (!H || H->mode != QC_SAMPLE || H->precision != handles[0]->precision || H->device != handles[0]->device) {
            delete B;
            return QC_ERR_ARG;
        }
    }
    B->device = handles[0]->device;
    B->precision = handles[0]->precision;
    B->sm_count = handles[0]->sm_count;
    cudaError_t e = qc::prepare_batch_kernels(handles[0]->smem_optin, &B->dyn_limit);
    if (e == cudaSuccess) e = batch_alloc(B, n_mol);
    for (auto& ev : B->ev)
        if (e == cudaSuccess) e = cudaEventCreate(&ev);
    if (e != cudaSuccess) {
        qc_batch_destroy(B);
        return e == cudaErrorMemoryAllocation ? QC_ERR_OOM : QC_ERR_CUDA;
    }
    *out = B;
    return QC_OK;
}

qc_status qc_batch_destroy(qc_batch* B) {
    if (!B) return QC_OK;
    drop_graph(B);
    for (void* p : {static_cast<void*>(B->d_mols), static_cast<void*>(B->d_work), static_cast<void*>(B->d_key_off),
                    static_cast<void*>(B->d_order), static_cast<void*>(B->d_arena),
                    static_cast<void*>(B->d_sums), static_cast<void*>(B->d_join)})
        if (p) cudaFree(p);
    for (auto& ev : B->ev)
        if (ev) cudaEventDestroy(ev);
    delete B;
    return QC_OK;
}

const char* qc_batch_last_error(const qc_batch* B) { return B ? B->err.c_str() : ""; }

qc_status qc_batch_set_inputs(qc_batch* B, int mol, const uint64_t* samples, const int64_t* counts,
                              const double* psi, int64_t n_u, double* eloc) {
    if (!B) return QC_ERR_ARG;
    if (mol < 0 || mol >= B->n_mol) return bfail(B, QC_ERR_ARG, "molecule index out of range");
    if (n_u < 0 || n_u >= (1LL << 31)) return bfail(B, QC_ERR_ARG, "bad n_u");
    if (n_u > 0 && (!samples || !counts || !psi || !eloc)) return bfail(B, QC_ERR_ARG, "NULL pointer");
    auto mis = [](const void* p, unsigned a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) != 0; };
    if (n_u > 0 && (mis(samples, 16) || mis(psi, 16) || mis(eloc, 16) || mis(counts, 8)))
        return bfail(B, QC_ERR_ARG, "device arrays must be 16-byte aligned (counts: 8)");
    BatchInput& I = B->in[mol];
    I = BatchInput{};
    I.samples = samples;
    I.counts = counts;
    I.psi = psi;
    I.n_u = n_u;
    I.eloc = eloc;
    B->dirty = true;
    drop_graph(B);
    return QC_OK;
}

qc_status qc_batch_set_rows(qc_batch* B, int mol, int64_t r0, int64_t r1) {
    if (!B) return QC_ERR_ARG;
    if (mol < 0 || mol >= B->n_mol) return bfail(B, QC_ERR_ARG, "mol out of range");
    BatchInput& I = B->in[mol];
    if (r1 < 0) r1 = I.n_u;
    if (r0 < 0 || r1 < r0 || r1 > I.n_u) return bfail(B, QC_ERR_ARG, "rows must satisfy 0 <= r0 <= r1 <= n_u");
    I.r0 = r0;
    I.r1 = r1;
    I.reduce = true;
    I.ctr = nullptr;
    I.piece = !(r0 == 0 && r1 == I.n_u);
    B->dirty = true;
    drop_graph(B);
    return QC_OK;
}

qc_status qc_batch_set_config(qc_batch* B, int unroll, int warps, int chunk) {
    if (!B) return QC_ERR_ARG;
    if (unroll != 0 && unroll != 2 && unroll != 4) return bfail(B, QC_ERR_ARG, "unroll: 0, 2 or 4");
    if (warps < 0 || warps > qc::kBatchMaxWarps) return bfail(B, QC_ERR_ARG, "warps: 0..20");
    if (chunk < 0 || chunk > 1024) return bfail(B, QC_ERR_ARG, "chunk: 0..1024");
    B->unroll = unroll ? unroll : 4;
    B->warps = warps;
    B->chunk = chunk ? chunk : 1;
    B->dirty = true;
    drop_graph(B);
    return QC_OK;
}

qc_status qc_batch_set_chunk_pairs(qc_batch* B, int64_t chunk_pairs) {
    if (!B) return QC_ERR_ARG;
    if (chunk_pairs < -1) return bfail(B, QC_ERR_ARG, "chunk_pairs: -1, 0 or pairs per chunk");
    B->chunk_pairs = chunk_pairs == 0 ? qc::kDefaultChunkPairs : (chunk_pairs < 0 ? 0 : chunk_pairs);
    B->dirty = true;
    drop_graph(B);
    return QC_OK;
}

qc_status qc_batch_eval(qc_batch* B, qc_eloc_summary* sums, void* stream) {
    if (!B) return QC_ERR_ARG;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != B->device) return bfail(B, QC_ERR_ARG, "batch belongs to another device");
    if (B->dirty) {
        qc_status st = prepare(B);
        if (st != QC_OK) return st;
    }
    qc_status st = enqueue(B, sums, static_cast<cudaStream_t>(stream), true);
    B->timed = (st == QC_OK);
    return st;
}

qc_status qc_batch_graph_launch(qc_batch* B, qc_eloc_summary* sums, void* stream) {
    if (!B) return QC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!s) return bfail(B, QC_ERR_ARG, "graph capture needs a non-default stream");
    if (B->dirty) {
        drop_graph(B);
        qc_status st = prepare(B);
        if (st != QC_OK) return st;
    }
    if (!B->exec || B->graph_sums != sums) {
        drop_graph(B);
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return bcuda(B, e, "cudaStreamBeginCapture");
        qc_status st = enqueue(B, sums, s, false);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(s, &g);
        if (st != QC_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return bcuda(B, e, "cudaStreamEndCapture");
        B->graph = g;
        e = cudaGraphInstantiate(&B->exec, g, 0);
        if (e != cudaSuccess) {
            drop_graph(B);
            return bcuda(B, e, "cudaGraphInstantiate");
        }
        B->graph_sums = sums;
    }
    cudaError_t e = cudaGraphLaunch(B->exec, s);
    if (e != cudaSuccess) return bcuda(B, e, "cudaGraphLaunch");
    B->timed = false;
    return QC_OK;
}

qc_status qc_batch_timings(qc_batch* B, float* ms3) {
    if (!B || !ms3) return QC_ERR_ARG;
    if (!B->timed) return bfail(B, QC_ERR_ARG, "no eager evaluation to time");
    cudaError_t e = cudaEventSynchronize(B->ev[3]);
    if (e != cudaSuccess) return bcuda(B, e, "cudaEventSynchronize");
    for (int i = 0; i < 3; ++i) {
        e = cudaEventElapsedTime(&ms3[i], B->ev[i], B->ev[i + 1]);
        if (e != cudaSuccess) return bcuda(B, e, "cudaEventElapsedTime");
    }
    return QC_OK;
}

qc_status qc_batch_config(const qc_batch* B, int64_t* cfg6) {
    if (!B || !cfg6) return QC_ERR_ARG;
    cfg6[0] = B->unroll;
    cfg6[1] = B->warps_used;
    cfg6[2] = B->chunk;
    cfg6[3] = B->grid;
    cfg6[4] = B->n_run;
    cfg6[5] = static_cast<int64_t>(B->smem);
    return QC_OK;
}

// Time every candidate shape on this batch (eager evaluations on `stream`, main kernel
// only, best of `iters`) and keep the fastest, then the excitation-chunk size at that
// shape.  best4 (optional): {unroll, warps, samples per fetch, pairs per chunk (-1: none)}.
qc_status qc_batch_autotune(qc_batch* B, void* stream, int iters, int64_t* best4) {
    if (!B) return QC_ERR_ARG;
    if (iters < 1) iters = 1;
    // best of `iters` timed steps (after one untimed) of the current shape; capacity -> skip
    auto time_shape = [&](float& t_best) -> qc_status {
        qc_status st = prepare(B);
        if (st != QC_OK) return st;
        t_best = 3.0e38f;
        for (int it = 0; it < iters + 1; ++it) {
            st = enqueue(B, nullptr, static_cast<cudaStream_t>(stream), true);
            if (st != QC_OK) return st;
            float ms3[3];
            B->timed = true;
            st = qc_batch_timings(B, ms3);
            if (st != QC_OK) return st;
            if (it > 0) t_best = std::min(t_best, ms3[1]);
        }
        return QC_OK;
    };
    const int warps_c[] = {8, 12, 16, 20};
    const int units_c[] = {1, 4};  // samples per fetch
    const int unroll_c[] = {2, 4};
    float best = 3.0e38f;
    int bu = 4, bw = 0, bp = 1;
    const long long keep_cp = B->chunk_pairs;
    for (int ur : unroll_c)
        for (int w : warps_c)
            for (int up : units_c) {
                qc_status st = qc_batch_set_config(B, ur, w, up);
                if (st != QC_OK) return st;
                B->chunk_pairs = keep_cp;
                float t = 0.f;
                st = time_shape(t);
                if (st == QC_ERR_CAPACITY) continue;
                if (st != QC_OK) return st;
                if (B->warps_used < w) continue;  // cap above what any molecule fits: tried already
                if (t < best) {
                    best = t;
                    bu = ur;
                    bw = w;
                    bp = up;
                }
            }
    // then the excitation-chunk size at that shape (0: one warp per sample)
    long long bc = keep_cp;
    const long long cp_c[] = {qc::kChunkPairsProbe / 2, qc::kChunkPairsProbe, qc::kChunkPairsProbe * 2, 0};
    qc_status st = qc_batch_set_config(B, bu, bw, bp);
    if (st != QC_OK) return st;
    for (long long cp : cp_c) {
        if (cp == keep_cp) continue;
        B->chunk_pairs = cp;
        B->dirty = true;
        float t = 0.f;
        st = time_shape(t);
        if (st == QC_ERR_CAPACITY) continue;
        if (st != QC_OK) return st;
        if (t < best) {
            best = t;
            bc = cp;
        }
    }
    B->chunk_pairs = bc;
    B->dirty = true;
    st = prepare(B);
    if (st != QC_OK) return st;
    if (best4) {
        best4[0] = bu;
        best4[1] = bw;
        best4[2] = bp;
        best4[3] = bc > 0 ? bc : -1;
    }
    return QC_OK;
}

}  // extern "C"
