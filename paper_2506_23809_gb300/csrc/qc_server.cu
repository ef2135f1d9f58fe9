// qc_server.cu -- the serving form: local-energy requests for different molecules and
// sample-set sizes arrive at any time (qc_eloc_submit) and are answered asynchronously
// (qc_eloc_poll).  A scheduler thread runs continuous batching:
//   * admission -- a request is admitted when its device footprint fits the memory budget
//     and a slot is free; a request that can never fit is refused (QC_ERR_BUDGET);
//   * residency -- a molecule's Hamiltonian (a qc_eloc handle) stays on the device for
//     later requests with the same molecule key, evicted least-recently-used when the
//     budget needs the room;
//   * waves -- admitted requests whose inputs are on the device join the next wave, one
//     qc_batch launch on one of several streams; a wave holds about `quantum` enumerated
//     pairs: the oldest request first (a guaranteed share of the quantum), then the others with
//     the least remaining work first, none with more than kWaveSpread times the oldest's
//     remaining work (it would hold the wave's short requests until it ends; it waits for a
//     wave of its own), and the wave's rows stay within `wave_rows` (a batch returns its
//     requests when all of them are done, so a long request batched with another would wait
//     for it: past that size a request runs alone, as the plain launch would, and batching
//     is kept for the short requests whose launch costs it saves).  A request too long for the room left runs a slice of
//     its rows against its whole sample table and comes back for the next wave, so a long
//     request never holds the GPU for more than a wave while short ones wait; after a wave
//     that ran a slice, the short requests that are ready (at most half a quantum each) get
//     a wave of their own before the next slice;
//   * completion -- found by polling CUDA events (no blocking device waits); results are
//     copied to the caller's host buffers and the request's memory is released.
// Admission (creating a Hamiltonian and uploading a request's inputs, the slow host-side
// part) runs on a thread of its own, so waves keep being launched and retired meanwhile;
// each lane's batch grows its device buffers stream-ordered on the lane's stream, so a
// wave's set-up never waits for another lane's wave.
// Because a batch runs the single-molecule per-sample code, and a sliced request's Eq. 1
// reduction runs once over all of its rows in its last wave, a request's E_loc and energy
// are bitwise the same alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "qc_eloc.h"
#include "qc_handle.h"
#include "qc_internal.h"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Resident {  // a molecule's Hamiltonian kept on the device
    qc_eloc* handle = nullptr;  // null while the scheduler creates it (outside the lock)
    qc_status failed = QC_OK;   // creation failed: requests pinned to it fail the same way
    size_t bytes = 0;
    int users = 0;        // requests in flight using it
    double last_use = 0.0;
    bool evaluating = false;  // a wave runs on the handle's own workspace (single-molecule path)
};

struct Request {
    uint64_t ticket = 0;
    qc_eloc_job job{};
    std::vector<double> h, eri;  // private copies when the molecule is not resident yet
    size_t bytes = 0;            // device footprint of the request (inputs, outputs, workspace)
    Resident* res = nullptr;
    uint64_t* d_keys = nullptr;
    int64_t* d_counts = nullptr;
    double* d_psi = nullptr;
    double* d_eloc = nullptr;
    qc::Counters* d_ctr = nullptr;  // accumulates over the request's slices
    long long next_row = 0;         // rows [0, next_row) are evaluated
    long long slice_end = 0;        // end of the slice in flight
    long long pairs_per_row = 1;
    qc_eloc_result result{};
    bool done = false;
};

struct Wave {
    std::vector<Request*> reqs;
    int stream = 0;  // index into the wave streams; its batch, summaries and event
    bool single = false;  // one whole request through the single-molecule path
};

struct Lane {  // one wave stream with the objects reused by its waves
    cudaStream_t stream = nullptr;
    qc_batch* batch[2] = {nullptr, nullptr};  // per precision, created on first use
    qc_eloc_summary* sums = nullptr;          // page-locked, max_slots entries
    cudaEvent_t ev = nullptr;
    bool busy = false;
};

size_t request_bytes(int64_t n_u) {
    const size_t n = static_cast<size_t>(std::max<int64_t>(n_u, 1));
    size_t nb = 1;
    while (nb < 2 * n) nb <<= 1;
    // keys + counts + psi + eloc, table + spin sets, filter, partials
    return n * (16 + 8 + 16 + 16) + 4 * nb * 8 + (1u << 17) + (1u << 15);
}

size_t hamiltonian_bytes(int n_orb, int precision) {
    const size_t K = static_cast<size_t>(n_orb / 2);
    const size_t w = precision == QC_FP64 ? 8 : 4;
    return K * K * K * K * w + 2 * K * K * K * w + 4 * K * K * 8 + 4096;
}

}  // namespace

struct qc_server {
    int device = 0;
    size_t budget = 0, used = 0;
    int max_slots = 0;
    cudaStream_t upload = nullptr;
    std::vector<Lane> lanes;
    std::mutex mu;
    std::condition_variable cv_submit;   // wakes the scheduler
    std::condition_variable cv_admit;    // wakes the admission thread (a submit, or memory freed)
    std::condition_variable cv_done;     // wakes pollers
    std::deque<Request*> pending;        // submitted, not admitted
    std::vector<Request*> ready;         // admitted, inputs on the device, not launched
    std::list<Wave> waves;               // launched, not finished
    std::map<uint64_t, Request*> all;    // every live request by ticket
    std::map<uint64_t, std::unique_ptr<Resident>> residents;  // by molecule key
    uint64_t next_ticket = 1;
    int active = 0;                      // admitted and not finished
    long long quantum = 1000000000000LL;  // enumerated pairs per wave (0: no slicing)
    int oldest_pct = 50;                 // share of a wave guaranteed to the oldest request
    long long wave_rows = 1LL << 16;     // sample rows a wave of several requests may hold (0: any)
    bool last_wave_sliced = false;       // the last wave ran a slice of a long request
    bool stop = false;
    std::thread worker;
    std::thread admitter;
    cudaError_t fatal = cudaSuccess;
};

namespace {

// Release a request's device memory (stream-ordered, after the work on `s`) and its budget.
void finish_request(qc_server* S, Request* r, cudaStream_t s) {
    if (r->d_keys) cudaFreeAsync(r->d_keys, s);
    if (r->d_counts) cudaFreeAsync(r->d_counts, s);
    if (r->d_psi) cudaFreeAsync(r->d_psi, s);
    if (r->d_eloc) cudaFreeAsync(r->d_eloc, s);
    if (r->d_ctr) cudaFreeAsync(r->d_ctr, s);
    r->d_ctr = nullptr;
    r->d_keys = nullptr;
    r->d_counts = nullptr;
    r->d_psi = nullptr;
    r->d_eloc = nullptr;
    if (r->res) {
        r->res->users--;
        r->res->last_use = now_s();
    }
    S->used -= r->bytes;
    S->active--;
    r->done = true;
    S->cv_admit.notify_all();  // memory and a slot came free
}

// Evict unused resident Hamiltonians, least recently used first, until `need` fits.
bool make_room(qc_server* S, size_t need) {
    while (S->used + need > S->budget) {
        Resident* victim = nullptr;
        uint64_t vkey = 0;
        for (auto& kv : S->residents)
            if (kv.second->users == 0 && (!victim || kv.second->last_use < victim->last_use)) {
                victim = kv.second.get();
                vkey = kv.first;
            }
        if (!victim) return false;
        S->used -= victim->bytes;
        qc_eloc_destroy(victim->handle);
        S->residents.erase(vkey);
    }
    return true;
}

// Admit pending requests in arrival order while memory and slots allow.  Called by the
// admission thread with the lock held; the lock is released while a new Hamiltonian is
// created and while a request's inputs are copied to the device, so submit, poll and the
// scheduler do not wait for those copies.  Only the admission thread admits, so a molecule
// created here is complete before a later request for it is admitted.
void admit(qc_server* S, std::unique_lock<std::mutex>& lk) {
    while (!S->pending.empty() && S->active < S->max_slots) {
        Request* r = S->pending.front();
        const qc_eloc_job& j = r->job;
        const uint64_t key = j.mol_key;
        Resident* res = r->res;  // pinned at submit when the molecule was resident
        if (!res && key) {
            auto it = S->residents.find(key);
            if (it != S->residents.end()) {
                res = it->second.get();
                res->users++;
                r->res = res;
            }
        }
        if (res && !res->handle && res->failed != QC_OK) {  // its Hamiltonian could not be created
            S->pending.pop_front();
            r->result.status = res->failed;
            res->users--;
            r->res = nullptr;
            r->done = true;
            S->cv_done.notify_all();
            continue;
        }
        const size_t ham = res ? 0 : hamiltonian_bytes(j.n_orb, j.precision);
        if (!make_room(S, r->bytes + ham)) break;  // wait for memory to free up
        S->pending.pop_front();
        r->result.t_admit = now_s();
        const bool create = (res == nullptr);
        if (create) {
            auto fresh = std::make_unique<Resident>();
            fresh->bytes = ham;
            fresh->users = 1;
            S->used += ham;
            res = fresh.get();
            r->res = res;
            // a request without a key gets a private key so its Hamiltonian can be evicted later
            const uint64_t k = key ? key : (0x8000000000000000ULL | r->ticket);
            S->residents[k] = std::move(fresh);
        }
        S->used += r->bytes;
        S->active++;
        lk.unlock();
        // ---- outside the lock: the Hamiltonian and the inputs go to the device ----
        qc_status st = QC_OK;
        qc_eloc* made = nullptr;
        if (create) {
            const bool own = !r->h.empty();  // copied at submit, else borrowed from the caller
            st = qc_eloc_create(own ? r->h.data() : j.h, own ? r->eri.data() : j.eri, j.e_core, j.n_orb, j.n_elec,
                                j.precision, QC_SAMPLE, &made);
        }
        r->h.clear();
        r->h.shrink_to_fit();
        r->eri.clear();
        r->eri.shrink_to_fit();
        const size_t n = static_cast<size_t>(j.n_u);
        cudaStream_t up = S->upload;
        cudaError_t e = cudaSuccess;
        if (st == QC_OK) {
            e = cudaMallocAsync(reinterpret_cast<void**>(&r->d_ctr), sizeof(qc::Counters), up);
            if (e == cudaSuccess) e = cudaMemsetAsync(r->d_ctr, 0, sizeof(qc::Counters), up);
            if (n > 0) {
                // stream-ordered allocations: no device-wide synchronisation while waves run
                if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&r->d_keys), n * 16, up);
                if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&r->d_counts), n * 8, up);
                if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&r->d_psi), n * 16, up);
                if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&r->d_eloc), n * 16, up);
                if (e == cudaSuccess) e = cudaMemcpyAsync(r->d_keys, j.samples, n * 16, cudaMemcpyHostToDevice, up);
                if (e == cudaSuccess) e = cudaMemcpyAsync(r->d_counts, j.counts, n * 8, cudaMemcpyHostToDevice, up);
                if (e == cudaSuccess) e = cudaMemcpyAsync(r->d_psi, j.psi, n * 16, cudaMemcpyHostToDevice, up);
                if (e == cudaSuccess) e = cudaStreamSynchronize(up);
            }
        }
        lk.lock();
        if (create) {
            if (st == QC_OK) res->handle = made;
            else res->failed = st;
        }
        res->last_use = now_s();
        if (st != QC_OK || e != cudaSuccess) {
            r->result.status = st != QC_OK ? st : (e == cudaErrorMemoryAllocation ? QC_ERR_OOM : QC_ERR_CUDA);
            finish_request(S, r, up);
            S->cv_done.notify_all();
            continue;
        }
        r->pairs_per_row = std::max<long long>(1, qc_eloc_pairs_per_sample(res->handle));
        S->ready.push_back(r);
        S->cv_submit.notify_all();
    }
}

void run_wave(qc_server* S, Lane& L, int lane_index, int prec, const std::vector<Request*>& take);

// The largest remaining work a wave admits beside its oldest request, as a multiple of the
// oldest's remaining work.
constexpr double kWaveSpread = 4.0;

// Launch one wave on a free lane: requests of one precision, about `quantum` enumerated
// pairs in all -- the oldest request first with at least `oldest_pct` percent of it, then
// the others by least remaining work; a request that does not fit whole runs a slice of
// its rows.
void launch_wave(qc_server* S, Lane& L, int lane_index) {
    const int prec = S->ready.front()->job.precision;
    std::vector<Request*> cand, keep;
    for (Request* r : S->ready) (r->job.precision == prec ? cand : keep).push_back(r);
    auto rows_left = [](const Request* r) { return r->job.n_u - r->next_row; };
    auto work_left = [&](const Request* r) {
        return static_cast<double>(rows_left(r)) * static_cast<double>(r->pairs_per_row);
    };
    std::stable_sort(cand.begin(), cand.end(), [](const Request* a, const Request* b) { return a->ticket < b->ticket; });
    if (cand.size() > 1)
        std::stable_sort(cand.begin() + 1, cand.end(),
                         [&](const Request* a, const Request* b) { return work_left(a) < work_left(b); });
    const double Q = S->quantum > 0 ? static_cast<double>(S->quantum) : 1e300;
    // after a wave that ran a slice of a long request, short requests that are ready get a
    // wave of their own first: they wait for at most one slice, never for a whole long job
    if (S->quantum > 0 && S->last_wave_sliced) {
        std::vector<Request*> small, rest;
        for (Request* r : cand) (r->next_row == 0 && work_left(r) <= 0.5 * Q ? small : rest).push_back(r);
        if (!small.empty()) {
            std::stable_sort(small.begin(), small.end(),
                             [&](const Request* a, const Request* b) { return work_left(a) < work_left(b); });
            std::vector<Request*> take;
            double room = Q;
            long long rows_in = 0;
            for (Request* r : small) {
                if (!take.empty() && (work_left(r) > room || (S->wave_rows > 0 && rows_in + rows_left(r) > S->wave_rows))) {
                    rest.push_back(r);
                    continue;
                }
                r->slice_end = r->job.n_u;
                room -= work_left(r);
                rows_in += rows_left(r);
                take.push_back(r);
            }
            for (Request* r : rest) keep.push_back(r);
            S->ready.swap(keep);
            S->last_wave_sliced = false;
            run_wave(S, L, lane_index, prec, take);
            return;
        }
    }
    // the oldest request is guaranteed its share of the quantum (no request starves); the others
    // fill the rest, least remaining work first; room left over goes back to the oldest
    Request* oldest = cand.front();
    const double reserve = std::min(work_left(oldest), 0.01 * S->oldest_pct * Q);
    double room = Q - reserve;
    std::vector<Request*> take{oldest};
    // a request far larger than the oldest would hold the wave's short requests back until it
    // ends: it waits for a wave of its own (on the next free lane) instead
    const double cap = kWaveSpread * std::max(work_left(oldest), 1.0);
    long long rows_in = rows_left(oldest);
    for (size_t i = 1; i < cand.size(); ++i) {
        Request* r = cand[i];
        if ((work_left(r) > cap && r->next_row == 0) || (S->wave_rows > 0 && rows_in + rows_left(r) > S->wave_rows)) {
            keep.push_back(r);
            continue;
        }
        long long rows = rows_left(r);
        if (rows > 0 && work_left(r) > room)
            rows = std::max<long long>(0, static_cast<long long>(room / static_cast<double>(r->pairs_per_row)));
        if (rows == 0 && rows_left(r) > 0) {
            keep.push_back(r);  // no room left in this wave
            continue;
        }
        r->slice_end = r->next_row + rows;
        room -= static_cast<double>(rows) * static_cast<double>(r->pairs_per_row);
        rows_in += rows;
        take.push_back(r);
    }
    {
        long long rows = rows_left(oldest);
        const double share = reserve + std::max(room, 0.0);
        if (work_left(oldest) > share)
            rows = std::max<long long>(1, static_cast<long long>(share / static_cast<double>(oldest->pairs_per_row)));
        oldest->slice_end = oldest->next_row + rows;
    }
    S->ready.swap(keep);
    bool sliced = false;
    for (Request* r : take) sliced = sliced || r->slice_end < r->job.n_u || r->next_row > 0;
    S->last_wave_sliced = sliced;
    run_wave(S, L, lane_index, prec, take);
}

// Launch `take` (with their row slices set) as one batch on lane L.  A wave of one whole
// request whose Hamiltonian no other wave is using runs the single-molecule path on that
// handle's own workspace instead: the widest launch shape, and E_loc exactly the handle API's.
void run_wave(qc_server* S, Lane& L, int lane_index, int prec, const std::vector<Request*>& take) {
    if (take.size() == 1 && take[0]->next_row == 0 && take[0]->slice_end == take[0]->job.n_u &&
        !take[0]->res->evaluating) {
        Request* r = take[0];
        qc_eloc_out out{};
        out.eloc = r->d_eloc;
        out.summary = L.sums;
        const double t0 = now_s();
        cudaError_t e = cudaEventRecord(L.ev, S->upload);   // after the request's uploads
        if (e == cudaSuccess) e = cudaStreamWaitEvent(L.stream, L.ev, 0);
        qc_status st = QC_ERR_CUDA;
        if (e == cudaSuccess)
            st = qc_eloc_eval(r->res->handle, r->d_keys, r->d_counts, r->d_psi, r->job.n_u, nullptr, nullptr, 0,
                              &out, L.stream);
        if (st == QC_OK) e = cudaEventRecord(L.ev, L.stream);
        if (st != QC_OK || e != cudaSuccess) {
            r->result.status = st != QC_OK ? st : QC_ERR_CUDA;
            finish_request(S, r, L.stream);
            S->cv_done.notify_all();
            return;
        }
        if (r->result.t_start == 0.0) r->result.t_start = t0;
        r->res->evaluating = true;
        Wave w;
        w.reqs = take;
        w.stream = lane_index;
        w.single = true;
        L.busy = true;
        S->waves.push_back(w);
        return;
    }
    std::vector<qc_eloc*> hs;
    for (Request* r : take) hs.push_back(r->res->handle);
    qc_status st = QC_OK;
    qc_batch*& B = L.batch[prec];
    if (!B) {
        st = qc_batch_create(hs.data(), static_cast<int>(hs.size()), &B);
        if (st == QC_OK) st = qc::batch_set_alloc_stream(B, L.stream);
    } else {
        st = qc::batch_retarget(B, hs.data(), static_cast<int>(hs.size()));
    }
    for (size_t m = 0; m < take.size() && st == QC_OK; ++m) {
        Request* r = take[m];
        st = qc_batch_set_inputs(B, static_cast<int>(m), r->d_keys, r->d_counts, r->d_psi, r->job.n_u, r->d_eloc);
        if (st == QC_OK)
            st = qc::batch_set_slice(B, static_cast<int>(m), r->next_row, r->slice_end, r->slice_end == r->job.n_u,
                                     r->d_ctr);
    }
    const double t0 = now_s();
    // the wave's stream waits for the uploads of its requests
    cudaError_t e = cudaEventRecord(L.ev, S->upload);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(L.stream, L.ev, 0);
    if (st == QC_OK && e == cudaSuccess) st = qc_batch_eval(B, L.sums, L.stream);
    if (st == QC_OK && e == cudaSuccess) e = cudaEventRecord(L.ev, L.stream);
    if (st != QC_OK || e != cudaSuccess) {
        for (Request* r : take) {
            r->result.status = st != QC_OK ? st : QC_ERR_CUDA;
            finish_request(S, r, L.stream);
        }
        S->cv_done.notify_all();
        return;
    }
    for (Request* r : take)
        if (r->result.t_start == 0.0) r->result.t_start = t0;
    Wave w;
    w.reqs = take;
    w.stream = lane_index;
    L.busy = true;
    S->waves.push_back(w);
}

// Retire finished waves (non-blocking event queries); E_loc goes to the callers' buffers.
bool retire(qc_server* S) {
    bool any = false;
    for (auto it = S->waves.begin(); it != S->waves.end();) {
        Lane& L = S->lanes[it->stream];
        const cudaError_t q = cudaEventQuery(L.ev);
        if (q == cudaErrorNotReady) {
            ++it;
            continue;
        }
        const double t = now_s();
        for (size_t m = 0; m < it->reqs.size(); ++m) {
            Request* r = it->reqs[m];
            if (q == cudaSuccess && r->slice_end < r->job.n_u) {  // more slices to go
                r->next_row = r->slice_end;
                S->ready.push_back(r);
                continue;
            }
            cudaError_t e = q;
            if (e == cudaSuccess && r->job.eloc_out && r->job.n_u > 0) {
                e = cudaMemcpyAsync(r->job.eloc_out, r->d_eloc, static_cast<size_t>(r->job.n_u) * 16,
                                    cudaMemcpyDeviceToHost, L.stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(L.stream);
            }
            r->result.summary = L.sums[m];
            r->result.status = e == cudaSuccess ? L.sums[m].status : QC_ERR_CUDA;
            r->result.t_done = now_s();
            (void)t;
            if (it->single && r->res) r->res->evaluating = false;  // its handle's workspace is free
            finish_request(S, r, L.stream);
        }
        L.busy = false;
        it = S->waves.erase(it);
        any = true;
    }
    return any;
}

// The admission thread: admits whatever fits whenever a request is submitted or memory
// and slots come free.
void admission(qc_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        admit(S, lk);
        if (S->stop && S->pending.empty()) break;
        S->cv_admit.wait_for(lk, std::chrono::milliseconds(50));
    }
}

void scheduler(qc_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        if (retire(S)) S->cv_done.notify_all();
        // continuous batching: every free lane takes the requests that are ready now
        for (size_t i = 0; i < S->lanes.size() && !S->ready.empty(); ++i)
            if (!S->lanes[i].busy) launch_wave(S, S->lanes[i], static_cast<int>(i));
        if (S->stop && S->pending.empty() && S->ready.empty() && S->waves.empty() && S->active == 0) break;
        if (S->waves.empty() && S->ready.empty())
            S->cv_submit.wait_for(lk, std::chrono::milliseconds(50));
        else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(50));
            lk.lock();
        }
    }
}

}  // namespace

extern "C" {

qc_status qc_server_create(int device, uint64_t budget_bytes, int max_slots, int n_streams, qc_server** out) {
    if (!out) return QC_ERR_ARG;
    *out = nullptr;
    if (budget_bytes == 0 || max_slots <= 0 || max_slots > 65535 || n_streams < 1 || n_streams > 16)
        return QC_ERR_ARG;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return QC_ERR_CUDA;
    qc_server* S = new (std::nothrow) qc_server();
    if (!S) return QC_ERR_OOM;
    S->device = device;
    S->budget = budget_bytes;
    S->max_slots = max_slots;
    S->lanes.resize(n_streams);
    e = cudaStreamCreateWithFlags(&S->upload, cudaStreamNonBlocking);
    for (auto& L : S->lanes) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMallocHost(&L.sums, static_cast<size_t>(max_slots) * sizeof(qc_eloc_summary));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        qc_server_destroy(S);
        return QC_ERR_CUDA;
    }
    S->worker = std::thread(scheduler, S);
    S->admitter = std::thread(admission, S);
    *out = S;
    return QC_OK;
}

qc_status qc_eloc_submit(qc_server* S, const qc_eloc_job* job, uint64_t* ticket) {
    if (!S || !job || !ticket) return QC_ERR_ARG;
    if (job->n_orb < 2 || job->n_orb > 128 || (job->n_orb & 1) || job->n_elec <= 0 || job->n_elec >= job->n_orb ||
        (job->n_elec & 1) || job->n_u < 0 || (job->n_u > 0 && (!job->samples || !job->counts || !job->psi)) ||
        !job->h || !job->eri || (job->precision != QC_FP64 && job->precision != QC_FP32_COMP))
        return QC_ERR_ARG;
    const double t_call = now_s();  // latency counts from the call, copies included
    if (job->flags & ~QC_JOB_BORROW_INTEGRALS) return QC_ERR_ARG;
    auto r = std::make_unique<Request>();
    r->job = *job;
    r->bytes = request_bytes(job->n_u);
    const size_t ham = hamiltonian_bytes(job->n_orb, job->precision);
    if (r->bytes + ham > S->budget) return QC_ERR_BUDGET;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->stop) return QC_ERR_ARG;
    auto rit = job->mol_key ? S->residents.find(job->mol_key) : S->residents.end();
    if (rit != S->residents.end()) {  // resident: pin it until this request finishes
        r->res = rit->second.get();
        r->res->users++;
    } else if (!(job->flags & QC_JOB_BORROW_INTEGRALS)) {
        // the caller may free its integrals after submit: copy them, outside the lock
        lk.unlock();
        const size_t K = static_cast<size_t>(job->n_orb / 2);
        r->h.assign(job->h, job->h + K * K);
        r->eri.assign(job->eri, job->eri + K * K * K * K);
        lk.lock();
        if (S->stop) return QC_ERR_ARG;
    }
    r->ticket = S->next_ticket++;
    r->result.t_submit = t_call;
    *ticket = r->ticket;
    Request* raw = r.release();
    S->all[raw->ticket] = raw;
    S->pending.push_back(raw);
    S->cv_admit.notify_all();
    return QC_OK;
}

qc_status qc_eloc_poll(qc_server* S, uint64_t ticket, qc_eloc_result* result, int timeout_us) {
    if (!S || !result) return QC_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return QC_ERR_ARG;
    Request* r = it->second;
    if (!r->done && timeout_us > 0)
        S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->done; });
    if (!r->done) return QC_PENDING;
    *result = r->result;
    S->all.erase(it);
    delete r;
    return QC_OK;
}

qc_status qc_server_set_option(qc_server* S, int option, int64_t value) {
    if (!S) return QC_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (option == QC_SRV_OPT_QUANTUM && value >= 0) S->quantum = value;
    else if (option == QC_SRV_OPT_OLDEST_PCT && value >= 1 && value <= 100) S->oldest_pct = static_cast<int>(value);
    else if (option == QC_SRV_OPT_WAVE_ROWS && value >= 0) S->wave_rows = value;
    else return QC_ERR_ARG;
    return QC_OK;
}

qc_status qc_server_stats(qc_server* S, uint64_t* stats4) {
    if (!S || !stats4) return QC_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    stats4[0] = S->used;
    stats4[1] = static_cast<uint64_t>(S->active);
    stats4[2] = S->pending.size();
    stats4[3] = S->residents.size();
    return QC_OK;
}

qc_status qc_server_destroy(qc_server* S) {
    if (!S) return QC_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_submit.notify_all();
        S->cv_admit.notify_all();
    }
    if (S->admitter.joinable()) S->admitter.join();
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->device);
    for (auto& kv : S->all) delete kv.second;
    for (auto& kv : S->residents) qc_eloc_destroy(kv.second->handle);
    for (auto& L : S->lanes) {
        for (qc_batch* b : L.batch)
            if (b) qc_batch_destroy(b);
        if (L.sums) cudaFreeHost(L.sums);
        if (L.ev) cudaEventDestroy(L.ev);
        if (L.stream) cudaStreamDestroy(L.stream);
    }
    if (S->upload) cudaStreamDestroy(S->upload);
    delete S;
    return QC_OK;
}

}  // extern "C"
