// qc_join.cu -- the sample-space join index: the table rows grouped by their alpha string
// and by their beta string.
//
// In the sample-space energy (Eq. 5 with x' restricted to the sampled set, Sec. IV-C-4)
// a connected x' = (alpha', beta') of a sample x = (alpha, beta) has either alpha' = alpha
// (a beta single or beta-beta double), beta' = beta (an alpha-alpha double) or alpha' a
// single excitation of alpha (an alpha single when beta' = beta, else an alpha-beta double
// with beta' a single excitation of beta).  So the rows that can connect to x are those of
// a few groups: the rows sharing x's alpha string, those sharing its beta string, and the
// rows of each alpha' group.  The local-energy kernel scans a short group row by row (one
// popcount of the other spin's string difference decides the connection) and enumerates the
// excitations into a long one through the filter and the bucket table.  An alpha-beta double
// also lies in the group of its beta' (a single excitation of beta), so for a sample with many
// long alpha' groups the kernel may scan short beta' groups for their rows instead.
//
// Built once per evaluation after K0, which leaves each row's slot in the alpha and beta
// spin-string sets as a sort key (alpha rows first, beta rows offset by the set size) and
// the group sizes:
//   starts:    exclusive prefix sum of the group sizes
//   J1 hist:   per-tile digit counts (11-bit digits of the slot key)
//   scan:      exclusive prefix over the (digit, tile) counts, digit-major
//   J2 scatter: stable scatter of (key, row) by digit; after the passes the pairs are in
//              (slot, row) order, so every group lists its rows in row order and the scan
//              order of a group -- and with it the order of accumulation -- is the same on
//              every run
//   J3 gather: each entry's row and the row's string of the other spin (16 bytes, so one
//              load brings the kernel both); the alpha entries leave each row's alpha-group
//              size in a per-row array
//   J4 mark:   each beta entry's row word gets the row's alpha-group size in its high 32
//              bits (the kernel's scan of a beta' group keeps the rows of long alpha' groups
//              by it, without a lookup)
// Traffic per row: 8 B read (hist) + 8 B read + 8 B written (scatter) per pass and key half,
// then 16 B read, 16 B written (gather) and 12 B read, 8 B written (mark); a few tens of
// microseconds at 10^5 rows.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "qc_device.cuh"
#include "qc_eloc.h"
#include "qc_internal.h"

namespace {

constexpr int kJTile = 2048;  // items per warp tile (64 steps of 32)
constexpr int kJWarps = 4;    // warps per block (32 KB of per-warp digit counts)
constexpr int kJBits = 11;
constexpr int kJBins = 1 << kJBits;

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

struct JLayout {
    size_t key1, val0, val1, table, sums, alen, total;
};

// sort space for m items and n_slots group sizes
JLayout jlayout(long long m, unsigned long long n_slots) {
    m = std::max<long long>(m, 2);
    const long long tiles = (m + kJTile - 1) / kJTile;
    const long long table_n = static_cast<long long>(kJBins) * tiles;
    const long long scan_n = std::max<long long>(table_n, static_cast<long long>(n_slots));
    JLayout L{};
    size_t off = 0;
    L.key1 = off; off = align256(off + static_cast<size_t>(m) * 4);
    L.val0 = off; off = align256(off + static_cast<size_t>(m) * 4);
    L.val1 = off; off = align256(off + static_cast<size_t>(m) * 4);
    L.table = off; off = align256(off + static_cast<size_t>(table_n) * 4);
    L.sums = off; off = align256(off + static_cast<size_t>(scan_n / 4096 + 2) * 4 + 4096);
    L.alen = off; off = align256(off + static_cast<size_t>(m / 2 + 1) * 4);
    L.total = off;
    return L;
}

// One block per tile of kJTile items: the tile's digit counts, table[d * tiles + t].
__global__ void __launch_bounds__(32 * kJWarps) join_hist_kernel(const unsigned* __restrict__ key, long long m,
                                                                 int shift, long long tiles,
                                                                 unsigned* __restrict__ table) {
    __shared__ unsigned hist[kJBins];
    for (int d = threadIdx.x; d < kJBins; d += blockDim.x) hist[d] = 0u;
    __syncthreads();
    const long long t = blockIdx.x;
    const long long i0 = t * kJTile;
    const long long i1 = i0 + kJTile < m ? i0 + kJTile : m;
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) atomicAdd(&hist[(key[i] >> shift) & (kJBins - 1)], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < kJBins; d += blockDim.x) table[static_cast<long long>(d) * tiles + t] = hist[d];
}

// Stable scatter of one tile per block: each warp takes a contiguous quarter of the tile,
// counts its digits, and the block turns the tile's offsets into per-warp bases (warps in
// tile order); then every warp walks its quarter in index order (__match_any_sync ranks
// equal digits within a step of 32).  The first pass takes the row from the index (item
// i < n is row i's alpha key, item n + i its beta key).
__global__ void __launch_bounds__(32 * kJWarps) join_scatter_kernel(const unsigned* __restrict__ key_in,
                                                                    const unsigned* __restrict__ val_in,
                                                                    long long n, unsigned* __restrict__ key_out,
                                                                    unsigned* __restrict__ val_out, long long m,
                                                                    int shift, long long tiles,
                                                                    const unsigned* __restrict__ offs) {
    __shared__ unsigned run[kJWarps][kJBins];
    constexpr int kSub = kJTile / kJWarps;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long t = blockIdx.x;
    for (int d = threadIdx.x; d < kJWarps * kJBins; d += blockDim.x) (&run[0][0])[d] = 0u;
    __syncthreads();
    const long long i0 = t * kJTile + static_cast<long long>(warp) * kSub;
    long long i1 = i0 + kSub;
    if (i1 > m) i1 = m;
    for (long long i = i0 + lane; i < i1; i += 32) atomicAdd(&run[warp][(key_in[i] >> shift) & (kJBins - 1)], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < kJBins; d += blockDim.x) {
        unsigned base = offs[static_cast<long long>(d) * tiles + t];
        for (int w = 0; w < kJWarps; ++w) {
            const unsigned c = run[w][d];
            run[w][d] = base;
            base += c;
        }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (long long b = i0; b < i1; b += 32) {
        const long long i = b + lane;
        const bool v = i < i1;
        const unsigned active = __ballot_sync(0xffffffffu, v);
        if (v) {
            const unsigned k = key_in[i];
            const unsigned val = val_in ? val_in[i] : static_cast<unsigned>(i < n ? i : i - n);
            const unsigned d = (k >> shift) & (kJBins - 1);
            const unsigned same = __match_any_sync(active, d);
            const unsigned base = run[warp][d];
            const unsigned pos = base + __popc(same & lt);
            key_out[pos] = k;
            val_out[pos] = val;
            __syncwarp(active);
            if ((same & lt) == 0u) run[warp][d] = base + __popc(same);  // the lowest lane of the group
        }
        __syncwarp();
    }
}

// (alen: each row's alpha-group size, from its alpha entry; with pa: each row's own alpha-
// and beta-group sizes into pa / pb, for the sample order)
__global__ void __launch_bounds__(256) join_gather_kernel(const ulonglong2* __restrict__ keys,
                                                          const unsigned* __restrict__ skey,
                                                          const unsigned* __restrict__ srow, long long m,
                                                          unsigned set_size, ulonglong2* __restrict__ gent,
                                                          const unsigned* __restrict__ jlen, unsigned* __restrict__ alen,
                                                          unsigned* pa, unsigned* pb) {
    for (long long p = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; p < m;
         p += static_cast<long long>(gridDim.x) * blockDim.x) {
        const unsigned k = skey[p];
        if (k >= 2u * set_size) continue;  // rows that failed validation: past every group
        const unsigned row = srow[p];
        // alpha groups list beta strings and the other way round
        gent[p] = make_ulonglong2(qc::spin_string(keys[row], k < set_size ? 1 : 0), row);
        if (k < set_size) alen[row] = jlen[k];
        if (pa != nullptr) (k < set_size ? pa : pb)[row] = jlen[k];
    }
}

// J4: the beta entries' row words get the row's alpha-group size in their high half.
__global__ void __launch_bounds__(256) join_mark_kernel(const unsigned* __restrict__ skey,
                                                        const unsigned* __restrict__ srow, long long m,
                                                        unsigned set_size, ulonglong2* __restrict__ gent,
                                                        const unsigned* __restrict__ alen) {
    for (long long p = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; p < m;
         p += static_cast<long long>(gridDim.x) * blockDim.x) {
        const unsigned k = skey[p];
        if (k < set_size || k >= 2u * set_size) continue;
        const unsigned row = srow[p];
        gent[p].y = static_cast<unsigned long long>(row) | (static_cast<unsigned long long>(alen[row]) << 32);
    }
}

// The molecule of a batch's sorted slot key k: the largest one with slot_base <= k.
__device__ __forceinline__ int batch_molecule(const unsigned* __restrict__ slot_base, int n_mol, unsigned k) {
    int lo = 0, hi = n_mol;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (slot_base[mid] <= k) lo = mid; else hi = mid;
    }
    return lo;
}

// A batch's entries: the molecule from the sorted key (slot_base: each molecule's first slot
// key, then the sentinel), the spin from the key's place in the molecule's two sets.
__global__ void __launch_bounds__(256) join_gather_batch_kernel(const qc::MolParams* __restrict__ mols,
                                                                const unsigned* __restrict__ slot_base, int n_mol,
                                                                const unsigned* __restrict__ skey,
                                                                const unsigned* __restrict__ srow, long long m,
                                                                ulonglong2* __restrict__ gent,
                                                                const unsigned* __restrict__ row_base,
                                                                const unsigned* __restrict__ jlen,
                                                                unsigned* __restrict__ alen, unsigned* pa,
                                                                unsigned* pb) {
    const unsigned sentinel = slot_base[n_mol];
    for (long long p = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; p < m;
         p += static_cast<long long>(gridDim.x) * blockDim.x) {
        const unsigned k = skey[p];
        if (k >= sentinel) continue;
        const int lo = batch_molecule(slot_base, n_mol, k);
        const unsigned size = (slot_base[lo + 1] - slot_base[lo]) / 2u;
        const unsigned row = srow[p];
        const bool alpha = k - slot_base[lo] < size;
        gent[p] = make_ulonglong2(qc::spin_string(mols[lo].tp.keys[row], alpha ? 1 : 0), row);
        if (alpha) alen[row_base[lo] + row] = jlen[k];
        if (pa != nullptr) (alpha ? pa : pb)[row_base[lo] + row] = jlen[k];
    }
}

// J4 of a batch: the beta entries' row words get the row's alpha-group size.
__global__ void __launch_bounds__(256) join_mark_batch_kernel(const unsigned* __restrict__ slot_base, int n_mol,
                                                              const unsigned* __restrict__ skey,
                                                              const unsigned* __restrict__ srow, long long m,
                                                              ulonglong2* __restrict__ gent,
                                                              const unsigned* __restrict__ row_base,
                                                              const unsigned* __restrict__ alen) {
    const unsigned sentinel = slot_base[n_mol];
    for (long long p = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; p < m;
         p += static_cast<long long>(gridDim.x) * blockDim.x) {
        const unsigned k = skey[p];
        if (k >= sentinel) continue;
        const int lo = batch_molecule(slot_base, n_mol, k);
        const unsigned size = (slot_base[lo + 1] - slot_base[lo]) / 2u;
        if (k - slot_base[lo] < size) continue;
        const unsigned row = srow[p];
        gent[p].y = static_cast<unsigned long long>(row) |
                    (static_cast<unsigned long long>(alen[row_base[lo] + row]) << 32);
    }
}

// Samples that are not the table's rows (a caller's table, e.g. one rank's rows against the
// whole sample set): each sample's own alpha- and beta-group sizes in the table, looked up by
// its spin strings in the table's sets (0 for a string the table does not hold), into pa / pb.
__global__ void __launch_bounds__(256) sample_group_sizes_kernel(const qc::TableParams tp,
                                                                 const ulonglong2* __restrict__ samples,
                                                                 long long n_u,
                                                                 const unsigned long long* __restrict__ T,
                                                                 unsigned set_size,
                                                                 const unsigned* __restrict__ jlen,
                                                                 unsigned* __restrict__ pa,
                                                                 unsigned* __restrict__ pb) {
    for (long long r = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; r < n_u;
         r += static_cast<long long>(gridDim.x) * blockDim.x) {
        const ulonglong2 key = samples[r];
        unsigned long long ha = 0, hb = 0;  // the alpha and beta parts of the key's linear hash
        for (unsigned long long w = key.x; w; w &= w - 1ULL) {
            const int bit = __ffsll(w) - 1;
            if (bit & 1) hb ^= __ldg(T + bit); else ha ^= __ldg(T + bit);
        }
        for (unsigned long long w = key.y; w; w &= w - 1ULL) {
            const int bit = __ffsll(w) - 1;
            if (bit & 1) hb ^= __ldg(T + 64 + bit); else ha ^= __ldg(T + 64 + bit);
        }
        const unsigned long long sa = qc::spin_string(key, 0), sb = qc::spin_string(key, 1);
        const unsigned la = sa != 0ULL ? qc::set_slot(tp.aset, tp.set_mask, sa, ha) : qc::kNoSlot;
        const unsigned lb = sb != 0ULL ? qc::set_slot(tp.bset, tp.set_mask, sb, hb) : qc::kNoSlot;
        pa[r] = la != qc::kNoSlot ? __ldg(jlen + la) : 0u;
        pb[r] = lb != qc::kNoSlot ? __ldg(jlen + set_size + lb) : 0u;
    }
}

// Sort key of the heavy-first sample order: 255 - (8 log2 of the sizes of the sample's own
// alpha and beta groups, in eighths of an octave); integer arithmetic only.
__device__ __forceinline__ unsigned order_priority_key(unsigned v) {
    unsigned bucket = 0;
    if (v != 0u) {
        const unsigned b = 31u - static_cast<unsigned>(__clz(v));
        const unsigned frac = b >= 3u ? (v >> (b - 3u)) & 7u : (v << (3u - b)) & 7u;
        bucket = 8u * b + frac;
    }
    return 255u - (bucket > 255u ? 255u : bucket);
}

__global__ void __launch_bounds__(256) order_key_kernel(const unsigned* __restrict__ pa,
                                                        const unsigned* __restrict__ pb, long long n,
                                                        unsigned* __restrict__ key) {
    for (long long r = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
         r += static_cast<long long>(gridDim.x) * blockDim.x)
        key[r] = order_priority_key(pa[r] + pb[r]);
}

// A batch's rows (row_base: each joining molecule's first row in pa / pb): key = molecule
// index << 8 | priority, value = the row within its molecule, so one stable sort gives every
// molecule's rows heavy first, molecule after molecule.
__global__ void __launch_bounds__(256) order_key_batch_kernel(const unsigned* __restrict__ row_base, int n_mol,
                                                              const unsigned* __restrict__ pa,
                                                              const unsigned* __restrict__ pb, long long n,
                                                              unsigned* __restrict__ key, unsigned* __restrict__ val) {
    for (long long r = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
         r += static_cast<long long>(gridDim.x) * blockDim.x) {
        int lo = 0, hi = n_mol;  // largest molecule with row_base <= r
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (row_base[mid] <= static_cast<unsigned>(r)) lo = mid; else hi = mid;
        }
        key[r] = (static_cast<unsigned>(lo) << 8) | order_priority_key(pa[r] + pb[r]);
        val[r] = static_cast<unsigned>(r) - row_base[lo];
    }
}

int bits_for(unsigned long long v) {  // bits to hold 0..v
    int b = 1;
    while (b < 64 && (v >> b) != 0ULL) ++b;
    return b;
}

cudaError_t radix_pairs(unsigned* key0, const unsigned* val_in, long long n_half, long long m,
                        unsigned long long max_key, unsigned* key1, unsigned* val0, unsigned* val1,
                        unsigned* table, unsigned* sums, const unsigned** skey, const unsigned** sval,
                        cudaStream_t s);

// Group starts (exclusive prefix of the n_slots sizes) and the stable sort of m (key, value)
// items by key, values from val_in or (val_in null) the item index modulo n_half.  Returns
// the sorted arrays (in the workspace or in jkey, which the sort uses as a buffer).
cudaError_t join_sort(unsigned* jkey, const unsigned* val_in, long long n_half, long long m,
                      unsigned long long n_slots, unsigned* jlen, unsigned* jstart, void* ws,
                      const unsigned** skey, const unsigned** sval, cudaStream_t s) {
    const JLayout L = jlayout(m, n_slots);
    unsigned char* W = static_cast<unsigned char*>(ws);
    unsigned* key1 = reinterpret_cast<unsigned*>(W + L.key1);
    unsigned* val0 = reinterpret_cast<unsigned*>(W + L.val0);
    unsigned* val1 = reinterpret_cast<unsigned*>(W + L.val1);
    unsigned* table = reinterpret_cast<unsigned*>(W + L.table);
    unsigned* sums = reinterpret_cast<unsigned*>(W + L.sums);
    cudaError_t e = cudaMemcpyAsync(jstart, jlen, n_slots * sizeof(unsigned), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = qc::exclusive_scan_u32(jstart, static_cast<long long>(n_slots), sums, s);
    if (e == cudaSuccess) e = radix_pairs(jkey, val_in, n_half, m, n_slots, key1, val0, val1, table, sums, skey, sval, s);
    return e;
}

// Stable LSD sort of m (key, value) items by key (keys up to max_key), values from val_in or
// (val_in null) the item index modulo n_half; key0 is overwritten (a buffer of the passes).
cudaError_t radix_pairs(unsigned* key0, const unsigned* val_in, long long n_half, long long m,
                        unsigned long long max_key, unsigned* key1, unsigned* val0, unsigned* val1,
                        unsigned* table, unsigned* sums, const unsigned** skey, const unsigned** sval,
                        cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    unsigned* jkey = key0;
    const int passes = (bits_for(max_key) + kJBits - 1) / kJBits;
    const long long tiles = (m + kJTile - 1) / kJTile;
    const unsigned blocks = static_cast<unsigned>(tiles);  // one block per tile
    const unsigned* src_k = jkey;
    const unsigned* src_v = val_in;
    unsigned* dk[2] = {key1, jkey};
    unsigned* dv[2] = {val0, val1};
    for (int p = 0; p < passes && e == cudaSuccess; ++p) {
        join_hist_kernel<<<blocks, 32 * kJWarps, 0, s>>>(src_k, m, p * kJBits, tiles, table);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = qc::exclusive_scan_u32(table, static_cast<long long>(kJBins) * tiles, sums, s);
        if (e == cudaSuccess) {
            join_scatter_kernel<<<blocks, 32 * kJWarps, 0, s>>>(src_k, src_v, n_half, dk[p & 1], dv[p & 1], m,
                                                               p * kJBits, tiles, table);
            e = cudaGetLastError();
        }
        src_k = dk[p & 1];
        src_v = dv[p & 1];
    }
    *skey = src_k;
    *sval = src_v;
    return e;
}

}  // namespace

size_t qc::join_workspace_bytes(long long n, unsigned set_size) { return jlayout(2 * n, 2ULL * set_size).total; }

cudaError_t qc::launch_join_index(const TableParams& tp, unsigned set_size, void* ws, unsigned* jkey,
                                  unsigned* jlen, unsigned* jstart, ulonglong2* gent, cudaStream_t s,
                                  unsigned* order, unsigned* pa, unsigned* pb, const ulonglong2* samples,
                                  long long n_samples, const unsigned long long* T) {
    if (tp.n <= 0) return cudaSuccess;
    const long long m = 2 * tp.n;
    const unsigned* skey = nullptr;
    const unsigned* sval = nullptr;
    cudaError_t e = join_sort(jkey, nullptr, tp.n, m, 2ULL * set_size, jlen, jstart, ws, &skey, &sval, s);
    const unsigned gblocks = static_cast<unsigned>(std::min<long long>((m + 255) / 256, 8192));
    unsigned* alen = reinterpret_cast<unsigned*>(static_cast<unsigned char*>(ws) + jlayout(m, 2ULL * set_size).alen);
    if (e == cudaSuccess) {
        join_gather_kernel<<<gblocks, 256, 0, s>>>(tp.keys, skey, sval, m, set_size, gent, jlen, alen,
                                                   order != nullptr && samples == nullptr ? pa : nullptr, pb);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        join_mark_kernel<<<gblocks, 256, 0, s>>>(skey, sval, m, set_size, gent, alen);
        e = cudaGetLastError();
    }
    // the samples to order: the table's rows, or a caller's samples (their groups looked up)
    const long long n = samples != nullptr ? n_samples : tp.n;
    if (e == cudaSuccess && order != nullptr && samples != nullptr && n > 0) {
        const unsigned sblocks = static_cast<unsigned>(std::min<long long>((n + 255) / 256, 8192));
        sample_group_sizes_kernel<<<sblocks, 256, 0, s>>>(tp, samples, n, T, set_size, jlen, pa, pb);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && order != nullptr && n > 0) {
        // heavy-first sample order: one stable 8-bit pass over the priority keys (the sort
        // buffers are free once the gather has run)
        const JLayout L = jlayout(m, 2ULL * set_size);
        unsigned char* W = static_cast<unsigned char*>(ws);
        unsigned* okey = reinterpret_cast<unsigned*>(W + L.key1);
        unsigned* okey2 = reinterpret_cast<unsigned*>(W + L.val0);
        unsigned* table = reinterpret_cast<unsigned*>(W + L.table);
        unsigned* sums = reinterpret_cast<unsigned*>(W + L.sums);
        order_key_kernel<<<std::min<unsigned>(gblocks, 4096u), 256, 0, s>>>(pa, pb, n, okey);
        e = cudaGetLastError();
        const long long tiles = (n + kJTile - 1) / kJTile;
        const unsigned blocks = static_cast<unsigned>(tiles);  // one block per tile
        if (e == cudaSuccess) {
            join_hist_kernel<<<blocks, 32 * kJWarps, 0, s>>>(okey, n, 0, tiles, table);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = qc::exclusive_scan_u32(table, static_cast<long long>(kJBins) * tiles, sums, s);
        if (e == cudaSuccess) {
            join_scatter_kernel<<<blocks, 32 * kJWarps, 0, s>>>(okey, nullptr, n, okey2, order, n, 0, tiles, table);
            e = cudaGetLastError();
        }
    }
    return e;
}

size_t qc::join_batch_workspace_bytes(long long m, unsigned long long n_slots) { return jlayout(m, n_slots).total; }

cudaError_t qc::launch_join_batch(const MolParams* mols, const unsigned* slot_base, int n_mol, long long m,
                                  unsigned long long n_slots, void* ws, unsigned* jkey, unsigned* jval,
                                  unsigned* jlen, unsigned* jstart, ulonglong2* gent, cudaStream_t s,
                                  const unsigned* row_base, unsigned* order, unsigned* pa, unsigned* pb) {
    if (m <= 0) return cudaSuccess;
    const unsigned* skey = nullptr;
    const unsigned* sval = nullptr;
    cudaError_t e = join_sort(jkey, jval, 0, m, n_slots, jlen, jstart, ws, &skey, &sval, s);
    const unsigned gblocks = static_cast<unsigned>(std::min<long long>((m + 255) / 256, 8192));
    unsigned* alen = reinterpret_cast<unsigned*>(static_cast<unsigned char*>(ws) + jlayout(m, n_slots).alen);
    if (e == cudaSuccess) {
        join_gather_batch_kernel<<<gblocks, 256, 0, s>>>(mols, slot_base, n_mol, skey, sval, m, gent, row_base, jlen,
                                                         alen, order ? pa : nullptr, pb);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        join_mark_batch_kernel<<<gblocks, 256, 0, s>>>(slot_base, n_mol, skey, sval, m, gent, row_base, alen);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && order != nullptr) {
        // every joining molecule's rows heavy first: keys and values into the sort's input
        // buffers (free once the gather has run), one stable sort, the values into order
        const long long R = m / 2;
        const JLayout L = jlayout(m, n_slots);
        unsigned char* W = static_cast<unsigned char*>(ws);
        order_key_batch_kernel<<<std::min<unsigned>(gblocks, 4096u), 256, 0, s>>>(row_base, n_mol, pa, pb, R, jkey,
                                                                                 jval);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = radix_pairs(jkey, jval, R, R, (static_cast<unsigned long long>(n_mol) << 8) | 255ULL,
                            reinterpret_cast<unsigned*>(W + L.key1), reinterpret_cast<unsigned*>(W + L.val0),
                            reinterpret_cast<unsigned*>(W + L.val1), reinterpret_cast<unsigned*>(W + L.table),
                            reinterpret_cast<unsigned*>(W + L.sums), &skey, &sval, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(order, sval, static_cast<size_t>(R) * sizeof(unsigned), cudaMemcpyDeviceToDevice, s);
    }
    return e;
}
