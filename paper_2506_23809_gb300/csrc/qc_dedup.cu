// qc_dedup.cu -- the sample table of Sec. IV-C-4 built on the device: a raw stream of
// sampled bitstrings (any order, repeats) becomes the ascending unique keys with their
// multiplicities, the input that qc_eloc_eval takes.  The paper names the construction of
// this lookup table as what limits scaling once the unique-sample count grows.
//
// A stable least-significant-digit radix sort over the n_orb significant bits (8-bit
// digits, ceil(n_orb / 8) passes), then run lengths:
//   per pass  KH hist:    every warp counts the digits of its tile of keys
//             scan:       exclusive prefix over the (digit, tile) counts, digit-major, so
//                         equal digits keep the order of their tiles
//             KS scatter: every warp walks its tile in order and sends each key to its
//                         digit's next slot (__match_any_sync ranks equal digits within
//                         the 32 keys of a step, so the sort is stable)
//   unique    KU flags:   head-of-run flags, per-block counts; scan; KE emit: the head
//                         keys, their positions; KC counts: differences of positions.
// Traffic per key: 16 B read (hist) + 16 B read + 16 B written (scatter) per pass, then
// 16 B read, 24 B written.  Every step is bound by HBM bandwidth.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "qc_eloc.h"
#include "qc_internal.h"

namespace {

constexpr int kTile = 2048;           // keys per warp tile (64 steps of 32)
constexpr int kWarpsPerBlock = 8;
constexpr int kBins = 256;
constexpr int kScanBlock = 1024;      // threads of a scan block
constexpr int kScanItems = 4;         // items per thread of a scan block
constexpr int kScanSeg = kScanBlock * kScanItems;

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

struct Layout {
    size_t bufA, bufB, heads, table, sums, flag, total;
};

Layout layout(long long n) {
    const long long tiles = (n + kTile - 1) / kTile;
    const long long table_n = static_cast<long long>(kBins) * std::max<long long>(tiles, 1);
    const long long scan_n = std::max(table_n, n);  // the unique stage scans n flags
    const long long segs = (scan_n + kScanSeg - 1) / kScanSeg;
    Layout L{};
    size_t off = 0;
    L.bufA = off; off = align256(off + static_cast<size_t>(std::max<long long>(n, 1)) * 16);
    L.bufB = off; off = align256(off + static_cast<size_t>(std::max<long long>(n, 1)) * 16);
    L.heads = off; off = align256(off + static_cast<size_t>(n + 1) * 8);
    L.table = off; off = align256(off + static_cast<size_t>(std::max(table_n, n)) * 4);
    L.sums = off; off = align256(off + static_cast<size_t>(segs + 1) * 4 + 4096);
    L.flag = off; off = align256(off + 16);
    L.total = off;
    return L;
}

__device__ __forceinline__ unsigned digit_of(const ulonglong2 k, int pass) {
    const int b = 8 * pass;
    return b < 64 ? static_cast<unsigned>((k.x >> b) & 255u) : static_cast<unsigned>((k.y >> (b - 64)) & 255u);
}

// KH: per-tile digit counts, table[d * tiles + t]; pass 0 also checks the unused bits
__global__ void __launch_bounds__(256) dedup_hist_kernel(const ulonglong2* __restrict__ src, long long n, int pass,
                                                         long long tiles, unsigned* __restrict__ table,
                                                         ulonglong2 high_mask, unsigned* __restrict__ flag) {
    __shared__ unsigned hist[kWarpsPerBlock][kBins];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = lane; d < kBins; d += 32) hist[warp][d] = 0u;
    __syncwarp();
    const long long t = static_cast<long long>(blockIdx.x) * kWarpsPerBlock + warp;
    if (t < tiles) {
        const long long i0 = t * kTile;
        const long long i1 = i0 + kTile < n ? i0 + kTile : n;
        bool bad = false;
        for (long long i = i0 + lane; i < i1; i += 32) {
            const ulonglong2 k = src[i];
            if (pass == 0) bad = bad || (k.x & high_mask.x) || (k.y & high_mask.y);
            atomicAdd(&hist[warp][digit_of(k, pass)], 1u);
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flag, 1u);
        __syncwarp();
        for (int d = lane; d < kBins; d += 32) table[static_cast<long long>(d) * tiles + t] = hist[warp][d];
    }
}

// KS: stable scatter of each tile in index order
__global__ void __launch_bounds__(256) dedup_scatter_kernel(const ulonglong2* __restrict__ src,
                                                            ulonglong2* __restrict__ dst, long long n, int pass,
                                                            long long tiles, const unsigned* __restrict__ offs) {
    __shared__ unsigned run[kWarpsPerBlock][kBins];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long t = static_cast<long long>(blockIdx.x) * kWarpsPerBlock + warp;
    if (t >= tiles) return;  // warp-uniform; no block-wide barrier below
    for (int d = lane; d < kBins; d += 32) run[warp][d] = offs[static_cast<long long>(d) * tiles + t];
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
    const long long i0 = t * kTile;
    const long long i1 = i0 + kTile < n ? i0 + kTile : n;
    for (long long b = i0; b < i1; b += 32) {
        const long long i = b + lane;
        const bool v = i < i1;
        const unsigned active = __ballot_sync(0xffffffffu, v);
        if (v) {
            const ulonglong2 k = src[i];
            const unsigned d = digit_of(k, pass);
            const unsigned same = __match_any_sync(active, d);
            const unsigned base = run[warp][d];
            dst[base + __popc(same & lt)] = k;
            __syncwarp(active);
            if ((same & lt) == 0u) run[warp][d] = base + __popc(same);  // the lowest lane of the group
        }
        __syncwarp();
    }
}

// exclusive scan of a u32 array in place: segment sums, a scan of the sums, segment scans
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned* sh, unsigned& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned s = lane < (blockDim.x >> 5) ? sh[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;  // inclusive warp totals
    }
    __syncthreads();
    total = sh[(blockDim.x >> 5) - 1];
    const unsigned before = warp > 0 ? sh[warp - 1] : 0u;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kScanBlock) scan_sums_kernel(const unsigned* __restrict__ a, long long n,
                                                               unsigned* __restrict__ sums) {
    __shared__ unsigned sh[32];
    const long long base = static_cast<long long>(blockIdx.x) * kScanSeg + threadIdx.x * kScanItems;
    unsigned v = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) v += a[base + k];
    unsigned total;
    block_exclusive_scan(v, sh, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanBlock) scan_top_kernel(unsigned* __restrict__ sums, long long m) {
    __shared__ unsigned sh[32];
    __shared__ unsigned carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long b = 0; b < m; b += kScanBlock) {
        const long long i = b + threadIdx.x;
        const unsigned v = i < m ? sums[i] : 0u;
        unsigned total;
        const unsigned ex = block_exclusive_scan(v, sh, total);
        if (i < m) sums[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[m] = carry;
}

__global__ void __launch_bounds__(kScanBlock) scan_down_kernel(unsigned* __restrict__ a, long long n,
                                                               const unsigned* __restrict__ sums) {
    __shared__ unsigned sh[32];
    const long long base = static_cast<long long>(blockIdx.x) * kScanSeg + threadIdx.x * kScanItems;
    unsigned v[kScanItems], s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? a[base + k] : 0u;
        s += v[k];
    }
    unsigned total;
    unsigned run = sums[blockIdx.x] + block_exclusive_scan(s, sh, total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) {
            a[base + k] = run;
            run += v[k];
        }
}


// KU: head-of-run flags of the sorted keys (as 0/1 in `f`)
__global__ void __launch_bounds__(256) dedup_flags_kernel(const ulonglong2* __restrict__ k, long long n,
                                                          unsigned* __restrict__ f) {
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const ulonglong2 a = k[i];
        bool head = i == 0;
        if (!head) {
            const ulonglong2 b = k[i - 1];
            head = a.x != b.x || a.y != b.y;
        }
        f[i] = head ? 1u : 0u;
    }
}

// KE: after the exclusive scan of the flags, each head writes its key and its position
__global__ void __launch_bounds__(256) dedup_emit_kernel(const ulonglong2* __restrict__ k, long long n,
                                                         const unsigned* __restrict__ pos,
                                                         const unsigned* __restrict__ total_flags,
                                                         ulonglong2* __restrict__ keys_out,
                                                         long long* __restrict__ heads,
                                                         long long* __restrict__ n_unique,
                                                         const unsigned* __restrict__ flag) {
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const ulonglong2 a = k[i];
        bool head = i == 0;
        if (!head) {
            const ulonglong2 b = k[i - 1];
            head = a.x != b.x || a.y != b.y;
        }
        if (head) {
            const unsigned j = pos[i];
            keys_out[j] = a;
            heads[j] = i;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const long long u = static_cast<long long>(*total_flags);
        heads[u] = n;
        *n_unique = (*flag != 0u) ? -1 : u;
    }
}

// KC: multiplicities = differences of consecutive head positions
__global__ void __launch_bounds__(256) dedup_counts_kernel(const long long* __restrict__ heads,
                                                           const unsigned* __restrict__ total_flags,
                                                           long long* __restrict__ counts_out) {
    const long long u = static_cast<long long>(*total_flags);
    for (long long j = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; j < u;
         j += static_cast<long long>(gridDim.x) * blockDim.x)
        counts_out[j] = heads[j + 1] - heads[j];
}

qc_status dfail(qc_status st, const char* msg) {
    qc::set_handleless_error(msg);
    return st;
}

}  // namespace

// Exclusive prefix sum of a u32 array in place (segment sums, a scan of the sums, segment
// scans); also the join index's group starts (qc_join.cu).
cudaError_t qc::exclusive_scan_u32(unsigned* a, long long n, unsigned* sums, cudaStream_t s) {
    const long long segs = (n + kScanSeg - 1) / kScanSeg;
    if (segs == 0) return cudaSuccess;
    scan_sums_kernel<<<static_cast<unsigned>(segs), kScanBlock, 0, s>>>(a, n, sums);
    scan_top_kernel<<<1, kScanBlock, 0, s>>>(sums, segs);
    scan_down_kernel<<<static_cast<unsigned>(segs), kScanBlock, 0, s>>>(a, n, sums);
    return cudaGetLastError();
}

extern "C" int64_t qc_dedup_workspace_bytes(int64_t n_raw) {
    if (n_raw < 0) return -1;
    return static_cast<int64_t>(layout(n_raw).total);
}

extern "C" qc_status qc_dedup(const uint64_t* raw, int64_t n_raw, int n_orb, uint64_t* keys_out,
                              int64_t* counts_out, int64_t* n_unique, void* work, size_t work_bytes,
                              void* stream) {
    if (n_raw < 0 || n_raw > 0x7fffffffLL || n_orb < 1 || n_orb > 128 || !n_unique)
        return dfail(QC_ERR_ARG, "qc_dedup: bad size or NULL n_unique");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n_raw == 0) {
        const cudaError_t e = cudaMemsetAsync(n_unique, 0, sizeof(int64_t), s);
        return e == cudaSuccess ? QC_OK : dfail(QC_ERR_CUDA, cudaGetErrorString(e));
    }
    if (!raw || !keys_out || !counts_out || !work)
        return dfail(QC_ERR_ARG, "qc_dedup: NULL pointer");
    auto mis = [](const void* p, unsigned a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) != 0; };
    if (mis(raw, 16) || mis(keys_out, 16) || mis(counts_out, 8) || mis(n_unique, 8) || mis(work, 256))
        return dfail(QC_ERR_ARG, "qc_dedup: alignment (keys 16, counts 8, work 256 bytes)");
    const long long n = n_raw;
    const Layout L = layout(n);
    if (work_bytes < L.total) return dfail(QC_ERR_CAPACITY, "qc_dedup: workspace too small");
    unsigned char* W = static_cast<unsigned char*>(work);
    ulonglong2* A = reinterpret_cast<ulonglong2*>(W + L.bufA);
    ulonglong2* Bf = reinterpret_cast<ulonglong2*>(W + L.bufB);
    long long* heads = reinterpret_cast<long long*>(W + L.heads);
    unsigned* table = reinterpret_cast<unsigned*>(W + L.table);
    unsigned* sums = reinterpret_cast<unsigned*>(W + L.sums);
    unsigned* flag = reinterpret_cast<unsigned*>(W + L.flag);
    const long long tiles = (n + kTile - 1) / kTile;
    const unsigned blocks = static_cast<unsigned>((tiles + kWarpsPerBlock - 1) / kWarpsPerBlock);
    ulonglong2 high{};
    high.x = n_orb >= 64 ? 0ULL : ~((1ULL << n_orb) - 1ULL);
    high.y = n_orb >= 128 ? 0ULL : (n_orb <= 64 ? ~0ULL : ~((1ULL << (n_orb - 64)) - 1ULL));
    cudaError_t e = cudaMemsetAsync(flag, 0, 16, s);
    const int passes = (n_orb + 7) / 8;
    const ulonglong2* src = reinterpret_cast<const ulonglong2*>(raw);
    ulonglong2* dst = A;
    for (int p = 0; p < passes && e == cudaSuccess; ++p) {
        dedup_hist_kernel<<<blocks, 256, 0, s>>>(src, n, p, tiles, table, high, flag);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = qc::exclusive_scan_u32(table, static_cast<long long>(kBins) * tiles, sums, s);
        if (e == cudaSuccess) {
            dedup_scatter_kernel<<<blocks, 256, 0, s>>>(src, dst, n, p, tiles, table);
            e = cudaGetLastError();
        }
        src = dst;
        dst = (dst == A) ? Bf : A;
    }
    // src holds the sorted keys; the table area holds the flags and their scan
    const unsigned gblocks = static_cast<unsigned>(std::min<long long>((n + 255) / 256, 8192));
    if (e == cudaSuccess) {
        dedup_flags_kernel<<<gblocks, 256, 0, s>>>(src, n, table);
        e = cudaGetLastError();
    }
    const long long segs = (n + kScanSeg - 1) / kScanSeg;
    if (e == cudaSuccess) e = qc::exclusive_scan_u32(table, n, sums, s);
    if (e == cudaSuccess) {
        dedup_emit_kernel<<<gblocks, 256, 0, s>>>(src, n, table, sums + segs, reinterpret_cast<ulonglong2*>(keys_out),
                                                 heads, reinterpret_cast<long long*>(n_unique), flag);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        dedup_counts_kernel<<<gblocks, 256, 0, s>>>(heads, sums + segs, reinterpret_cast<long long*>(counts_out));
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return dfail(QC_ERR_CUDA, cudaGetErrorString(e));
    return QC_OK;
}
