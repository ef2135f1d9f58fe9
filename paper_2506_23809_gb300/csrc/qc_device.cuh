// qc_device.cuh -- device code shared by the sm_103a kernels of libqc_eloc.
//
// The method (arxiv 2506.23809, Sec. III-B, Eq. 5 and Alg. 3): for every unique sample x,
// E_loc(x) = <x|H|x> + sum over single and double excitations x' of x of
// <x|H|x'> psi(x')/psi(x), with H of Eq. 2 and, in sample-space mode, x' restricted to the
// table of unique samples (the lookup table of Sec. IV-C-4).  Alg. 3 spreads the sum as
// processes -> threads -> SIMD lanes; here it is grid -> warp per sample -> lanes over
// excitations.  Its three SIMD devices map as follows:
//   * qubit packing    -> a key is one 128-bit word pair (ulonglong2 loads);
//   * branch elimination -> excitations are enumerated class by class (singles, same-spin
//     and opposite-spin doubles) as products of two short per-sample lists, so no lane
//     ever tests the excitation degree;
//   * SIMD parity      -> the fermionic phase is a sum of four prefix popcounts.
//
// Lookup: every key k has a linear hash H(k) = XOR of T[b] over its set bits b, so the hash
// of x' = x ^ {i, j, a, b} is H(x) ^ T[i] ^ T[j] ^ T[a] ^ T[b] -- four XORs, no key walk.
// The low 32 bits of H index a blocked Bloom filter (two bits in one 32-bit word) that
// every CTA holds in shared memory (loaded by a 1-D bulk async copy); lanes whose x' passes
// are compacted into a per-warp queue and resolved 32 at a time against an open-addressing
// bucket table in global memory (L2 resident), keyed by the high 32 bits of H and
// checked against the stored 128-bit key.  Only then are the matrix element (Slater-Condon)
// and psi(x') read.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "qc_internal.h"
#include "qc_eloc.h"

namespace qc {

#define QC_FULLMASK 0xffffffffu

// Bounds checks of the QC_CHECKED build (a library compiled with -DQC_CHECKED): every integral,
// table and list index goes through QC_IX(i, n, err); out of [0, n) it sets QC_FLAG_BOUNDS in
// *err and yields 0, so the access stays inside the array and nothing traps.  In the normal
// build QC_IX(i, n, err) is i.
#ifdef QC_CHECKED
__device__ __forceinline__ long long checked_index(long long i, long long n, unsigned* err) {
    if (i >= 0 && i < n) return i;
    if (err != nullptr) atomicOr(err, QC_FLAG_BOUNDS);
    return 0;
}
#define QC_IX(i, n, err) (::qc::checked_index(static_cast<long long>(i), static_cast<long long>(n), (err)))
#else
#define QC_IX(i, n, err) (i)
#endif
#define QC_K2(sp) (static_cast<long long>((sp).K) * (sp).K)
#define QC_K3(sp) (QC_K2(sp) * (sp).K)
#define QC_K4(sp) (QC_K2(sp) * QC_K2(sp))

// ------------------------------------------------------------------------------------
// small device helpers
// ------------------------------------------------------------------------------------
// Exclusive prefix parity of a 128-bit occupation: bit k is the parity of the number of
// occupied spin orbitals below k (doubling prefix XOR within each word, then the low
// word's total parity carried into the high word).
__device__ __forceinline__ ulonglong2 prefix_parity(ulonglong2 x) {
    unsigned long long lo = x.x, hi = x.y;
#pragma unroll
    for (int sh = 1; sh < 64; sh <<= 1) {
        lo ^= lo << sh;
        hi ^= hi << sh;
    }
    ulonglong2 p;
    p.x = lo ^ x.x;
    p.y = (hi ^ x.y) ^ ((__popcll(x.x) & 1) ? ~0ULL : 0ULL);
    return p;
}

// Spatial occupation string of one spin (0 alpha, 1 beta) of an interleaved key: bit k is
// spin orbital 2k + spin.
__device__ __forceinline__ unsigned long long gather_even(unsigned long long w) {
    w &= 0x5555555555555555ULL;
    w = (w | (w >> 1)) & 0x3333333333333333ULL;
    w = (w | (w >> 2)) & 0x0F0F0F0F0F0F0F0FULL;
    w = (w | (w >> 4)) & 0x00FF00FF00FF00FFULL;
    w = (w | (w >> 8)) & 0x0000FFFF0000FFFFULL;
    w = (w | (w >> 16)) & 0x00000000FFFFFFFFULL;
    return w;
}
__device__ __forceinline__ unsigned long long spin_string(ulonglong2 k, int spin) {
    return gather_even(k.x >> spin) | (gather_even(k.y >> spin) << 32);
}

__device__ __forceinline__ int pbit(ulonglong2 p, int k) {
    const unsigned long long w = (k < 64) ? p.x : p.y;
    return static_cast<int>((w >> (k & 63)) & 1ULL);
}

__device__ __forceinline__ void flip(ulonglong2& x, int k) {
    const unsigned long long bit = 1ULL << (k & 63);
    x.x ^= (k < 64) ? bit : 0ULL;
    x.y ^= (k < 64) ? 0ULL : bit;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(QC_FULLMASK, v, o);
    return v;
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(QC_FULLMASK, v, o);
    return v;
}
__device__ __forceinline__ unsigned long long warp_xor_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v ^= __shfl_xor_sync(QC_FULLMASK, v, o);
    return v;
}

// Knuth's TwoSum accumulation in FP32: (s, c) holds the running sum and its error.
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
    float t = __fadd_rn(s, x);
    float bp = __fsub_rn(t, s);
    float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    s = t;
    c = __fadd_rn(c, e);
}

// ------------------------------------------------------------------------------------
// mbarrier + 1-D bulk async copy (global -> shared), bounded waits
// ------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

constexpr unsigned kWaitLimit = 1u << 24;  // bounded spin on the filter copy

// ------------------------------------------------------------------------------------
// lookup in the bucket table
// ------------------------------------------------------------------------------------
// Bits of the 64-bit linear key hash H:  the low 32 bits g feed the shared-memory Bloom
// filter (bits 0-4 and 22-31 pick the bits, bits 5.. the word) and are also the bucket
// entry's fingerprint; the home bucket comes from g by multiplicative hashing (its top
// bits after a multiply by an odd constant), so it does not follow the filter word.  A
// random GF(2)-linear map sends any two distinct keys to independent uniform hashes, so
// the bucket load, the fingerprint collisions and the filter false-positive rate are those
// of a 2-universal hash family.  Because every key with fingerprint g has the same home
// bucket, whether some key of the table has fingerprint g does not depend on the order of
// insertion, and a probe by fingerprint alone is deterministic.
__device__ __forceinline__ unsigned home_bucket(unsigned g, unsigned nb_mask) {
    return __umulhi(g * 0x9E3779B1u, nb_mask + 1u);
}

// Returns the table row of key (low hash bits g), or -1.  Buckets hold two 64-bit entries
// (fingerprint << 32 | row + 1); an empty entry ends the probe sequence.  Called only on a
// fingerprint collision (about 0.2% of hits), so it is kept out of line: its loop would
// otherwise sit in the middle of the hit stage's code.
static __device__ __noinline__ long long table_find(const TableParams& tp, ulonglong2 key, unsigned g) {
    unsigned b = home_bucket(g, tp.nb_mask);
    const ulonglong2* buckets = reinterpret_cast<const ulonglong2*>(tp.slots);
    for (unsigned it = 0; it <= tp.nb_mask; ++it) {
        const ulonglong2 e = __ldg(buckets + QC_IX(b, tp.nb_mask + 1LL, tp.err));
        if (e.x == 0ULL) return -1;
        if (static_cast<unsigned>(e.x >> 32) == g) {
            const long long r = static_cast<long long>(static_cast<unsigned>(e.x)) - 1;
            const ulonglong2 k = __ldg(tp.keys + QC_IX(r, tp.n, tp.err));
            if (k.x == key.x && k.y == key.y) return r;
        }
        if (e.y == 0ULL) return -1;
        if (static_cast<unsigned>(e.y >> 32) == g) {
            const long long r = static_cast<long long>(static_cast<unsigned>(e.y)) - 1;
            const ulonglong2 k = __ldg(tp.keys + QC_IX(r, tp.n, tp.err));
            if (k.x == key.x && k.y == key.y) return r;
        }
        b = (b + 1u) & tp.nb_mask;
    }
    return -1;
}

// The first row along the probe sequence of g whose entry carries fingerprint g, or -1 if
// no key of the table has fingerprint g.  Needs only g, not the key: the caller confirms
// the key of the row (table_find resolves the rare 32-bit fingerprint collision).
__device__ __forceinline__ long long probe_fp(unsigned g, const TableParams& tp) {
    unsigned b = home_bucket(g, tp.nb_mask);
    const ulonglong2* buckets = reinterpret_cast<const ulonglong2*>(tp.slots);
    for (unsigned it = 0; it <= tp.nb_mask; ++it) {
        const ulonglong2 e = __ldg(buckets + QC_IX(b, tp.nb_mask + 1LL, tp.err));
        if (e.x == 0ULL) return -1;
        if (static_cast<unsigned>(e.x >> 32) == g) return static_cast<long long>(static_cast<unsigned>(e.x)) - 1;
        if (e.y == 0ULL) return -1;
        if (static_cast<unsigned>(e.y >> 32) == g) return static_cast<long long>(static_cast<unsigned>(e.y)) - 1;
        b = (b + 1u) & tp.nb_mask;
    }
    return -1;
}

// ------------------------------------------------------------------------------------
// K0: table build (hash index + Bloom filter + validation)
// ------------------------------------------------------------------------------------
// Filter bits of a 32-bit hash g: word (g >> 5) & wmask, bits g & 31, (g >> 27) and
// (g >> 22) & 31 of that word.
__device__ __forceinline__ unsigned filter_bits(unsigned g) {
    return (1u << (g & 31u)) | (1u << (g >> 27)) | (1u << ((g >> 22) & 31u));
}

// Insert a spin string into an exact set (open addressing on the high hash bits).  Returns
// the slot that holds it, or kNoSlot when the set is full.
constexpr unsigned kNoSlot = 0xffffffffu;
__device__ __forceinline__ unsigned set_insert(unsigned long long* set, unsigned mask, unsigned long long v,
                                               unsigned long long h) {
    unsigned b = static_cast<unsigned>(h >> 32) & mask;
    for (unsigned it = 0; it <= mask; ++it) {
        const unsigned long long old = atomicCAS(set + b, 0ULL, v);
        if (old == 0ULL || old == v) return b;
        b = (b + 1u) & mask;
    }
    return kNoSlot;
}

// The slot that holds spin string v, or kNoSlot.
__device__ __forceinline__ unsigned set_slot(const unsigned long long* __restrict__ set, unsigned mask,
                                             unsigned long long v, unsigned long long h) {
    unsigned b = static_cast<unsigned>(h >> 32) & mask;
    for (unsigned it = 0; it <= mask; ++it) {
        const unsigned long long e = __ldg(set + (b & mask));
        if (e == v) return b;
        if (e == 0ULL) return kNoSlot;
        b = (b + 1u) & mask;
    }
    return kNoSlot;
}

__device__ __forceinline__ bool set_contains(const unsigned long long* __restrict__ set, unsigned mask,
                                             unsigned long long v, unsigned long long h) {
    return set_slot(set, mask, v, h) != kNoSlot;
}

// Insert row r of the table: validation, filter bits, spin-string sets, bucket entry.  With
// jkey (the sample-space join index), also the row's two set slots as sort keys -- jkey[r]
// jbase + the alpha slot, jkey[n + r] jbase + set size + the beta slot (jsent for a row that
// fails validation) -- their group counts in jlen[key], and with jval the row as the value
// of both (a batch sorts every molecule's keys together, each with its own jbase).
__device__ __forceinline__ void build_one(const TableParams& tp, int n_orb, int na, int nb,
                                          const unsigned long long* __restrict__ T,
                                          unsigned long long* slots, uint32_t* filter,
                                          unsigned long long* aset, unsigned long long* bset,
                                          Counters* ctr, long long r, unsigned* jkey = nullptr,
                                          unsigned* jlen = nullptr, unsigned jbase = 0u, unsigned jsent = 0u,
                                          unsigned* jval = nullptr) {
    const ulonglong2 key = tp.keys[QC_IX(r, tp.n, tp.err)];
    unsigned flags = 0;
    if (r > 0) {
        const ulonglong2 prev = tp.keys[QC_IX(r - 1, tp.n, tp.err)];
        const bool eq = prev.x == key.x && prev.y == key.y;
        const bool gt = (prev.y > key.y) || (prev.y == key.y && prev.x > key.x);
        if (eq) flags |= QC_FLAG_DUP;
        if (gt) flags |= QC_FLAG_UNSORTED;
    }
    const unsigned long long even = 0x5555555555555555ULL;
    const int ea = __popcll(key.x & even) + __popcll(key.y & even);
    const int eb = __popcll(key.x & ~even) + __popcll(key.y & ~even);
    bool high = false;
    if (n_orb < 128) {
        if (n_orb <= 64) high = (key.y != 0ULL) || (n_orb < 64 && (key.x >> n_orb) != 0ULL);
        else high = (key.y >> (n_orb - 64)) != 0ULL;
    }
    if (ea != na || eb != nb || high) flags |= QC_FLAG_NELEC;

    // key hash, and its alpha / beta parts with the spatial strings they belong to
    unsigned long long ha = 0, hb = 0, sa = 0, sb = 0;
    for (unsigned long long w = key.x; w; w &= w - 1ULL) {
        const int bit = __ffsll(w) - 1;
        if (bit & 1) { hb ^= __ldg(T + bit); sb |= 1ULL << (bit >> 1); }
        else { ha ^= __ldg(T + bit); sa |= 1ULL << (bit >> 1); }
    }
    for (unsigned long long w = key.y; w; w &= w - 1ULL) {
        const int bit = __ffsll(w) - 1;
        if (bit & 1) { hb ^= __ldg(T + 64 + bit); sb |= 1ULL << ((64 + bit) >> 1); }
        else { ha ^= __ldg(T + 64 + bit); sa |= 1ULL << ((64 + bit) >> 1); }
    }
    const unsigned long long h = ha ^ hb;

    if (tp.filter != nullptr) {
        const unsigned g = static_cast<unsigned>(h);
        const unsigned wmask = (1u << tp.fw) - 1u;
        atomicOr(filter + ((g >> 5) & wmask), filter_bits(g));
    }
    unsigned slot_a = kNoSlot, slot_b = kNoSlot;
    if (aset != nullptr && sa != 0ULL) slot_a = set_insert(aset, tp.set_mask, sa, ha);
    if (bset != nullptr && sb != 0ULL) slot_b = set_insert(bset, tp.set_mask, sb, hb);
    if (jkey != nullptr) {
        // the join is only built when both spins hold electrons (no string is 0); a row that
        // fails validation joins no group (its keys sort past every group)
        const unsigned size = tp.set_mask + 1u;
        if (slot_a == kNoSlot || slot_b == kNoSlot) flags |= QC_FLAG_TABLE_FULL;
        const bool ok = (flags & QC_FLAG_NELEC) == 0u && slot_a != kNoSlot && slot_b != kNoSlot;
        jkey[r] = ok ? jbase + slot_a : jsent;
        jkey[tp.n + r] = ok ? jbase + size + slot_b : jsent;
        if (jval != nullptr) {
            jval[r] = static_cast<unsigned>(r);
            jval[tp.n + r] = static_cast<unsigned>(r);
        }
        if (ok) {
            atomicAdd(jlen + jbase + slot_a, 1u);
            atomicAdd(jlen + jbase + size + slot_b, 1u);
        }
    }
    const unsigned fp = static_cast<unsigned>(h);
    const unsigned long long entry =
        (static_cast<unsigned long long>(fp) << 32) | static_cast<unsigned long long>(static_cast<unsigned>(r + 1));
    unsigned b = home_bucket(fp, tp.nb_mask);
    bool placed = false;
    for (unsigned it = 0; it <= tp.nb_mask && !placed; ++it) {
        if (atomicCAS(slots + 2 * b, 0ULL, entry) == 0ULL) { placed = true; break; }
        if (atomicCAS(slots + 2 * b + 1, 0ULL, entry) == 0ULL) { placed = true; break; }
        b = (b + 1u) & tp.nb_mask;
    }
    if (!placed) flags |= QC_FLAG_TABLE_FULL;
    if (flags) atomicOr(&ctr->flags, flags);
}



// ------------------------------------------------------------------------------------
// shared-memory layout of the main kernels
// ------------------------------------------------------------------------------------
//   [kOffBar]   mbarrier of the filter copy
//   [kOffT]     T[128]: the linear key hash, 64-bit entries
//   [kOffLut]   colex pair table: p = C(hi, 2) + lo  ->  lo | hi << 8   (p < 2016)
//   [kOffDiv]   single-excitation index -> occupied position, per spin (u8, < 1024 each)
//   [kOffVar]   filter words (filtered kernel only), then one region per warp:
//               occA[64] virA[64] occB[64] virB[64] (u8) | reference-determinant masks (4 x
//               u64) | candidate queue (u32) | hit queue (uint2) | scanned-singles queue
//               (uint2, join only) | hash lists (u32) and single-list maps (u16), filtered only
constexpr size_t kOffBar = 0;
constexpr size_t kOffT = 16;
constexpr size_t kOffLut = kOffT + 128 * 8;
constexpr size_t kOffDiv = kOffLut + kPairLut * 2;
constexpr size_t kOffVar = ((kOffDiv + 2 * 1024 + 127) / 128) * 128;

// Slots of a warp's alpha single list.  Without the join it holds every alpha single that
// passes the spin-string prefilter.  With the sample-space join it holds only the alpha
// singles whose alpha' group is too long to scan (enumerated as classes 0 and 4); the host
// may give it fewer slots than there are alpha singles (acap > 0) when that fits more warps,
// and a sample with more long alpha' groups than slots enumerates them in segments.
__host__ __device__ inline int alpha_slots(const SysParams& sp, int acap) {
    return acap > 0 && acap < sp.nsa ? acap : sp.nsa;
}

// u32 words of a warp's hash lists: the zero entry, the two single lists, then either the
// four pair lists (occupied and empty pairs per spin) or, in the lean layout, only the
// per-orbital values they are built from (a pair's value is the XOR of two of them).
__host__ __device__ inline size_t list_words(const SysParams& sp, bool lean = false, int acap = 0) {
    return static_cast<size_t>(1 + alpha_slots(sp, acap) + sp.nsb) +
           static_cast<size_t>(lean ? sp.oa + sp.va + sp.ob + sp.vb : sp.npoa + sp.npva + sp.npob + sp.npvb);
}


// CTA-wide tables: T, pair LUT, single-excitation division tables
__device__ inline void fill_cta_tables(const SysParams& sp, const unsigned long long* __restrict__ Tg,
                                unsigned char* smem) {
    unsigned long long* T64 = reinterpret_cast<unsigned long long*>(smem + kOffT);
    unsigned short* lut = reinterpret_cast<unsigned short*>(smem + kOffLut);
    unsigned char* divA = smem + kOffDiv;
    unsigned char* divB = divA + 1024;
    for (int t = threadIdx.x; t < 128; t += blockDim.x) T64[t] = Tg[t];
    for (int p = threadIdx.x; p < kPairLut; p += blockDim.x) {
        int hi = static_cast<int>((1.0f + sqrtf(1.0f + 8.0f * static_cast<float>(p))) * 0.5f);
        while (hi * (hi - 1) / 2 > p) --hi;
        while ((hi + 1) * hi / 2 <= p) ++hi;
        const int lo = p - hi * (hi - 1) / 2;
        lut[p] = static_cast<unsigned short>(lo | (hi << 8));
    }
    for (int t = threadIdx.x; t < sp.nsa; t += blockDim.x) divA[t] = static_cast<unsigned char>(t / sp.va);
    for (int t = threadIdx.x; t < sp.nsb; t += blockDim.x) divB[t] = static_cast<unsigned char>(t / sp.vb);
}

// ------------------------------------------------------------------------------------
// accumulators and the three batch stages of candidate resolution
// ------------------------------------------------------------------------------------
struct Acc {
    double re, im;         // FP64 accumulation of sum H psi(x')
    float sr, cr, si, ci;  // FP32 TwoSum accumulation of sum H psi(x')/psi(x)
    unsigned hits;
    unsigned long long rowsum;
    long long signsum;
    unsigned long long missing;
};

// x' = x with spin orbitals (i, j) emptied and (a, b) filled (j = b = 255: a single).
__device__ __forceinline__ ulonglong2 excited_key(unsigned orbs, ulonglong2 x) {
    const int i = orbs & 255u, a = (orbs >> 8) & 255u, j = (orbs >> 16) & 255u, b = orbs >> 24;
    ulonglong2 xp = x;
    flip(xp, i);
    flip(xp, a);
    if (j != 255) {
        flip(xp, j);
        flip(xp, b);
    }
    return xp;
}

// The linear hash of that x', updated from that of x by the four orbitals' entries of T.
__device__ __forceinline__ unsigned long long excited_hash(unsigned orbs, unsigned long long hx,
                                                           const unsigned long long* __restrict__ T64) {
    const int i = orbs & 255u, a = (orbs >> 8) & 255u, j = (orbs >> 16) & 255u, b = orbs >> 24;
    unsigned long long h = hx ^ T64[i] ^ T64[a];
    if (j != 255) h ^= T64[j] ^ T64[b];
    return h;
}

__device__ __forceinline__ ulonglong2 excite(unsigned orbs, ulonglong2 x, unsigned long long hx,
                                             const unsigned long long* __restrict__ T64,
                                             unsigned long long& h) {
    h = excited_hash(orbs, hx, T64);
    return excited_key(orbs, x);
}

// Add one hit: <x|H|x'> (phase included) times psi(x') [FP64], or times psi(x')/psi(x)
// [FP32, compensated], plus (DIAG) the per-sample digests of the exported phase convention.
template <int PREC, bool DIAG>
__device__ __forceinline__ void add_hit(double h64, float h32, long long row, bool sneg, double2 pp,
                                        float2 ip32, Acc& acc) {
    if (PREC == QC_FP64) {
        acc.re = fma(h64, pp.x, acc.re);
        acc.im = fma(h64, pp.y, acc.im);
    } else {
        const float px = static_cast<float>(pp.x), py = static_cast<float>(pp.y);
        const float rr = __fsub_rn(__fmul_rn(px, ip32.x), __fmul_rn(py, ip32.y));
        const float ri = __fadd_rn(__fmul_rn(px, ip32.y), __fmul_rn(py, ip32.x));
        two_sum_acc(acc.sr, acc.cr, __fmul_rn(h32, rr));
        two_sum_acc(acc.si, acc.ci, __fmul_rn(h32, ri));
    }
    acc.hits++;
    if (DIAG) {
        acc.rowsum += static_cast<unsigned long long>(row + 1);
        acc.signsum += sneg ? -(row + 1) : (row + 1);
    }
}

// Stage 2 common part: with the stored key and psi of a stage-1 row already on their way
// (the caller issues those loads before decoding the excitation), let `element` load the
// integrals, then confirm the key (exact walk on a fingerprint collision) and add the hit.
// A row found by the join's scan is exact (its group fixes one spin string and the scan
// compared the other), so its key is not loaded.  Returns phase * (row + 1) of the hit
// added, or 0 when the key is not in the table.
template <int PREC, bool DIAG, typename Element>
__device__ __forceinline__ long long verify_and_add(uint2 e, bool exact, ulonglong2 key, double2 pp, ulonglong2 x,
                                                    unsigned long long hx, const TableParams& tp, int mode,
                                                    const unsigned long long* __restrict__ T64,
                                                    float2 ip32, Acc& acc, Element element) {
    const ulonglong2 xp = excited_key(e.x, x);
    if (exact) key = xp;
    double h64 = 0.0;
    float h32 = 0.f;
    bool sneg = false;
    element(h64, h32, sneg);
    long long row = e.y;
    if (key.x != xp.x || key.y != xp.y) {
        row = table_find(tp, xp, static_cast<unsigned>(excited_hash(e.x, hx, T64)));
        if (row >= 0) pp = __ldg(tp.psi + QC_IX(row, tp.n, tp.err));
        else if (mode == QC_FULL) acc.missing++;
    }
    if (row < 0) return 0;
    add_hit<PREC, DIAG>(h64, h32, row, sneg, pp, ip32, acc);
    return sneg ? -(row + 1) : row + 1;
}

// Pair-by-pair diagnostics: the lanes' hits of one resolution batch (ent: phase * (row + 1),
// 0 for none) go to sample s's list at the positions its cursor hands out, one atomic add
// per batch; a position beyond the list's capacity is not written and is flagged.
__device__ __forceinline__ void list_hits(const EvalParams& ep, long long s, long long ent, int lane) {
    const unsigned m = __ballot_sync(QC_FULLMASK, ent != 0);
    if (m == 0u) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(reinterpret_cast<unsigned long long*>(ep.hit_cursor + s), __popc(m));
    base = __shfl_sync(QC_FULLMASK, base, 0);
    if (ent != 0) {
        const unsigned long long pos = base + static_cast<unsigned long long>(__popc(m & lanemask_lt()));
        if (pos < static_cast<unsigned long long>(ep.hit_list_cap)) ep.hit_list[pos] = ent;
        else atomicOr(&ep.ctr->flags, QC_FLAG_LIST_FULL);
    }
}

// Sample-space join.  Kinds of scanned groups (low bits of a scan descriptor's kind; an
// alpha' or beta' group also carries its excitation ki << 8 | ka << 16, a beta' group in bit 2
// whether x's beta single is taken from it), and the classes of the hits it finds: their codes
// pack four spatial orbitals, 6 bits each.  Odd kinds scan beta strings against x's, even ones
// alpha strings.
constexpr unsigned kScanBetaP = 0u;   // rows of a beta' = single excitation of x's beta string
constexpr unsigned kScanAlpha = 1u;   // rows sharing x's alpha string (beta strings scanned)
constexpr unsigned kScanBeta = 2u;    // rows sharing x's beta string (alpha strings scanned)
constexpr unsigned kScanAlphaP = 3u;  // rows of an alpha' = single excitation of x's alpha string
constexpr unsigned kCodeSingleA = 5u, kCodeSingleB = 6u, kCodeDoubleAA = 7u, kCodeDoubleBB = 8u,
                   kCodeDoubleAB = 9u;
// beta' groups are scanned only for samples with at least this many long alpha' groups
constexpr int kMinLongAlpha = 8;

// Code of a scanned hit: d is the popcount of the scanned string against x's, emptied and
// filled its bits set only in x's string and only in the row's (BETA: beta' groups exist).
template <bool BETA>
__device__ __forceinline__ unsigned scan_code(unsigned kind, int d, unsigned long long emptied,
                                              unsigned long long filled) {
    // the highest bits; at d == 2 the strings differ in one orbital each way, so these are
    // the only ones
    const unsigned e1 = static_cast<unsigned>(63 - __clzll(emptied)) & 63u;
    const unsigned f1 = static_cast<unsigned>(63 - __clzll(filled)) & 63u;
    if ((kind & 3u) == kScanAlphaP) {
        const unsigned ki = (kind >> 8) & 63u, ka = (kind >> 16) & 63u;
        if (d == 0) return (kCodeSingleA << 24) | ki | (ka << 6);
        return (kCodeDoubleAB << 24) | ki | (ka << 6) | (e1 << 12) | (f1 << 18);
    }
    if (BETA && (kind & 3u) == kScanBetaP) {  // the beta orbitals in the kind, the alpha ones scanned
        const unsigned kj = (kind >> 8) & 63u, kb = (kind >> 16) & 63u;
        if (d == 0) return (kCodeSingleB << 24) | kj | (kb << 6);
        return (kCodeDoubleAB << 24) | e1 | (f1 << 6) | (kj << 12) | (kb << 18);
    }
    if (d == 2) return (kCodeSingleB << 24) | e1 | (f1 << 6);  // x's alpha group only
    const unsigned e0 = static_cast<unsigned>(__ffsll(emptied) - 1) & 63u;
    const unsigned f0 = static_cast<unsigned>(__ffsll(filled) - 1) & 63u;
    const unsigned cls = (kind & 3u) == kScanAlpha ? kCodeDoubleBB : kCodeDoubleAA;
    return (cls << 24) | e0 | (e1 << 6) | (f0 << 12) | (f1 << 18);
}

// Stage 1 -- decode a candidate (class, u, w) into the spin orbitals it empties (i, j)
// and fills (a, b); j = b = 255 for singles.  Classes: 0 alpha single (w), 1 beta single
// (w), 2 alpha-alpha double (u: occupied pair, w: empty pair), 3 beta-beta double,
// 4 alpha-beta double (u: alpha single, w: beta single), and the classes of scanned hits
// (kCodeSingleA ..).  Same-spin doubles come out with i < j and a < b.  Single indices go
// through IA / IB (the compacted single lists of the filtered kernel) when given.  Returns the packed orbitals i | a << 8 | j << 16 | b << 24.
__device__ __forceinline__ unsigned decode(unsigned code, const SysParams& sp,
                                           const unsigned char* __restrict__ wl,
                                           const unsigned char* __restrict__ smem,
                                           const unsigned short* __restrict__ IA,
                                           const unsigned short* __restrict__ IB) {
    const unsigned short* lut = reinterpret_cast<const unsigned short*>(smem + kOffLut);
    const unsigned char* divA = smem + kOffDiv;
    const unsigned char* divB = divA + 1024;
    const unsigned char* occA = wl;
    const unsigned char* virA = wl + 64;
    const unsigned char* occB = wl + 128;
    const unsigned char* virB = wl + 192;
    const unsigned cls = code >> 24;
    if (cls >= kCodeSingleA) {  // a scanned hit: spatial orbitals in the code
        const unsigned k0 = code & 63u, k1 = (code >> 6) & 63u, k2 = (code >> 12) & 63u, k3 = (code >> 18) & 63u;
        if (cls <= kCodeSingleB) {
            const unsigned sb = cls - kCodeSingleA;
            return (2u * k0 + sb) | ((2u * k1 + sb) << 8) | 0xFFFF0000u;
        }
        if (cls == kCodeDoubleAB) return (2u * k0) | ((2u * k1) << 8) | ((2u * k2 + 1u) << 16) | ((2u * k3 + 1u) << 24);
        const unsigned sb = cls - kCodeDoubleAA;
        return (2u * k0 + sb) | ((2u * k2 + sb) << 8) | ((2u * k1 + sb) << 16) | ((2u * k3 + sb) << 24);
    }
    const int u = static_cast<int>((code >> 12) & 4095u);
    const int w = static_cast<int>(code & 4095u);
    // the filtered kernel's single lists are compacted by the spin-string prefilter; their maps
    // IA / IB hold each entry's spatial orbitals (occupied | empty << 8)
    if (IA != nullptr && (cls <= 1u || cls == 4u)) {
        if (cls == 4u) {
            const unsigned pa = IA[QC_IX(u, sp.nsa, sp.err)], pb = IB[QC_IX(w, sp.nsb, sp.err)];
            return (2u * (pa & 255u)) | ((2u * (pa >> 8)) << 8) | ((2u * (pb & 255u) + 1u) << 16) |
                   ((2u * (pb >> 8) + 1u) << 24);
        }
        const unsigned p = cls == 0u ? IA[QC_IX(w, sp.nsa, sp.err)] : IB[QC_IX(w, sp.nsb, sp.err)];
        return (2u * (p & 255u) + cls) | ((2u * (p >> 8) + cls) << 8) | 0xFFFF0000u;
    }
    unsigned i, a, j = 255u, b = 255u;
    if (cls == 4u) {
        const int io = divA[QC_IX(u, sp.nsa, sp.err)], jo = divB[QC_IX(w, sp.nsb, sp.err)];
        i = 2u * occA[QC_IX(io, sp.oa, sp.err)];
        a = 2u * virA[QC_IX(u - io * sp.va, sp.va, sp.err)];
        j = 2u * occB[QC_IX(jo, sp.ob, sp.err)] + 1u;
        b = 2u * virB[QC_IX(w - jo * sp.vb, sp.vb, sp.err)] + 1u;
    } else if (cls >= 2u) {
        const unsigned po = lut[QC_IX(u, cls == 2u ? sp.npoa : sp.npob, sp.err)];
        const unsigned pv = lut[QC_IX(w, cls == 2u ? sp.npva : sp.npvb, sp.err)];
        const unsigned char* occ = cls == 2u ? occA : occB;
        const unsigned char* vir = cls == 2u ? virA : virB;
        const unsigned s = cls - 2u;
        i = 2u * occ[po & 255u] + s;
        j = 2u * occ[po >> 8] + s;
        a = 2u * vir[pv & 255u] + s;
        b = 2u * vir[pv >> 8] + s;
    } else {
        const unsigned char* dv = cls == 0u ? divA : divB;
        const unsigned char* occ = cls == 0u ? occA : occB;
        const unsigned char* vir = cls == 0u ? virA : virB;
        const int vv = cls == 0u ? sp.va : sp.vb;
        const int io = dv[QC_IX(w, cls == 0u ? sp.nsa : sp.nsb, sp.err)];
        i = 2u * occ[QC_IX(io, cls == 0u ? sp.oa : sp.ob, sp.err)] + cls;
        a = 2u * vir[QC_IX(w - io * vv, vv, sp.err)] + cls;
    }
    return i | (a << 8) | (j << 16) | (b << 24);
}

// x or -x, by flipping the sign bit with an integer operation (the FP64 pipe, 1/64 of the
// FP32 rate on this GPU, is kept for the arithmetic that needs it)
__device__ __forceinline__ double with_sign(double v, bool neg) {
    return __hiloint2double(__double2hiint(v) ^ (neg ? static_cast<int>(0x80000000u) : 0), __double2loint(v));
}
__device__ __forceinline__ float with_sign(float v, bool neg) {
    return __int_as_float(__float_as_int(v) ^ (neg ? static_cast<int>(0x80000000u) : 0));
}

// Stage 2 -- single i -> a (Slater-Condon): h_ai + sum_{k occ} (ai|kk) - sum_{k occ, same
// spin} (ak|ki), phase <x'| a+_a a_i |x> = (-1)^{P(i) + P(a) + [i < a]}, P = occupied below
// (read from the prefix-parity mask px).
template <int PREC>
__device__ __forceinline__ void single_element(unsigned orbs, ulonglong2 px, const SysParams& sp,
                                               const unsigned char* __restrict__ wl,
                                               const unsigned long long* __restrict__ dref, double& h64,
                                               float& h32, bool& sneg) {
    const int i = orbs & 255u, a = (orbs >> 8) & 255u;
    const int K = sp.K, ki = i >> 1, ka = a >> 1, s = i & 1;
    // K <= 64: every integral index fits 32 bits (K^4 <= 2^24)
    const unsigned rowk = QC_IX((static_cast<unsigned>(ka) * K + ki) * K, QC_K3(sp) - K + 1, sp.err);
    const unsigned char* occA = wl;
    const unsigned char* occB = wl + 128;
    const bool neg = (pbit(px, i) ^ pbit(px, a) ^ (i < a ? 1 : 0)) != 0;
    if (PREC == QC_FP64) {
        const double* jt = sp.Jt + rowk;
        const double* xt = sp.Xt + rowk;
        const int os = s == 0 ? sp.oa : sp.ob;
        // x differs from the reference determinant in a few orbitals (dref: the spatial
        // orbitals x fills and empties against it, alpha then beta): start from the
        // reference's sum and correct by those, when that is the shorter sum (the same for
        // every lane of a batch: one sample)
        unsigned long long aP = 0, aM = 0, bP = 0, bM = 0;
        int nd = 1 << 30;
        if (dref != nullptr) {
            aP = dref[0];
            aM = dref[1];
            bP = dref[2];
            bM = dref[3];
            nd = __popcll(aP | bP) + __popcll(aM | bM) + __popcll(s ? bP : aP) + __popcll(s ? bM : aM);
        }
        double f;
        if (nd < sp.oa + sp.ob + os) {
            double f0 = sp.Fref[QC_IX((static_cast<unsigned>(s) * K + ka) * K + ki, 2 * QC_K2(sp), sp.err)], f1 = 0.0,
                   f2 = 0.0, f3 = 0.0;
            for (unsigned long long m = aP | bP; m; m &= m - 1ULL) {
                const int k = __ffsll(m) - 1;
                f1 += ((aP >> k) & (bP >> k) & 1ULL) ? 2.0 * jt[k] : jt[k];
            }
            for (unsigned long long m = aM | bM; m; m &= m - 1ULL) {
                const int k = __ffsll(m) - 1;
                f2 -= ((aM >> k) & (bM >> k) & 1ULL) ? 2.0 * jt[k] : jt[k];
            }
            for (unsigned long long m = s ? bP : aP; m; m &= m - 1ULL) f3 -= xt[__ffsll(m) - 1];
            for (unsigned long long m = s ? bM : aM; m; m &= m - 1ULL) f0 += xt[__ffsll(m) - 1];
            f = (f0 + f3) + (f1 + f2);
        } else {
            // sum over the occupied orbitals of both spins, four independent partial sums
            double f0 = sp.h[QC_IX(ka * K + ki, QC_K2(sp), sp.err)], f1 = 0.0, f2 = 0.0, f3 = 0.0;
            const unsigned char* occS = s == 0 ? occA : occB;
            int q = 0;
            for (; q + 1 < sp.oa; q += 2) { f0 += jt[occA[q]]; f1 += jt[occA[q + 1]]; }
            if (q < sp.oa) f0 += jt[occA[q]];
            for (q = 0; q + 1 < sp.ob; q += 2) { f2 += jt[occB[q]]; f3 += jt[occB[q + 1]]; }
            if (q < sp.ob) f2 += jt[occB[q]];
            double g0 = 0.0, g1 = 0.0;
            for (q = 0; q + 1 < os; q += 2) { g0 += xt[occS[q]]; g1 += xt[occS[q + 1]]; }
            if (q < os) g0 += xt[occS[q]];
            f = ((f0 + f1) + (f2 + f3)) - (g0 + g1);
        }
        h64 = with_sign(f, neg);
    } else {
        float f0 = sp.h32[QC_IX(ka * K + ki, QC_K2(sp), sp.err)], f1 = 0.f, f2 = 0.f, f3 = 0.f;
        const float* jt = sp.Jt32 + rowk;
        const float* xt = sp.Xt32 + rowk;
        const unsigned char* occS = s == 0 ? occA : occB;
        const int os = s == 0 ? sp.oa : sp.ob;
        int q = 0;
        for (; q + 1 < sp.oa; q += 2) { f0 += jt[occA[q]]; f1 += jt[occA[q + 1]]; }
        if (q < sp.oa) f0 += jt[occA[q]];
        for (q = 0; q + 1 < sp.ob; q += 2) { f2 += jt[occB[q]]; f3 += jt[occB[q + 1]]; }
        if (q < sp.ob) f2 += jt[occB[q]];
        float g0 = 0.f, g1 = 0.f;
        for (q = 0; q + 1 < os; q += 2) { g0 += xt[occS[q]]; g1 += xt[occS[q + 1]]; }
        if (q < os) g0 += xt[occS[q]];
        const float f = ((f0 + f1) + (f2 + f3)) - (g0 + g1);
        h32 = with_sign(f, neg);
    }
    sneg = neg;
}

// Stage 2 -- double (i, j) -> (a, b): <ab||ij> = (ai|bj) - (aj|bi) for equal spins,
// (ai|bj) for alpha i, a and beta j, b; phase <x'| a+_a a+_b a_j a_i |x> =
// (-1)^{P(i)+P(j)+P(a)+P(b) + [i<j]+[i<b]+[j<b]+[i<a]+[j<a]+[b<a]}.
template <int PREC>
__device__ __forceinline__ void double_element(unsigned orbs, ulonglong2 px, const SysParams& sp,
                                               double& h64, float& h32, bool& sneg) {
    const int i = orbs & 255u, a = (orbs >> 8) & 255u, j = (orbs >> 16) & 255u, b = orbs >> 24;
    const int K = sp.K, ki = i >> 1, ka = a >> 1, kj = j >> 1, kb = b >> 1;
    // K <= 64: the index fits 32 bits (K^4 <= 2^24)
    const unsigned d = QC_IX(((static_cast<unsigned>(ka) * K + ki) * K + kb) * K + kj, QC_K4(sp), sp.err);  // (ai|bj)
    const int par = (pbit(px, i) ^ pbit(px, j) ^ pbit(px, a) ^ pbit(px, b)) + (i < j) + (i < b) +
                    (j < b) + (i < a) + (j < a) + (b < a);
    const bool neg = (par & 1) != 0;
    const bool same = (i & 1) == (j & 1);
    if (PREC == QC_FP64) {
        double e = sp.eri[d];
        if (same) e -= sp.eri[QC_IX(((static_cast<unsigned>(ka) * K + kj) * K + kb) * K + ki, QC_K4(sp), sp.err)];  // (aj|bi)
        h64 = with_sign(e, neg);
    } else {
        float e = sp.eri32[d];
        if (same) e -= sp.eri32[QC_IX(((static_cast<unsigned>(ka) * K + kj) * K + kb) * K + ki, QC_K4(sp), sp.err)];
        h32 = with_sign(e, neg);
    }
    // exported convention sorts the emptied and the filled pair
    sneg = neg != ((((i > j) ? 1 : 0) + ((a > b) ? 1 : 0)) & 1);
}

// Per-sample set-up shared by both main kernels.  Returns false when x does not hold
// na alpha and nb beta electrons below n_orb (then nothing is written to the lists).
__device__ __forceinline__ bool sample_setup(const SysParams& sp, ulonglong2 x, int lane,
                                             unsigned char* wl,
                                             const unsigned long long* __restrict__ T64,
                                             unsigned long long& hx, double& ediag,
                                             unsigned long long& As, unsigned long long& Bs,
                                             unsigned long long& hxa) {
    unsigned char* occA = wl;
    unsigned char* virA = wl + 64;
    unsigned char* occB = wl + 128;
    unsigned char* virB = wl + 192;
    const unsigned long long even = 0x5555555555555555ULL;
    const int ea = __popcll(x.x & even) + __popcll(x.y & even);
    const int eb = __popcll(x.x & ~even) + __popcll(x.y & ~even);
    bool high = false;
    if (sp.n_orb < 128) {
        if (sp.n_orb <= 64) high = (x.y != 0ULL) || (sp.n_orb < 64 && (x.x >> sp.n_orb) != 0ULL);
        else high = (x.y >> (sp.n_orb - 64)) != 0ULL;
    }
    if (ea != sp.na || eb != sp.nb || high) return false;
    // spatial occupation strings: lane l owns spatial orbitals l and l + 32
    const unsigned alo = __ballot_sync(QC_FULLMASK, (x.x >> (2 * lane)) & 1ULL);
    const unsigned ahi = __ballot_sync(QC_FULLMASK, (x.y >> (2 * lane)) & 1ULL);
    const unsigned blo = __ballot_sync(QC_FULLMASK, (x.x >> (2 * lane + 1)) & 1ULL);
    const unsigned bhi = __ballot_sync(QC_FULLMASK, (x.y >> (2 * lane + 1)) & 1ULL);
    const unsigned long long A = static_cast<unsigned long long>(alo) |
                                 (static_cast<unsigned long long>(ahi) << 32);
    const unsigned long long B = static_cast<unsigned long long>(blo) |
                                 (static_cast<unsigned long long>(bhi) << 32);
    for (int k = lane; k < sp.K; k += 32) {
        const unsigned long long lowm = (1ULL << k) - 1ULL;
        const int ca = __popcll(A & lowm), cb = __popcll(B & lowm);
        if ((A >> k) & 1ULL) occA[QC_IX(ca, 64, sp.err)] = static_cast<unsigned char>(k);
        else virA[QC_IX(k - ca, 64, sp.err)] = static_cast<unsigned char>(k);
        if ((B >> k) & 1ULL) occB[QC_IX(cb, 64, sp.err)] = static_cast<unsigned char>(k);
        else virB[QC_IX(k - cb, 64, sp.err)] = static_cast<unsigned char>(k);
    }
    // linear hash of x: XOR of T over set bits (lane l: bits l, l+32, l+64, l+96)
    unsigned long long hv = 0;
    if ((x.x >> lane) & 1ULL) hv ^= T64[lane];
    if ((x.x >> (lane + 32)) & 1ULL) hv ^= T64[lane + 32];
    if ((x.y >> lane) & 1ULL) hv ^= T64[lane + 64];
    if ((x.y >> (lane + 32)) & 1ULL) hv ^= T64[lane + 96];
    hx = warp_xor_u64(hv);
    hxa = warp_xor_u64((lane & 1) ? 0ULL : hv);  // even spin orbitals: the alpha part
    As = A;
    Bs = B;
    __syncwarp();
    // diagonal: sum_p h_pp + 1/2 sum_{p,q occ} [(pp|qq) - d(sp,sq) (pq|qp)]  (FP64).  The
    // n_occ^2 ordered pairs of occupied spatial orbitals (positions 0 .. oa - 1 alpha, then
    // beta) are spread over the 32 lanes, one load and one add each: X holds the same-spin
    // term (kk|ll) - (kl|lk), J the other (for p = q the same-spin term is 0)
    const int K = sp.K;
    const int no = sp.oa + sp.ob;
    double e0 = 0.0, e1 = 0.0;
    for (int p = lane; p < no; p += 32) {
        const int k = p < sp.oa ? occA[p] : occB[p - sp.oa];
        e1 += sp.h[QC_IX(k * K + k, QC_K2(sp), sp.err)];
    }
    if (no > 0) {
        const int q32 = 32 / no, r32 = 32 - q32 * no;
        int p = lane / no, r = lane - (lane / no) * no;
        for (int t = lane; t < no * no; t += 32) {
            const bool pa = p < sp.oa, ra = r < sp.oa;
            const int k = pa ? occA[p] : occB[p - sp.oa];
            const int l = ra ? occA[r] : occB[r - sp.oa];
            e0 += (pa == ra ? sp.X : sp.J)[QC_IX(k * K + l, QC_K2(sp), sp.err)];
            r += r32;
            p += q32;
            if (r >= no) {
                r -= no;
                ++p;
            }
        }
    }
    ediag = warp_sum(fma(0.5, e0, e1)) + sp.e_core;
    return true;
}

// Lane 0's part of a sample's finish: E_loc from the warp sums and the outputs.
template <int PREC>
__device__ __forceinline__ void write_sample(const EvalParams& ep, long long s, double ediag, double2 psix,
                                             double sre, double sim, unsigned long long hits,
                                             unsigned long long rows, long long sgn, unsigned long long miss) {
    double2 e;
    const double n2 = psix.x * psix.x + psix.y * psix.y;
    unsigned flags = 0;
    bool bad = false;
    if (n2 == 0.0) {
        flags |= QC_FLAG_ZERO_PSI;
        bad = true;
    }
    if (miss) {
        flags |= QC_FLAG_MISSING;
        bad = true;
    }
    if (bad) {
        e.x = __longlong_as_double(0x7ff8000000000000LL);
        e.y = e.x;
    } else if (PREC == QC_FP64) {
        // sum H psi(x') / psi(x) = S conj(psi) / |psi|^2
        const double inv = 1.0 / n2;
        e.x = ediag + (sre * psix.x + sim * psix.y) * inv;
        e.y = (sim * psix.x - sre * psix.y) * inv;
    } else {
        e.x = ediag + sre;
        e.y = sim;
    }
    ep.eloc[QC_IX(s, ep.n_u, &ep.ctr->flags)] = e;
    if (ep.hit_count) ep.hit_count[s] = static_cast<uint32_t>(hits);
    if (ep.hit_rowsum) ep.hit_rowsum[s] = rows;
    if (ep.hit_signsum) ep.hit_signsum[s] = sgn;
    if (hits) atomicAdd(&ep.ctr->hits, hits);
    if (miss) atomicAdd(&ep.ctr->missing, miss);
    if (bad) atomicAdd(&ep.ctr->bad, 1ULL);
    if (flags) atomicOr(&ep.ctr->flags, flags);
}

// Per-sample finish: reduce the lane accumulators and write the outputs.  With several
// excitation chunks per sample (C > 1) each chunk stores its warp sums; the warp that
// finishes the last chunk of the sample adds the C records in chunk order (the result does
// not depend on which warp finishes last) and writes the outputs.
template <int PREC, bool DIAG, bool FILTER>
__device__ __forceinline__ void sample_finish(const EvalParams& ep, long long s, int lane,
                                              double ediag, double2 psix, Acc& acc, int c = 0, int C = 1) {
    double sre, sim;
    if (PREC == QC_FP64) {
        sre = warp_sum(acc.re);
        sim = warp_sum(acc.im);
    } else {
        sre = warp_sum(static_cast<double>(acc.sr) + static_cast<double>(acc.cr));
        sim = warp_sum(static_cast<double>(acc.si) + static_cast<double>(acc.ci));
    }
    const unsigned long long hits = __reduce_add_sync(QC_FULLMASK, acc.hits);
    // the digests exist in the diagnostic kernels only; missing x' only without the filter
    // (the accurate-energy kernel)
    const unsigned long long rows = DIAG ? warp_sum_u64(acc.rowsum) : 0ULL;
    const long long sgn = DIAG ? static_cast<long long>(warp_sum_u64(static_cast<unsigned long long>(acc.signsum))) : 0LL;
    const unsigned long long miss = FILTER ? 0ULL : warp_sum_u64(acc.missing);
    if (lane != 0) return;
    if (C <= 1) {
        write_sample<PREC>(ep, s, ediag, psix, sre, sim, hits, rows, sgn, miss);
        return;
    }
    ChunkRec* rec = static_cast<ChunkRec*>(ep.cpart) + s * C;
    ChunkRec mine;
    mine.re = sre;
    mine.im = sim;
    mine.hits = hits;
    mine.rowsum = rows;
    mine.signsum = sgn;
    mine.missing = miss;
    rec[c] = mine;
    __threadfence();
    if (atomicAdd(ep.cticket + s, 1u) != static_cast<unsigned>(C - 1)) return;
    __threadfence();
    double re = 0.0, im = 0.0;
    unsigned long long th = 0, tr = 0, tm = 0;
    long long ts = 0;
    for (int k = 0; k < C; ++k) {
        const volatile ChunkRec* r = rec + k;
        re += r->re;
        im += r->im;
        th += r->hits;
        tr += r->rowsum;
        ts += r->signsum;
        tm += r->missing;
    }
    write_sample<PREC>(ep, s, ediag, psix, re, im, th, tr, ts, tm);
}

static __device__ __noinline__ void invalid_sample(const EvalParams& ep, long long s, int lane) {
    if (lane == 0) {
        double2 e;
        e.x = __longlong_as_double(0x7ff8000000000000LL);
        e.y = e.x;
        ep.eloc[s] = e;
        if (ep.hit_count) ep.hit_count[s] = 0;
        if (ep.hit_rowsum) ep.hit_rowsum[s] = 0;
        if (ep.hit_signsum) ep.hit_signsum[s] = 0;
        atomicAdd(&ep.ctr->bad, 1ULL);
        atomicAdd(&ep.ctr->invalid, 1ULL);
        atomicOr(&ep.ctr->flags, QC_FLAG_NELEC);
    }
}

__device__ __forceinline__ float2 inv_psi32(double2 p) {
    const double n2 = p.x * p.x + p.y * p.y;
    const double inv = n2 > 0.0 ? 1.0 / n2 : 0.0;
    return make_float2(static_cast<float>(p.x * inv), static_cast<float>(-p.y * inv));
}

// ------------------------------------------------------------------------------------
// K2: the local-energy kernel
// ------------------------------------------------------------------------------------
// One warp per sample (persistent grid).  The five excitation classes are walked as
// outer x inner products of per-sample hash lists by a flat state machine; each step
// tests U x 32 excitations.  With FILTER, an excitation becomes a candidate only if its
// three bits are set in the shared-memory Bloom filter; without it (accurate-energy mode,
// or the unfiltered variant) every excitation is a candidate.  Candidates queue up per
// warp and are resolved 32 at a time in two full-warp stages: probe the bucket table by
// the candidate's fingerprint (its low hash bits, rebuilt from two list entries, so most
// filter false positives are rejected without decoding the excitation), then decode the
// hits, confirm their keys and compute their matrix elements.  Both stages sit at one
// place in the loop; the end of a sample flushes the partial batches through the same code.
constexpr int kCandCap = 160;  // >= 31 + 32 * 4 (the largest U with a single flush site)
constexpr size_t kWarpQueues = 4 * kCandCap + 64 * 8;  // candidate queue + hit queue

constexpr int kSingleCap = 64;  // join: the hit queue of scanned singles (uint2)
// The current sample's constants, kept in the warp's shared memory rather than registers (the
// main loop reads them only in its hit and finish stages).
struct WarpSample {
    ulonglong2 x;             // the sample
    ulonglong2 px;            // prefix parity of x (the phases of its excitations)
    double2 psix;             // psi(x)
    unsigned long long hx;    // linear hash of x
    double ediag;             // <x|H|x>
    float2 ip32;              // 1/psi(x) in FP32 (precision form)
    unsigned long long as, bs, hxa;  // join: x's alpha and beta spatial strings, alpha part of hx
    unsigned a_next;          // join: first alpha single not yet in an alpha-list segment
    unsigned a_seen;          // join: alpha singles below this were classified (short groups scanned)
    unsigned athr;            // join, segments: an alpha' group is long when its len exceeds this
    unsigned pad;
};
constexpr size_t kOffWarpSample = 288;
// per warp: occupation lists (4 x 64 B), reference masks (32 B), the sample's constants
constexpr size_t kOccBytes = kOffWarpSample + sizeof(WarpSample);
static_assert(kOccBytes % 16 == 0, "warp regions stay 16-byte aligned");
// join: the kernel has the join's queue of scanned singles; acap: the alpha list's slots
// (alpha_slots; 0 for all)
__host__ __device__ inline size_t main_warp_bytes(const SysParams& sp, bool filter, bool lean = false,
                                                  bool join = false, int acap = 0) {
    // hash lists (u32) and, for the two single lists, their compaction maps (u16)
    const size_t lists = filter ? 4 * list_words(sp, lean, acap) +
                                      2 * static_cast<size_t>(alpha_slots(sp, acap) + sp.nsb)
                                : 0;
    return (kOccBytes + kWarpQueues + (join ? 8 * kSingleCap : 0) + lists + 15) / 16 * 16;
}



// One sample, one warp: set-up, the filtered (or unfiltered) walk over its excitations,
// resolution of the candidates and the per-sample outputs.  wl is the warp's region of
// shared memory, filt the CTA's copy of the Bloom filter.  LEAN: 0 the pair lists are
// stored, 1 they are formed on the fly from per-orbital values (less shared memory per
// warp, so more warps fit for large orbital counts), 2 as ep.lean says.  Both layouts give
// the same hash values in the same order, so the same results.  JOIN: the sample-space join
// is taken when the table carries its index (false compiles it out).  DIAG: the pair-by-pair
// hit lists and the work counters are written when the launch asks for them (false compiles
// them out: the checks alone cost the timed kernel a third of its speed).  SEG: the join's
// alpha list may have fewer slots than alpha singles (tp.alpha_cap) and is then enumerated in
// segments (false compiles the segments out: 2% of the kernel's time when no list is capped).
// BETA: the join's beta' phase (with SEG only, and run only when the alpha list is capped, as
// in the single-molecule kernel with segments; false compiles it out: compiled into the kernel
// without segments, it made that kernel 5% slower at 52 spin orbitals with the phase switched
// off, more than the phase saved there with it on).
template <int PREC, int U, bool FILTER, int LEAN, bool JOIN = true, bool DIAG = false, bool SEG = false,
          bool BETA = false>
__device__ __forceinline__ void run_sample(const SysParams& sp, const TableParams& tp,
                                           const EvalParams& ep, long long s, int lane,
                                           unsigned char* smem, unsigned char* wl,
                                           const uint32_t* filt, int c = 0, int C = 1) {
    static_assert(!BETA || (JOIN && SEG), "the beta' phase runs in the join kernels with segments");
    const unsigned long long* T64 = reinterpret_cast<const unsigned long long*>(smem + kOffT);
    const unsigned short* lut = reinterpret_cast<const unsigned short*>(smem + kOffLut);
    uint32_t* q = reinterpret_cast<uint32_t*>(wl + kOccBytes);
    uint2* hq = reinterpret_cast<uint2*>(wl + kOccBytes + 4 * kCandCap);
    uint2* hs = hq + 64;  // join kernels only: scanned singles
    uint32_t* H = reinterpret_cast<uint32_t*>(wl + kOccBytes + kWarpQueues + (JOIN ? 8 * kSingleCap : 0));
    // the FP64 singles' differences against the reference determinant (set after set-up)
    unsigned long long* dref = (PREC == QC_FP64 && sp.Fref != nullptr)
                                   ? reinterpret_cast<unsigned long long*>(wl + 256) : nullptr;
    const bool lean = FILTER && (LEAN == 1 || (LEAN == 2 && ep.lean != 0));
    // list offsets inside H: 0 zero | SA | SB | PAo | PAv | PBo | PBv, or in the lean layout
    // 0 zero | SA | SB | occupied alpha | empty alpha | occupied beta | empty beta; with the
    // join the alpha list may have fewer slots (tp.alpha_cap), filled in segments
    const bool join_lists = JOIN && FILTER && tp.jlen != nullptr;
    const int nA = alpha_slots(sp, SEG && join_lists ? tp.alpha_cap : 0);
    const int oSA = 1, oSB = oSA + nA, oPAo = oSB + sp.nsb;
    const int oPAv = oPAo + (lean ? sp.oa : sp.npoa);
    const int oPBo = oPAv + (lean ? sp.va : sp.npva);
    const int oPBv = oPBo + (lean ? sp.ob : sp.npob);
    unsigned short* IA =
        FILTER ? reinterpret_cast<unsigned short*>(H + list_words(sp, lean, SEG && join_lists ? tp.alpha_cap : 0))
               : nullptr;
    unsigned short* IB = FILTER ? IA + nA : nullptr;
    const int nH = FILTER ? static_cast<int>(list_words(sp, lean, SEG && join_lists ? tp.alpha_cap : 0)) : 0;
    (void)nH;  // the list's length, for the checked build's bounds checks
    int nsa2 = sp.nsa, nsb2 = sp.nsb;  // single-list lengths after the spin-string prefilter
    const uint32_t wmask4 = FILTER ? ((1u << tp.fw) - 1u) << 2 : 0u;
    const unsigned ltmask = lanemask_lt();
    const unsigned char* divA = smem + kOffDiv;
    const unsigned char* divB = divA + 1024;


    const ulonglong2 x = ep.samples[QC_IX(s, ep.n_u, sp.err)];
    unsigned long long hx, As, Bs, hxa;
    double ediag;
    if (!sample_setup(sp, x, lane, wl, T64, hx, ediag, As, Bs, hxa)) {
        if (c == 0) invalid_sample(ep, s, lane);  // reported once, by the first chunk
        return;
    }
    if (DIAG && ep.work != nullptr && lane == 0 && c == 0) atomicAdd(&ep.work->samples, 1ULL);
    if (dref != nullptr && lane == 0) {
        dref[0] = As & ~sp.refA;
        dref[1] = sp.refA & ~As;
        dref[2] = Bs & ~sp.refB;
        dref[3] = sp.refB & ~Bs;
    }
    // the sample's constants go to the warp's shared memory: the hit and finish stages read
    // them there, so the enumeration and scan states keep their registers
    WarpSample* wsp = reinterpret_cast<WarpSample*>(wl + kOffWarpSample);
    if (lane == 0) {
        WarpSample w;
        w.x = x;
        w.px = prefix_parity(x);
        w.psix = ep.psi[QC_IX(s, ep.n_u, sp.err)];
        w.hx = hx;
        w.ediag = ediag;
        w.ip32 = PREC == QC_FP64 ? make_float2(0.f, 0.f) : inv_psi32(w.psix);
        w.as = As;
        w.bs = Bs;
        w.hxa = hxa;
        w.a_next = 0u;
        w.a_seen = 0u;
        w.athr = 0u;
        w.pad = 0u;
        *wsp = w;
    }
    __syncwarp();
    Acc acc{};
    int qn = 0, nh = 0;
    // sample-space join: short groups of table rows are scanned (the scan state, first phase
    // of the main loop; chunk 0 only), the excitations into long ones enumerated (classes 1 and
    // 3 only when x's alpha group is long, class 2 only when its beta group is, classes 0 and 4
    // only over long alpha' groups)
    const bool join = JOIN && FILTER && tp.jlen != nullptr;
    bool enumA = true, enumB = true;

    // hits: 32 from a hit queue -- decode, key check, psi(x') and integrals, then the
    // element.  Singles come in their own classes (and, from the join's scans, in their own
    // queue), so a batch rarely mixes the kinds.
    int ns = 0;  // join: scanned singles queued in hs
    auto hit_batch = [&](uint2* Q, int& nq) {
        const int n = nq < 32 ? nq : 32;
        const bool v = lane < n;
        uint2 e = v ? Q[lane] : make_uint2(0u, 0u);
        __syncwarp();
        if (lane < nq - n) Q[lane] = Q[n + lane];
        nq -= n;
        __syncwarp();
        const bool exact = JOIN && FILTER && (e.x >> 24) >= kCodeSingleA;  // found by the join's scan
        // the row's psi and (unless exact) stored key load while the excitation is decoded
        ulonglong2 key = make_ulonglong2(0ULL, 0ULL);
        double2 pp = make_double2(0.0, 0.0);
        if (v) {
            if (!exact) key = __ldg(tp.keys + QC_IX(e.y, tp.n, tp.err));
            pp = __ldg(tp.psi + QC_IX(e.y, tp.n, tp.err));
        }
        if (FILTER && v) e.x = decode(e.x, sp, wl, smem, IA, IB);
        long long ent = 0;
        if (v) {
            const ulonglong2 xs = wsp->x, px = wsp->px;
            ent = verify_and_add<PREC, DIAG>(e, exact, key, pp, xs, wsp->hx, tp, ep.mode, T64,
                                             PREC == QC_FP64 ? make_float2(0.f, 0.f) : wsp->ip32, acc,
                                             [&](double& h64, float& h32, bool& sneg) {
                if ((e.x >> 16) == 0xFFFFu)
                    single_element<PREC>(e.x, px, sp, wl, dref, h64, h32, sneg);
                else
                    double_element<PREC>(e.x, px, sp, h64, h32, sneg);
            });
        }
        if (DIAG && ep.hit_list != nullptr) list_hits(ep, s, ent, lane);
        if (DIAG && ep.work != nullptr) {
            const bool sgl = (e.x >> 16) == 0xFFFFu;
            const bool same = !sgl && ((e.x ^ (e.x >> 16)) & 1u) == 0u;
            const unsigned m1 = __ballot_sync(QC_FULLMASK, ent != 0 && sgl);
            const unsigned m2 = __ballot_sync(QC_FULLMASK, ent != 0 && same);
            const unsigned m3 = __ballot_sync(QC_FULLMASK, ent != 0 && !sgl && !same);
            const unsigned m4 = __ballot_sync(QC_FULLMASK, ent != 0 && exact);
            if (lane == 0) {
                if (m1) atomicAdd(&ep.work->hits_single, static_cast<unsigned long long>(__popc(m1)));
                if (m2) atomicAdd(&ep.work->hits_same, static_cast<unsigned long long>(__popc(m2)));
                if (m3) atomicAdd(&ep.work->hits_ab, static_cast<unsigned long long>(__popc(m3)));
                if (m4) atomicAdd(&ep.work->hits_scanned, static_cast<unsigned long long>(__popc(m4)));
            }
        }
    };

    // Scan state of the join (the first phase of the main loop, before any candidate is
    // queued, so it owns the candidate queue's space): a chunk of up to 32 non-empty groups of
    // table rows -- start, exclusive row offset and kind in q[0..95], packed to the front (an
    // unused entry's offset is 0xFFFFFFFF) -- scanned as one list of q[102] rows, 32 per step;
    // the next alpha single excitation to classify in q[103] (shared memory keeps the scan state
    // out of the registers of the enumeration loop).  When the alpha list is full, the
    // enumeration runs over that segment and the scan state is entered again for the remaining
    // alpha singles (classes 0 and 4 only).  In the kernels with the beta' phase (BETA), after
    // the first segment's last alpha' chunk, a
    // sample with at least kMinLongAlpha long alpha' groups in it classifies its beta' (the
    // prefiltered beta singles, q[101] the next one, q[100] those kept): a beta' group short
    // against the number of those groups is scanned for the rows of long alpha' groups (alpha-
    // beta doubles, told by the row's alpha-group size in its entry against the sample's alpha'
    // threshold, which stays that of the full beta list; and x's beta single when class 1 is
    // enumerated) and leaves the beta list, which classes 1 and 4 of every segment then
    // enumerate compacted.
    auto store_chunk = [&](unsigned gst, unsigned gln, unsigned kind) {
        unsigned inc = gln;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(QC_FULLMASK, inc, o);
            if (lane >= o) inc += y;
        }
        const unsigned ne = __ballot_sync(QC_FULLMASK, gln != 0u);
        const int pos = __popc(ne & ltmask);
        if (lane >= __popc(ne)) q[32 + lane] = 0xFFFFFFFFu;
        if (gln != 0u) {
            q[pos] = gst;
            q[32 + pos] = inc - gln;
            q[64 + pos] = kind;
        }
        if (lane == 31) {
            q[102] = inc;
            if (DIAG && ep.work != nullptr && inc != 0u) atomicAdd(&ep.work->scan_rows, static_cast<unsigned long long>(inc));
        }
        __syncwarp();
    };

    if (FILTER) {
        const unsigned char* occA = wl;
        const unsigned char* virA = wl + 64;
        const unsigned char* occB = wl + 128;
        const unsigned char* virB = wl + 192;
        if (lane == 0) H[0] = 0u;
        // per-sample hash lists (low 32 bits of the linear hash contributions).  A single
        // excitation whose new spin string is absent from every table key can take part in
        // no hit (nor can any alpha-beta double built on it): the spin-string prefilter
        // drops it, compacting the single lists (IA / IB map back to the full index).
        const unsigned long long hxb = hx ^ hxa;
        nsb2 = 0;
        for (int t0 = 0; t0 < sp.nsb; t0 += 32) {
            const int t = t0 + lane;
            bool keep = false;
            uint32_t hv32 = 0u;
            unsigned pk = 0u;  // the single's spatial orbitals, occupied | empty << 8
            if (t < sp.nsb) {
                const int io = divB[t];
                const int ki = occB[io], ka = virB[t - io * sp.vb];
                const unsigned long long tm = T64[2 * ki + 1] ^ T64[2 * ka + 1];
                hv32 = static_cast<uint32_t>(tm);
                pk = static_cast<unsigned>(ki) | (static_cast<unsigned>(ka) << 8);
                keep = tp.bset == nullptr ||
                       set_contains(tp.bset, tp.set_mask, Bs ^ (1ULL << ki) ^ (1ULL << ka), hxb ^ tm);
            }
            const unsigned m = __ballot_sync(QC_FULLMASK, keep);
            if (keep) {
                const int pos = nsb2 + __popc(m & ltmask);
                H[QC_IX(oSB + pos, nH, sp.err)] = hv32;
                IB[QC_IX(pos, sp.nsb, sp.err)] = static_cast<unsigned short>(pk);
            }
            nsb2 += __popc(m);
        }
        if (join) {
            // x's own groups: lane 0 its alpha group (scanned, or classes 1 and 3), lane 1
            // its beta group (scanned, or class 2); an absent or empty group has no hits
            unsigned gst = 0u, gln = 0u, kind = 0u;
            bool en = false;
            if (lane < 2) {
                const unsigned off = lane == 0 ? 0u : tp.set_mask + 1u;
                const unsigned sl = lane == 0 ? set_slot(tp.aset, tp.set_mask, As, hxa)
                                              : set_slot(tp.bset, tp.set_mask, Bs, hxb);
                const unsigned len = sl != kNoSlot ? __ldg(tp.jlen + QC_IX(off + sl, 2LL * (tp.set_mask + 1LL), tp.err)) : 0u;
                const long long pairs = lane == 0 ? static_cast<long long>(nsb2) + static_cast<long long>(sp.npob) * sp.npvb
                                                  : static_cast<long long>(sp.npoa) * sp.npva;
                if (len > 0u) {
                    if (static_cast<long long>(len) * tp.scan_cost <= 4 * pairs) {
                        gst = __ldg(tp.jstart + QC_IX(off + sl, 2LL * (tp.set_mask + 1LL), tp.err));
                        gln = len;
                    } else {
                        en = true;
                    }
                }
                kind = lane == 0 ? kScanAlpha : kScanBeta;
            }
            enumA = __shfl_sync(QC_FULLMASK, en, 0);
            enumB = __shfl_sync(QC_FULLMASK, en, 1);
            if (lane == 0) {
                q[103] = 0u;
                if (BETA) {
                    q[100] = 0u;  // beta' phase: entries kept in the beta single list
                    q[101] = 0u;  // beta' phase: next entry to classify
                    // len * scan_cost > 4 (nsb2 + 1), as len > floor(4 (nsb2 + 1) / scan_cost), by
                    // the beta list before the beta' phase
                    wsp->athr = 4u * static_cast<unsigned>(nsb2 + 1) / static_cast<unsigned>(tp.scan_cost);
                }
            }
            store_chunk(gst, c == 0 ? gln : 0u, kind);  // later chunks classify but scan nothing
            nsa2 = 0;  // the alpha' groups are classified in the scan state
        } else {
            nsa2 = 0;
            for (int t0 = 0; t0 < sp.nsa; t0 += 32) {
                const int t = t0 + lane;
                bool keep = false;
                uint32_t hv32 = 0u;
                unsigned pk = 0u;
                if (t < sp.nsa) {
                    const int io = divA[t];
                    const int ki = occA[io], ka = virA[t - io * sp.va];
                    const unsigned long long tm = T64[2 * ki] ^ T64[2 * ka];
                    hv32 = static_cast<uint32_t>(tm);
                    pk = static_cast<unsigned>(ki) | (static_cast<unsigned>(ka) << 8);
                    keep = tp.aset == nullptr ||
                           set_contains(tp.aset, tp.set_mask, As ^ (1ULL << ki) ^ (1ULL << ka), hxa ^ tm);
                }
                const unsigned m = __ballot_sync(QC_FULLMASK, keep);
                if (keep) {
                    const int pos = nsa2 + __popc(m & ltmask);
                    H[QC_IX(oSA + pos, nH, sp.err)] = hv32;
                    IA[QC_IX(pos, nA, sp.err)] = static_cast<unsigned short>(pk);
                }
                nsa2 += __popc(m);
            }
        }
        // the same-spin pair lists serve classes 2 (alpha) and 3 (beta) alone, which the join
        // enumerates only when x's beta (alpha) group is too long to scan
        const bool needA = !join || enumB, needB = !join || enumA;
        if (lean) {
            if (needA) {
                for (int t = lane; t < sp.oa; t += 32) H[oPAo + t] = static_cast<uint32_t>(T64[2 * occA[t]]);
                for (int t = lane; t < sp.va; t += 32) H[oPAv + t] = static_cast<uint32_t>(T64[2 * virA[t]]);
            }
            if (needB) {
                for (int t = lane; t < sp.ob; t += 32) H[oPBo + t] = static_cast<uint32_t>(T64[2 * occB[t] + 1]);
                for (int t = lane; t < sp.vb; t += 32) H[oPBv + t] = static_cast<uint32_t>(T64[2 * virB[t] + 1]);
            }
        } else {
            if (needA) {
                for (int t = lane; t < sp.npoa; t += 32) {
                    const unsigned p = lut[t];
                    H[oPAo + t] = static_cast<uint32_t>(T64[2 * occA[p & 255u]] ^ T64[2 * occA[p >> 8]]);
                }
                for (int t = lane; t < sp.npva; t += 32) {
                    const unsigned p = lut[t];
                    H[oPAv + t] = static_cast<uint32_t>(T64[2 * virA[p & 255u]] ^ T64[2 * virA[p >> 8]]);
                }
            }
            if (needB) {
                for (int t = lane; t < sp.npob; t += 32) {
                    const unsigned p = lut[t];
                    H[oPBo + t] = static_cast<uint32_t>(T64[2 * occB[p & 255u] + 1] ^ T64[2 * occB[p >> 8] + 1]);
                }
                for (int t = lane; t < sp.npvb; t += 32) {
                    const unsigned p = lut[t];
                    H[oPBv + t] = static_cast<uint32_t>(T64[2 * virB[p & 255u] + 1] ^ T64[2 * virB[p >> 8] + 1]);
                }
            }
        }
        __syncwarp();
    }
    const uint32_t hx32 = static_cast<uint32_t>(hx);
    // iterator over (class, outer block u0, inner block w0)
    int cls = -1, oo = 0, n1 = 0, io = 0, n2 = 0, u0 = 0, w0 = 0;
    bool done = false, need_class = true, need_outer = true;
    bool pairs = false;  // lean layout, same-spin doubles: list entries are formed from pairs
    // outer hash values (the low 32 bits of x's hash XOR the outer entry)
    uint32_t hu[U];
    unsigned umask = 0;
#pragma unroll
    for (int k = 0; k < U; ++k) hu[k] = 0u;
    bool scanning = join;
    bool bph = false;     // join: the beta' phase of the scan state is due
    bool seg2 = false;    // join: a later segment of the alpha list (classes 0 and 4 only)
    unsigned sbase = 0u;  // next row of the current scan chunk
    while (true) {
        if (scanning) {
            const unsigned stotal = q[102];
            const int st0 = static_cast<int>(q[103]);
            if (sbase < stotal) {
                // steps of 32 rows of the chunk, while both hit queues have room for another
                // step.  Lane l's row sbase + l lies in group g = (the groups starting at or
                // before sbase) - 1 + (the groups starting at window positions 1..l): one ballot
                // over the groups' offsets and one OR-reduction of their start positions.  A
                // row connects to x when the popcount of its string of the other spin against
                // x's is 2 or 4 (x's alpha group: a beta single or beta-beta double), 4 (x's beta
                // group: an alpha-alpha double) or 0 or 2 (an alpha' group: the alpha single or
                // an alpha-beta double).  Singles and doubles go to separate queues, so that hit
                // batches do not mix the two element paths.
                const unsigned offj = q[32 + lane];  // group lane's first row in the chunk
                const unsigned long long ras = wsp->as, rbs = wsp->bs;
                const unsigned lthr = BETA ? wsp->athr : 0u;
                const unsigned lemask = ltmask | (1u << lane);
                do {
                    const unsigned v = sbase + lane;
                    const unsigned rel = offj - sbase;
                    const unsigned starts = __reduce_or_sync(QC_FULLMASK, rel - 1u < 31u ? 1u << rel : 0u);
                    const int g = __popc(__ballot_sync(QC_FULLMASK, offj <= sbase)) - 1 + __popc(starts & lemask);
                    bool dbl = false, sgl = false;
                    unsigned code = 0u, row = 0u;
                    if (v < stotal) {
                        const unsigned kd = q[64 + g];
                        const ulonglong2 e = __ldg(tp.gent + QC_IX(q[g] + (v - q[32 + g]), 2 * tp.n, tp.err));
                        const unsigned kk = kd & 3u;
                        const unsigned long long ref = (BETA ? (kk & 1u) == 0u : kk == kScanBeta) ? ras : rbs;
                        const unsigned long long dm = e.x ^ ref;
                        const int d = __popcll(dm);
                        if (BETA) {
                            // an alpha' or beta' group: its single at d == 0, alpha-beta doubles
                            // at d == 2 (a beta' group's only where the row's alpha' group is long)
                            const bool prime = kk == kScanAlphaP || kk == kScanBetaP;
                            sgl = prime ? d == 0 && (kd & (kk == kScanAlphaP ? 3u : 4u)) != 0u
                                        : (kk == kScanAlpha && d == 2);
                            dbl = prime ? d == 2 && (kk == kScanAlphaP || static_cast<unsigned>(e.y >> 32) > lthr)
                                        : d == 4;
                        } else {
                            sgl = kk == kScanAlpha ? d == 2 : (kk == kScanAlphaP && d == 0);
                            dbl = kk == kScanAlphaP ? d == 2 : d == 4;
                        }
                        if (sgl || dbl) {
                            code = scan_code<BETA>(kd, d, dm & ref, dm & e.x);
                            row = static_cast<unsigned>(e.y);
                        }
                    }
                    const unsigned md = __ballot_sync(QC_FULLMASK, dbl), ms = __ballot_sync(QC_FULLMASK, sgl);
                    if (dbl) hq[QC_IX(nh + __popc(md & ltmask), 64, sp.err)] = make_uint2(code, row);
                    if (sgl) hs[QC_IX(ns + __popc(ms & ltmask), kSingleCap, sp.err)] = make_uint2(code, row);
                    nh += __popc(md);
                    ns += __popc(ms);
                    sbase += 32u;
                    __syncwarp();
                } while (sbase < stotal && nh < 32 && ns < 32);
            } else if (st0 < sp.nsa) {
                // the next 32 alpha' = single excitations of x's alpha string: a long group
                // joins the lists of classes 0 and 4, a short one becomes a scan descriptor
                const unsigned char* occA = wl;
                const unsigned char* virA = wl + 64;
                const int t = st0 + lane;
                const int a_next = SEG ? static_cast<int>(wsp->a_next) : 0;
                const int a_seen = SEG ? static_cast<int>(wsp->a_seen) : 0;
                bool lng = false;
                uint32_t hv32 = 0u;
                unsigned gst = 0u, gln = 0u, kd = 0u, len = 0u, start = 0u;
                // singles below a_next are in an earlier segment; between a_next and a_seen only
                // their long groups are left (the short ones were scanned)
                if (t < sp.nsa && t >= a_next) {
                    const int oi = divA[t];
                    const int ki = occA[oi], ka = virA[t - oi * sp.va];
                    const unsigned long long tm = T64[2 * ki] ^ T64[2 * ka];
                    hv32 = static_cast<uint32_t>(tm);
                    const unsigned sl = set_slot(tp.aset, tp.set_mask, wsp->as ^ (1ULL << ki) ^ (1ULL << ka), wsp->hxa ^ tm);
                    if (sl != kNoSlot) {
                        len = __ldg(tp.jlen + QC_IX(sl, tp.set_mask + 1LL, tp.err));
                        start = __ldg(tp.jstart + QC_IX(sl, tp.set_mask + 1LL, tp.err));
                    }
                    lng = BETA ? len > wsp->athr : static_cast<long long>(len) * tp.scan_cost > 4LL * (nsb2 + 1);
                    kd = kScanAlphaP | (static_cast<unsigned>(ki) << 8) | (static_cast<unsigned>(ka) << 16);
                }
                // a long group joins the alpha list while it has room; the first that does not
                // fit ends this segment's classification (a_next), and short groups are
                // scanned once (t >= a_seen)
                const unsigned m = __ballot_sync(QC_FULLMASK, lng);
                const int pos = nsa2 + __popc(m & ltmask);
                const bool keep = SEG ? (lng && pos < nA) : lng;
                if (keep) {
                    H[QC_IX(oSA + pos, nH, sp.err)] = hv32;
                    IA[QC_IX(pos, nA, sp.err)] = static_cast<unsigned short>((kd >> 8) & 0xFFFFu);
                } else if (!lng && (!SEG || t >= a_seen)) {
                    gst = start;
                    gln = len;
                }
                nsa2 = SEG ? min(nA, nsa2 + __popc(m)) : nsa2 + __popc(m);
                // after the first segment's last chunk: the beta' phase (judged by the long alpha'
                // groups of that segment when the list is full; the later segments enumerate the
                // same compacted beta list)
                bool whole = st0 + 32 >= sp.nsa;
                if (SEG) {
                    const unsigned md = __ballot_sync(QC_FULLMASK, lng && !keep);
                    whole = (whole || md != 0u) && !seg2;
                    __syncwarp();
                    if (lane == 0) {
                        const int end = min(st0 + 32, sp.nsa);
                        wsp->a_next = static_cast<unsigned>(md ? st0 + __ffs(md) - 1 : end);
                        wsp->a_seen = static_cast<unsigned>(max(a_seen, end));
                        q[103] = static_cast<unsigned>(md ? sp.nsa : st0 + 32);
                    }
                } else {
                    __syncwarp();
                    if (lane == 0) q[103] = static_cast<unsigned>(st0 + 32);
                }
                bph = BETA && whole && tp.alpha_cap > 0 && tp.beta_cost > 0 && nsa2 >= kMinLongAlpha && nsb2 > 0;
                store_chunk(gst, c == 0 ? gln : 0u, kd);
                sbase = 0u;
            } else if (BETA && bph) {
                // the next 32 beta' of the beta single list: a group with len beta_cost <= 4
                // (long alpha' groups) becomes a scan descriptor, the others stay in the list
                // (compacted in place: every entry of the chunk is read before any is written)
                const int tb = static_cast<int>(q[101]);
                const int kept0 = static_cast<int>(q[100]);
                const int t = tb + lane;
                bool keep = false;
                uint32_t hv32 = 0u;
                unsigned short pk = 0;
                unsigned gst = 0u, gln = 0u, kd = 0u;
                if (t < nsb2) {
                    hv32 = H[QC_IX(oSB + t, nH, sp.err)];
                    pk = IB[QC_IX(t, sp.nsb, sp.err)];
                    const unsigned kj = pk & 255u, kb = static_cast<unsigned>(pk) >> 8;
                    const unsigned long long tm = T64[2 * kj + 1] ^ T64[2 * kb + 1];
                    const unsigned sl = set_slot(tp.bset, tp.set_mask, wsp->bs ^ (1ULL << kj) ^ (1ULL << kb),
                                                 wsp->hx ^ wsp->hxa ^ tm);
                    const long long jo = static_cast<long long>(tp.set_mask) + 1LL + sl;
                    const unsigned len =
                        sl != kNoSlot ? __ldg(tp.jlen + QC_IX(jo, 2LL * (tp.set_mask + 1LL), tp.err)) : 0u;
                    keep = !(len > 0u && static_cast<long long>(len) * tp.beta_cost <= 4LL * nsa2);
                    if (!keep) {
                        gst = __ldg(tp.jstart + QC_IX(jo, 2LL * (tp.set_mask + 1LL), tp.err));
                        gln = len;
                        // bit 2: x's beta single is taken from the group (class 1 is enumerated)
                        kd = kScanBetaP | (enumA ? 4u : 0u) | (kj << 8) | (kb << 16);
                    }
                }
                const unsigned m = __ballot_sync(QC_FULLMASK, keep);
                if (DIAG && ep.work != nullptr && lane == 0 && c == 0) {
                    const int nv = min(32, nsb2 - tb);
                    atomicAdd(&ep.work->beta_looked, static_cast<unsigned long long>(nv));
                    atomicAdd(&ep.work->beta_groups, static_cast<unsigned long long>(nv - __popc(m)));
                }
                __syncwarp();
                if (keep) {
                    const int pos = kept0 + __popc(m & ltmask);
                    H[QC_IX(oSB + pos, nH, sp.err)] = hv32;
                    IB[QC_IX(pos, sp.nsb, sp.err)] = pk;
                }
                const int kept = kept0 + __popc(m);
                if (lane == 0) {
                    q[100] = static_cast<unsigned>(kept);
                    q[101] = static_cast<unsigned>(tb + 32);
                }
                if (tb + 32 >= nsb2) {
                    bph = false;
                    nsb2 = kept;
                }
                store_chunk(gst, c == 0 ? gln : 0u, kd);
                sbase = 0u;
            } else {
                scanning = false;
            }
        } else if (!done) {
            if (need_class) {
                do {
                    ++cls;
                    if (cls == 0) { oo = 0; n1 = 1; io = oSA; n2 = nsa2; }
                    else if (cls == 1) { oo = 0; n1 = 1; io = oSB; n2 = nsb2; }
                    else if (cls == 2) { oo = oPAo; n1 = sp.npoa; io = oPAv; n2 = sp.npva; }
                    else if (cls == 3) { oo = oPBo; n1 = sp.npob; io = oPBv; n2 = sp.npvb; }
                    else if (cls == 4) { oo = oSA; n1 = nsa2; io = oSB; n2 = nsb2; }
                } while (cls < 5 && (n1 == 0 || n2 == 0 || (cls < 2 ? c != 0 : c * U >= n1) ||
                                     ((cls == 1 || cls == 3) && !enumA) || (cls == 2 && !enumB) ||
                                     (SEG && seg2 && cls >= 1 && cls <= 3)));
                done = cls >= 5;
                pairs = lean && (cls == 2 || cls == 3);
                // excitation chunk c of C: the singles in chunk 0, outer blocks c, c + C, ...
                u0 = cls >= 2 ? c * U : 0;
                w0 = 0;
                need_class = false;
                need_outer = true;
            }
            if (!done) {
                if (need_outer) {
                    umask = 0;
#pragma unroll
                    for (int k = 0; k < U; ++k) {
                        const bool v = u0 + k < n1;
                        if (FILTER) {
                            uint32_t e = 0u;
                            if (v) {
                                if (pairs) {
                                    const unsigned pp = lut[u0 + k];
                                    e = H[QC_IX(oo + (pp & 255u), nH, sp.err)] ^ H[QC_IX(oo + (pp >> 8), nH, sp.err)];
                                } else {
                                    e = H[QC_IX(oo + u0 + k, nH, sp.err)];
                                }
                            }
                            hu[k] = hx32 ^ e;
                        }
                        umask |= (v ? 1u : 0u) << k;
                    }
                    if (DIAG && FILTER && ep.work != nullptr && lane == 0)
                        atomicAdd(&ep.work->tests, static_cast<unsigned long long>(__popc(umask)) * n2);
                    need_outer = false;
                }
                // steps over this block of U outer entries until its inner list ends or the
                // candidate queue holds a batch for the resolution stages (a step adds at
                // most 32 U entries, so the queue never exceeds 31 + 32 U)
                const unsigned cbase = (static_cast<unsigned>(cls) << 24) | (static_cast<unsigned>(u0) << 12);
                do {
                    const int w = w0 + lane;
                    const bool wv = w < n2;
                    const unsigned vm = wv ? umask : 0u;
                    uint32_t hw = 0u;
                    if (FILTER && wv) {
                        if (LEAN != 0 && pairs) {
                            const unsigned pp = lut[w];
                            hw = H[QC_IX(io + (pp & 255u), nH, sp.err)] ^ H[QC_IX(io + (pp >> 8), nH, sp.err)];
                        } else {
                            hw = H[QC_IX(io + w, nH, sp.err)];
                        }
                    }
                    const unsigned ccode = cbase | static_cast<unsigned>(w);
#pragma unroll
                    for (int k = 0; k < U; ++k) {
                        bool pass;
                        if (FILTER) {
                            // the hash's low bits g pick the filter word (bits 5.., a byte offset
                            // of g >> 3 masked to whole words) and its three bits
                            const uint32_t g = hu[k] ^ hw;
                            const uint32_t word = *reinterpret_cast<const uint32_t*>(
                                reinterpret_cast<const unsigned char*>(filt) + QC_IX((g >> 3) & wmask4, 4LL << tp.fw, sp.err));
                            const uint32_t t = __funnelshift_r(word, word, g) &
                                               __funnelshift_r(word, word, g >> 27) &
                                               __funnelshift_r(word, word, g >> 22);
                            pass = ((t & (vm >> k)) & 1u) != 0u;
                        } else {
                            pass = ((vm >> k) & 1u) != 0u;
                        }
                        const unsigned m = __ballot_sync(QC_FULLMASK, pass);
                        if (pass) q[QC_IX(qn + __popc(m & ltmask), kCandCap, sp.err)] = ccode + (static_cast<unsigned>(k) << 12);
                        qn += __popc(m);
                    }
                    w0 += 32;
                } while (w0 < n2 && qn < 32);
                if (w0 >= n2) {
                    w0 = 0;
                    u0 += cls >= 2 ? U * C : U;
                    need_outer = true;
                    if (u0 >= n1) need_class = true;
                }
            }
        }
        __syncwarp();
        // resolution stages (the hit queue first, so it never exceeds 63 entries)
        while (true) {
            const bool dh = nh >= 32 || (done && qn == 0 && nh > 0);
            const bool dsg = JOIN && (ns >= 32 || (done && qn == 0 && ns > 0));
            if (dh || dsg) {
                hit_batch(dh ? hq : hs, dh ? nh : ns);
            } else if (qn >= 32 || (done && qn > 0)) {
                const int n = qn < 32 ? qn : 32;
                const bool v = lane < n;
                const unsigned code = v ? q[lane] : 0u;
                if (DIAG && ep.work != nullptr && lane == 0) atomicAdd(&ep.work->probes, static_cast<unsigned long long>(n));
                __syncwarp();
                for (int t = lane; t < qn - n; t += 32) q[t] = q[n + t];
                qn -= n;
                __syncwarp();
                unsigned item = 0u;
                long long row = -1;
                if (v) {
                    unsigned g;
                    if (FILTER) {
                        // the low hash bits of x' again from the hash lists: g = hx ^ outer
                        // ^ inner entry of the candidate's class (no decode, no excite)
                        const unsigned cc = code >> 24;
                        const int u = static_cast<int>((code >> 12) & 4095u);
                        const int w = static_cast<int>(code & 4095u);
                        const int ob = cc == 2u ? oPAo : cc == 3u ? oPBo : cc == 4u ? oSA : 0;
                        const int ib = cc == 0u ? oSA : cc == 1u ? oSB : cc == 2u ? oPAv : cc == 3u ? oPBv : oSB;
                        uint32_t ho, hi;
                        if (LEAN != 0 && lean && (cc == 2u || cc == 3u)) {
                            const unsigned pu = lut[u], pw = lut[w];
                            ho = H[QC_IX(ob + (pu & 255u), nH, sp.err)] ^ H[QC_IX(ob + (pu >> 8), nH, sp.err)];
                            hi = H[QC_IX(ib + (pw & 255u), nH, sp.err)] ^ H[QC_IX(ib + (pw >> 8), nH, sp.err)];
                        } else {
                            ho = H[QC_IX(ob + u, nH, sp.err)];
                            hi = H[QC_IX(ib + w, nH, sp.err)];
                        }
                        g = hx32 ^ ho ^ hi;
                        item = code;
                    } else {
                        item = decode(code, sp, wl, smem, IA, IB);
                        unsigned long long h;
                        excite(item, wsp->x, wsp->hx, T64, h);
                        g = static_cast<unsigned>(h);
                    }
                    row = probe_fp(g, tp);
                    if (row < 0 && ep.mode == QC_FULL) acc.missing++;
                }
                const bool hit = row >= 0;
                const unsigned mh = __ballot_sync(QC_FULLMASK, hit);
                if (hit) hq[QC_IX(nh + __popc(mh & ltmask), 64, sp.err)] = make_uint2(item, static_cast<unsigned>(row));
                nh += __popc(mh);
                __syncwarp();
            } else {
                break;
            }
        }
        if (done) {
            // join: long alpha' groups that did not fit the alpha list: classify and enumerate
            // the next segment (the queues are empty here)
            if (!(SEG && join && static_cast<int>(wsp->a_next) < sp.nsa)) break;
            scanning = true;
            seg2 = true;
            done = false;
            need_class = true;
            cls = -1;
            nsa2 = 0;
            sbase = 0u;
            if (lane == 0) {
                q[102] = 0u;
                q[103] = wsp->a_next / 32u * 32u;
            }
            __syncwarp();
        }
    }
    sample_finish<PREC, DIAG, FILTER>(ep, s, lane, wsp->ediag, wsp->psix, acc, c, C);
    __syncwarp();
}

// ------------------------------------------------------------------------------------
// K3: Eq. 1 reduction (two passes, deterministic order, last-block finish)
// ------------------------------------------------------------------------------------
constexpr int kRedThreads = 256;


template <typename Tv>
__device__ __forceinline__ Tv block_sum(Tv v, Tv* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = sh[threadIdx.x] + sh[threadIdx.x + o];
        __syncthreads();
    }
    Tv r = sh[0];
    __syncthreads();
    return r;
}

// Pass 1 of one molecule over its rows [lo, hi), as block `bid` of `nblk`: W, sum c E and the
// count of finite samples; the last block to finish writes the mean.
__device__ __forceinline__ void reduce_pass1_body(const EvalParams& ep, double* part, unsigned bid,
                                                  unsigned nblk, long long lo, long long hi) {
    __shared__ double shd[kRedThreads];
    __shared__ long long shl[kRedThreads];
    __shared__ bool last;
    long long w = 0, used = 0;
    double sr = 0.0, si = 0.0;
    bool neg = false;
    for (long long i = lo + static_cast<long long>(bid) * kRedThreads + threadIdx.x; i < hi;
         i += static_cast<long long>(nblk) * kRedThreads) {
        const double2 e = ep.eloc[i];
        const long long c = ep.counts[i];
        if (c < 0) {
            neg = true;
            continue;
        }
        if (isfinite(e.x) && isfinite(e.y)) {
            w += c;
            sr += static_cast<double>(c) * e.x;
            si += static_cast<double>(c) * e.y;
            used++;
        }
    }
    if (neg) atomicOr(&ep.ctr->flags, QC_FLAG_NEG_COUNT);
    const long long bw = block_sum<long long>(w, shl);
    const long long bu = block_sum<long long>(used, shl);
    const double bsr = block_sum<double>(sr, shd);
    const double bsi = block_sum<double>(si, shd);
    if (threadIdx.x == 0) {
        part[4 * bid + 0] = bsr;
        part[4 * bid + 1] = bsi;
        part[4 * bid + 2] = __longlong_as_double(bw);
        part[4 * bid + 3] = __longlong_as_double(bu);
        __threadfence();
        last = (atomicAdd(&ep.ctr->ticket, 1u) == nblk - 1);
    }
    __syncthreads();
    if (last) {
        // the last block adds the partials: thread t those of blocks t, t + 256, ..., then a
        // fixed tree over the threads (the same order on every run)
        __threadfence();
        double tr = 0.0, ti = 0.0;
        long long tw = 0, tu = 0;
        for (unsigned b = threadIdx.x; b < nblk; b += kRedThreads) {
            tr += __ldcg(part + 4 * b + 0);
            ti += __ldcg(part + 4 * b + 1);
            tw += __double_as_longlong(__ldcg(part + 4 * b + 2));
            tu += __double_as_longlong(__ldcg(part + 4 * b + 3));
        }
        tr = block_sum<double>(tr, shd);
        ti = block_sum<double>(ti, shd);
        tw = block_sum<long long>(tw, shl);
        tu = block_sum<long long>(tu, shl);
        if (threadIdx.x != 0) return;
        Counters* c = ep.ctr;
        c->w = tw;
        c->used = static_cast<unsigned long long>(tu);
        c->sce_re = tr;
        c->sce_im = ti;
        c->mean_re = tr / static_cast<double>(tw);
        c->mean_im = ti / static_cast<double>(tw);
        c->ticket = 0u;
    }
}

// Pass 2 of one molecule over its rows [lo, hi): sum c |E - Ebar|^2; the last block writes the
// summary.
__device__ __forceinline__ void reduce_pass2_body(const EvalParams& ep, double* part, qc_eloc_summary* out,
                                                  long long pairs_per_sample, unsigned bid, unsigned nblk,
                                                  long long lo, long long hi) {
    __shared__ double shd[kRedThreads];
    __shared__ bool last;
    const double mr = ep.ctr->mean_re, mi = ep.ctr->mean_im;
    double v = 0.0;
    for (long long i = lo + static_cast<long long>(bid) * kRedThreads + threadIdx.x; i < hi;
         i += static_cast<long long>(nblk) * kRedThreads) {
        const double2 e = ep.eloc[i];
        const long long c = ep.counts[i];
        if (c < 0 || !isfinite(e.x) || !isfinite(e.y)) continue;
        const double dr = e.x - mr, di = e.y - mi;
        v += static_cast<double>(c) * (dr * dr + di * di);
    }
    const double bv = block_sum<double>(v, shd);
    if (threadIdx.x == 0) {
        part[4 * bid] = bv;
        __threadfence();
        last = (atomicAdd(&ep.ctr->ticket, 1u) == nblk - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double tv = 0.0;
        for (unsigned b = threadIdx.x; b < nblk; b += kRedThreads) tv += __ldcg(part + 4 * b);
        tv = block_sum<double>(tv, shd);
        if (threadIdx.x != 0) return;
        Counters* c = ep.ctr;
        const unsigned f = c->flags;
        int st = QC_OK;
        if (f & QC_FLAG_UNSORTED) st = QC_ERR_UNSORTED;
        else if (f & QC_FLAG_DUP) st = QC_ERR_DUP;
        else if (f & QC_FLAG_NELEC) st = QC_ERR_NELEC;
        else if (f & QC_FLAG_NEG_COUNT) st = QC_ERR_COUNTS;
        else if (f & (QC_FLAG_TABLE_FULL | QC_FLAG_LIST_FULL)) st = QC_ERR_CAPACITY;
        else if (f & QC_FLAG_BOUNDS) st = QC_ERR_BOUNDS;
        else if (f & QC_FLAG_TIMEOUT) st = QC_ERR_TIMEOUT;
        else if (f & QC_FLAG_MISSING) st = QC_ERR_MISSING;
        else if (f & QC_FLAG_ZERO_PSI) st = QC_ERR_ZERO_PSI;
        const double w = static_cast<double>(c->w);
        out->e_re = c->mean_re;
        out->e_im = c->mean_im;
        out->var = tv / w;
        out->w = w;
        out->sum_ce_re = c->sce_re;
        out->sum_ce_im = c->sce_im;
        out->n_used = c->used;
        out->n_pairs = static_cast<unsigned long long>(hi - lo - static_cast<long long>(c->invalid)) *
                       static_cast<unsigned long long>(pairs_per_sample);
        out->n_hits = c->hits;
        out->n_missing = c->missing;
        out->n_bad = c->bad;
        out->flags = f;
        out->status = st;
        c->ticket = 0u;
    }
}

}  // namespace qc
