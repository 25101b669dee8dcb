// paulib_slots.cuh -- canonical form by slot sort (PauLIB Sec. III-H
// sort_and_combine on the outer product of Sec. IV-C), laid out for one GB300.
//
// The paper sorts an index array by the lexicographic key of the packed words
// and merges equal neighbours in a linear scan.  Here the records (products,
// or the terms of one sum) pass through:
//
//   level 1   coarse key ranges, as in paulib_pipeline.cuh (sample, splitters,
//             a tiled count over the product space, a scatter of 32-bit
//             record numbers);
//   split     per coarse range: a sample of its keys sorted in shared memory
//             gives up to kFmax fine splitters ("slots"); every record is
//             located among them (k_slot_locate), slots get offsets, and the
//             record's term -- key and coefficient with the phase i^k folded
//             in -- is formed once and written into its slot (k_slot_place);
//   leaves    runs of consecutive slots holding at most leaf_cap records are
//             ordered in shared memory by full key (k_slot_leaf), equal keys
//             are summed, and the merged terms are written straight into the
//             output sum at an offset found by a decoupled look-back over the
//             leaves in key order (Merrill and Garland's single-pass scan).
//
// The output sum's key array is the term array itself: a leaf reads all of
// its terms into shared memory before it publishes its distinct count, and
// every merged term lands at or below the position of the first term of its
// leaf, so no leaf overwrites terms another leaf has still to read.
//
// A slot holding one repeated key (found when its sample run fills a whole
// slot) is summed without sorting, whatever its size.  A slot larger than a
// leaf (sampling bad luck) is ordered in sub-ranges by a multi-pass leaf.
// Every device wait is bounded; failures set bits of a device error word.
#pragma once
#include "paulib_pipeline.cuh"

namespace paulib {
namespace slot {

constexpr uint32_t kFmax = 2048;        // fine splitter pairs per coarse range
constexpr uint32_t kMaxSlots = 2 * kFmax - 1;
constexpr uint32_t kSampleMax = 16384;  // sample keys per coarse range
constexpr int kSplThreads = 1024;
constexpr uint32_t kChunkRecs = 8192;   // records per chunk of the locate/place passes
constexpr int kPartThreads = 512;
constexpr int kLeafThreads = 512;
constexpr uint32_t kSubMax = 16;        // sub-ranges of one oversized slot
constexpr uint64_t kPad = ~0ull;        // sort padding, above every element

// Records per leaf: 64 KB of keys in shared memory, at most 2048.
// Records per leaf: what fits two leaf CTAs on one SM (keys, values, two
// 64-bit sort side words, the order and the run starts).
template <int NW>
__host__ __device__ constexpr uint32_t cap() {
    return NW <= 8 ? 1024u : 8192u / NW;
}

// Device checks (bits of the error word).  SE_ORDER: a leaf's whole-key order
// check failed (possible only after a key-hash collision); SE_ORDER_SPLIT:
// the same for a range's sample.
enum : int32_t {
    SE_OVERLAP = 64, SE_SUBRANGE = 128, SE_TIMEOUT = 256, SE_BOUNDS = 512, SE_ORDER = 1024,
    SE_ORDER_SPLIT = 2048
};
enum : uint32_t { LF_UNIFORM = 1u, LF_OVERSIZE = 2u };

struct Leaf {
    uint64_t off;  // first term (position in the term array)
    uint32_t n;    // terms
    uint32_t flags;
};

// Look-back status of a leaf: state in the top two bits, count below.
constexpr uint64_t kAgg = 1ull << 62;
constexpr uint64_t kIncl = 2ull << 62;
constexpr uint64_t kValMask = (1ull << 62) - 1ull;

// ---------------------------------------------------------------- key access

// Word-major keys in shared memory: word q of element i at s[q*stride + i].
struct SKeys {
    const uint64_t* s;
    uint32_t stride;
    __device__ __forceinline__ uint64_t w(uint32_t i, int q) const { return s[(size_t)q * stride + i]; }
};
// Term keys in global memory, NW words per element.
template <int NW>
struct GKeys {
    const uint64_t* g;
    __device__ __forceinline__ uint64_t w(uint32_t i, int q) const { return g[(size_t)i * NW + q]; }
};

// 64 key bits starting at bit position P (word 0's top bit is position 0).
template <int NW, class K>
__device__ __forceinline__ uint64_t bits_at(const K& k, uint32_t i, uint32_t P) {
    const uint32_t w = P >> 6, sh = P & 63u;
    const uint64_t v = w < (uint32_t)NW ? k.w(i, (int)w) : 0ull;
    const uint64_t nx = w + 1u < (uint32_t)NW ? k.w(i, (int)w + 1) : 0ull;
    return sh ? (v << sh) | (nx >> (64u - sh)) : v;
}

__host__ __device__ constexpr uint32_t pow2_at_least(uint32_t n) {
    uint32_t p = 1;
    while (p < n) p <<= 1;
    return p;
}

// First bit position where keys of the set differ (64*NW when all are
// equal), from the per-word OR of (key ^ key0) that every thread passes in.
// s_or holds NW words of shared scratch; whole CTA.
template <int NW>
__device__ __forceinline__ uint32_t block_first_diff(uint64_t (&acc)[NW], unsigned long long* s_or, uint32_t* s_P) {
    for (int q = threadIdx.x; q < NW; q += blockDim.x) s_or[q] = 0ull;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        uint64_t v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicOr(&s_or[q], (unsigned long long)v);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t P = 64u * NW;
        for (int q = 0; q < NW; ++q)
            if (s_or[q]) {
                P = 64u * q + (uint32_t)__clzll((long long)s_or[q]);
                break;
            }
        *s_P = P;
    }
    __syncthreads();
    return *s_P;
}


// Whole-key comparison of elements ia, ib from word w0 on: -1, 0, 1.
template <int NW, class K>
__device__ __forceinline__ int key_cmp_k(const K& k, uint32_t ia, uint32_t ib, int w0) {
    for (int q = w0; q < NW; ++q) {
        const uint64_t x = k.w(ia, q), y = k.w(ib, q);
        if (x != y) return x < y ? -1 : 1;
    }
    return 0;
}

// 64-bit hash of a whole key: the SplitMix64 finaliser applied after each
// word (it spreads a difference in any bit over all bits, so differences in
// several words cannot cancel the way a plain multiply-xor chain lets
// differences in matching high bits cancel).  Used only to recognise equal
// keys quickly; the ordered result is verified against whole keys.
template <int NW, class K>
__device__ __forceinline__ uint64_t key_hash(const K& k, uint32_t i) {
    uint64_t h = 0x243f6a8885a308d3ull;
#pragma unroll
    for (int q = 0; q < NW; ++q) h = mix64(h ^ k.w(i, q));
    return h;
}

// Per-element side data of an ordering: key bits [P+48, P+112) and the key
// hash, indexed by element.
struct OrdAux {
    uint64_t* c2;
    uint64_t* h;
};

// Sort element: key bits [P, P+48) above a 16-bit element index (all keys
// of the set agree before bit P).  Equal codes compare the second window,
// then the hashes: equal hashes are taken as equal keys (ordered by index),
// different hashes fall back to whole keys from the first word the two
// windows leave open.  The result is verified by run_heads.
template <int NW, class K>
__device__ __forceinline__ bool el_less(uint64_t a, uint64_t b, const K& k, const OrdAux& x, int w2) {
    if ((a >> 16) != (b >> 16) || a == kPad || b == kPad) return a < b;
    const uint32_t ia = (uint32_t)(a & 0xffffu), ib = (uint32_t)(b & 0xffffu);
    const uint64_t ca = x.c2[ia], cb = x.c2[ib];
    if (ca != cb) return ca < cb;
    if (x.h[ia] == x.h[ib]) return ia < ib;
    const int c = key_cmp_k<NW>(k, ia, ib, w2);
    return c != 0 ? c < 0 : ia < ib;
}

// Bitonic sort of s[0, N) (N a power of two) by el_less, whole CTA.  A warp
// handles 32 consecutive pairs of a stage, so the stages of distance at most
// 32 stay inside one 64-element block per warp and need only a warp barrier.
template <int THREADS, int NW, class K>
__device__ void block_sort_keys(uint64_t* s, uint32_t N, const K& k, const OrdAux& x, int w2) {
    for (uint32_t kk = 2; kk <= N; kk <<= 1) {
        for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
            for (uint32_t t = threadIdx.x; t < (N >> 1); t += THREADS) {
                const uint32_t i = ((t & ~(j - 1u)) << 1) | (t & (j - 1u));
                const uint32_t l = i | j;
                const uint64_t a = s[i], b = s[l];
                const bool asc = (i & kk) == 0u;
                if (asc ? el_less<NW>(b, a, k, x, w2) : el_less<NW>(a, b, k, x, w2)) {
                    s[i] = b;
                    s[l] = a;
                }
            }
            if (j >= 64u) __syncthreads();
            else __syncwarp();
        }
        if (kk >= 64u && kk < N) __syncthreads();  // the next level starts at distance kk
    }
    __syncthreads();
}

struct OrderScratch {
    unsigned long long s_or[32];
    uint32_t s_P, s_err;
};

// Orders the n elements of k (n <= 65536) by full key, equal keys by index:
// s[0, n) receives (code | index) in that order, s[n, pow2(n)) padding.
// Returns P, the first bit where any two keys differ (64*NW when all are
// equal).  Whole CTA.
template <int NW, int THREADS, class K>
__device__ uint32_t order_keys(uint32_t n, const K& k, uint64_t* s, const OrdAux& x, OrderScratch& m) {
    uint64_t acc[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) acc[w] = 0;
    for (uint32_t i = threadIdx.x; i < n; i += THREADS)
#pragma unroll
        for (int w = 0; w < NW; ++w) acc[w] |= k.w(i, w) ^ k.w(0, w);
    const uint32_t P = block_first_diff<NW>(acc, m.s_or, &m.s_P);
    const uint32_t N2 = pow2_at_least(n);
    for (uint32_t i = threadIdx.x; i < N2; i += THREADS) {
        if (i < n) {
            s[i] = ((bits_at<NW>(k, i, P) >> 16) << 16) | i;
            x.c2[i] = bits_at<NW>(k, i, P + 48u);
            x.h[i] = key_hash<NW>(k, i);
        } else {
            s[i] = kPad;
        }
    }
    __syncthreads();
    block_sort_keys<THREADS, NW>(s, N2, k, x, (int)((P + 112u) >> 6));
    return P;
}

// Positions where a new key starts in the ordered elements s[0, n): writes
// s_hd[r] = first position of distinct key r and s_hd[D] = n; returns D.
// Every adjacent pair is compared as whole keys (from word w0, before which
// all keys agree), which also verifies the order: a pair out of order (only
// possible after a hash collision) sets *err.  Whole CTA.
template <int NW, int THREADS, class K, class HD>
__device__ uint32_t run_heads(uint32_t n, const K& k, const uint64_t* s, int w0, HD* s_hd, uint32_t* s_warp,
                              uint32_t* err) {
    const uint32_t per = (n + THREADS - 1) / THREADS;
    const uint32_t p0 = threadIdx.x * per, p1 = mn<uint32_t>(n, p0 + per);
    uint32_t cnt = 0, bad = 0;
    for (uint32_t p = p0; p < p1; ++p) {
        const int c = p == 0 ? -1 : key_cmp_k<NW>(k, (uint32_t)(s[p - 1] & 0xffffu), (uint32_t)(s[p] & 0xffffu), w0);
        cnt += c < 0 ? 1u : 0u;
        bad |= c > 0 ? 1u : 0u;
    }
    if (bad) atomicOr(err, 1u);
    uint32_t D;
    uint32_t r = block_excl_scan<THREADS>(cnt, s_warp, D);
    for (uint32_t p = p0; p < p1; ++p)
        if (p == 0 || key_cmp_k<NW>(k, (uint32_t)(s[p - 1] & 0xffffu), (uint32_t)(s[p] & 0xffffu), w0) < 0)
            s_hd[r++] = (HD)p;
    if (threadIdx.x == 0) s_hd[D] = (HD)n;
    __syncthreads();
    return D;
}

// ---------------------------------------------------------------- split

// Per coarse range b: fine splitters (pairs as in k_select), the 128-bit code
// windows of locate_coarse, its top-bits table, and flags of the slots that
// hold one repeated key.
// ms (at most kMaxSlots) is the slot capacity of one range.
struct SplitOut {
    uint64_t* spl;    // [nbk][ms - 1][NW]
    uint64_t* codes;  // [nbk][2][ms - 1]
    uint32_t* meta;   // [nbk][2]: splitter count, shared prefix length L
    uint16_t* top;    // [nbk][kTopStride]
    uint8_t* sflag;   // [nbk][ms]
    uint32_t ms;
};
constexpr uint32_t kTopStride = (1u << kTopBits) + 1u;

// One CTA per coarse range (grid stride).  A sample of the range's keys is
// gathered into skeys (this CTA's region), sorted in shared memory, and every
// (S/F)-th sample key becomes a splitter.  A key whose sample run fills a
// whole slot becomes the pair (key, key+1): the slot between holds that key
// only.  Later ranks inside the same run give (key+1, key+1), which keeps
// the splitters sorted.
template <class Src>
__global__ void __launch_bounds__(kSplThreads) k_slot_split(Src src, const uint32_t* __restrict__ rec,
                                                            const uint64_t* __restrict__ boff,
                                                            const uint8_t* __restrict__ bflags, uint32_t nbk,
                                                            uint32_t target, uint32_t ov, uint32_t fcap,
                                                            uint64_t seed, uint64_t* skeys_all, SplitOut o,
                                                            int32_t* err) {
    constexpr int NW = Src::NW;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_code = reinterpret_cast<uint64_t*>(smem);              // [kSampleMax] ordered sample
    uint16_t* s_hd = reinterpret_cast<uint16_t*>(s_code + kSampleMax);    // [kSampleMax + 1] run starts
    __shared__ OrderScratch so;
    __shared__ uint32_t s_warp[32];
    uint64_t* skeys = skeys_all + (size_t)blockIdx.x * kSampleMax * (NW + 2);
    const OrdAux aux{skeys + (size_t)kSampleMax * NW, skeys + (size_t)kSampleMax * (NW + 1)};
    for (uint32_t b = blockIdx.x; b < nbk; b += gridDim.x) {
        const uint64_t base = boff[b];
        const uint64_t N = boff[b + 1] - base;
        uint8_t* sflag = o.sflag + (size_t)b * o.ms;
        uint32_t F = (uint32_t)mn<uint64_t>((o.ms + 1) / 2, mn<uint64_t>(fcap, (N + target - 1) / target));
        if (F < 1) F = 1;
        const bool uni = bflags && bflags[b];
        if (uni || F == 1) {
            if (threadIdx.x == 0) {
                o.meta[2 * b] = 0;
                o.meta[2 * b + 1] = 0;
                sflag[0] = uni ? (uint8_t)LF_UNIFORM : (uint8_t)0;
            }
            continue;
        }
        const uint32_t S = (uint32_t)mn<uint64_t>(mn<uint64_t>(N, (uint64_t)F * ov), kSampleMax);
        const uint64_t step = N / S;  // >= 1
        for (uint32_t q = threadIdx.x; q < S; q += kSplThreads) {
            uint64_t pos = (uint64_t)q * N / S;
            if (step > 1) pos += mix64(seed ^ ((uint64_t)b << 20) ^ q) % step;
            uint64_t k[NW];
            src.key(rec[base + pos], k);
            key_store<NW>(skeys, q, k);
        }
        for (uint32_t q = threadIdx.x; q < 2 * F - 1; q += kSplThreads) sflag[q] = 0;
        __syncthreads();
        const GKeys<NW> gk{skeys};
        if (threadIdx.x == 0) so.s_err = 0;
        const uint32_t P = order_keys<NW, kSplThreads>(S, gk, s_code, aux, so);
        const uint32_t Dm = run_heads<NW, kSplThreads>(S, gk, s_code, (int)(P >> 6), s_hd, s_warp, &so.s_err);
        if (threadIdx.x == 0 && so.s_err) atomicOr(err, SE_ORDER_SPLIT);
        const uint32_t nsp = 2 * (F - 1);
        uint64_t* spl = o.spl + (size_t)b * (o.ms - 1) * NW;
        for (uint32_t t = 1 + threadIdx.x; t < F; t += kSplThreads) {
            const uint32_t tau = (uint32_t)(((uint64_t)t * S) / F);
            // run [a, e) of equal keys holding sorted position tau
            uint32_t lo = 0, len = Dm;
            while (len > 0) {
                const uint32_t half = len >> 1, mid = lo + half;
                if (s_hd[mid] <= tau) {
                    lo = mid + 1;
                    len -= half + 1;
                } else {
                    len = half;
                }
            }
            const uint32_t a = s_hd[lo - 1], e = s_hd[lo];
            const bool heavy = (uint64_t)(e - a) * F >= S;
            const uint32_t prev = (uint32_t)(((uint64_t)(t - 1) * S) / F);
            const bool repeat = heavy && t > 1 && prev >= a;  // rank t-1 lies in the same run
            uint64_t k[NW], k2[NW];
            key_load_g<NW>(skeys, s_code[tau] & 0xffffu, k);
            bool ok = true;
            if (heavy) ok = key_succ<NW>(k, k2);
            if (heavy && ok) {
                if (repeat) {
                    key_store<NW>(spl, 2 * (t - 1), k2);
                } else {
                    key_store<NW>(spl, 2 * (t - 1), k);
                    sflag[2 * t - 1] = (uint8_t)LF_UNIFORM;
                }
                key_store<NW>(spl, 2 * (t - 1) + 1, k2);
            } else {
                key_store<NW>(spl, 2 * (t - 1), k);
                key_store<NW>(spl, 2 * (t - 1) + 1, k);
                if (heavy) sflag[nsp] = (uint8_t)LF_UNIFORM;  // the largest key: the last slot
            }
        }
        __syncthreads();
        // code windows after the splitters' shared prefix (as k_spl_codes)
        uint64_t acc[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) acc[w] = 0;
        for (uint32_t t = threadIdx.x; t < nsp; t += kSplThreads)
#pragma unroll
            for (int w = 0; w < NW; ++w) acc[w] |= spl[(size_t)t * NW + w] ^ spl[w];
        const uint32_t L = block_first_diff<NW>(acc, so.s_or, &so.s_P);
        uint64_t* c1 = o.codes + (size_t)b * 2 * (o.ms - 1);
        uint64_t* sc1 = s_code;  // the sample order is no longer needed
        for (uint32_t t = threadIdx.x; t < nsp; t += kSplThreads) {
            uint64_t k[NW];
            key_load_g<NW>(spl, t, k);
            const uint64_t v1 = reg_bits64<NW>(k, L), v2 = reg_bits64<NW>(k, L + 64u);
            c1[t] = v1;
            c1[(o.ms - 1) + t] = v2;
            sc1[t] = v1;
        }
        __syncthreads();
        uint16_t* s_top = s_hd;  // the run starts are no longer needed
        build_top(sc1, nsp, s_top);
        __syncthreads();
        for (uint32_t v = threadIdx.x; v < kTopStride; v += kSplThreads) o.top[(size_t)b * kTopStride + v] = s_top[v];
        if (threadIdx.x == 0) {
            o.meta[2 * b] = nsp;
            o.meta[2 * b + 1] = L;
        }
        __syncthreads();
    }
}

// Chunks of the locate and place passes never cross a coarse range:
// cb[b] = first chunk of range b, cb[nbk] = number of chunks (single CTA).
static __global__ void __launch_bounds__(1024) k_slot_chunks(const uint64_t* __restrict__ boff, uint32_t nbk,
                                                             uint32_t* cb) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < nbk; base += 1024) {
        const uint32_t b = base + threadIdx.x;
        const uint32_t c = b < nbk ? (uint32_t)((boff[b + 1] - boff[b] + kChunkRecs - 1) / kChunkRecs) : 0u;
        uint32_t total;
        const uint32_t ex = block_excl_scan<1024>(c, s_warp, total);
        if (b < nbk) cb[b] = s_carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) cb[nbk] = s_carry;
}

// Range of chunk c: the b with cb[b] <= c < cb[b+1].
__device__ __forceinline__ uint32_t chunk_range(const uint32_t* __restrict__ cb, uint32_t nbk, uint32_t c) {
    uint32_t lo = 0, len = nbk;
    while (len > 0) {
        const uint32_t half = len >> 1, mid = lo + half;
        if (cb[mid + 1] <= c) {
            lo = mid + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo;
}

template <int NW>
constexpr size_t locate_smem() {
    return (size_t)(kMaxSlots - 1) * 16 + (size_t)NW * 8 + (size_t)kMaxSlots * 4 + (size_t)kTopStride * 2 + 16;
}

// Every record's slot: the number of fine splitters <= its key.  A CTA walks
// a contiguous run of chunks, so it reloads a range's splitter codes only
// when the range changes.
template <class Src>
__global__ void __launch_bounds__(kPartThreads, 2) k_slot_locate(Src src, const uint32_t* __restrict__ rec,
                                                                 const uint64_t* __restrict__ boff,
                                                                 const uint32_t* __restrict__ cb, uint32_t nbk,
                                                                 SplitOut o, uint16_t* sid, uint32_t* scount) {
    constexpr int NW = Src::NW;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_c1 = reinterpret_cast<uint64_t*>(smem);
    uint64_t* s_c2 = s_c1 + (kMaxSlots - 1);
    uint64_t* s_p0 = s_c2 + (kMaxSlots - 1);
    uint32_t* s_hist = reinterpret_cast<uint32_t*>(s_p0 + NW);
    uint16_t* s_top = reinterpret_cast<uint16_t*>(s_hist + kMaxSlots);
    const uint32_t nch = cb[nbk];
    const uint32_t per = (nch + gridDim.x - 1) / gridDim.x;
    const uint32_t c0 = blockIdx.x * per, c1e = mn<uint32_t>(nch, c0 + per);
    uint32_t cur = 0xffffffffu, nsp = 0, L = 0;
    const uint64_t* spl = nullptr;
    for (uint32_t c = c0; c < c1e; ++c) {
        const uint32_t b = chunk_range(cb, nbk, c);
        __syncthreads();
        if (b != cur) {
            cur = b;
            nsp = o.meta[2 * b];
            L = o.meta[2 * b + 1];
            spl = o.spl + (size_t)b * (o.ms - 1) * NW;
            const uint64_t* cc = o.codes + (size_t)b * 2 * (o.ms - 1);
            for (uint32_t q = threadIdx.x; q < nsp; q += kPartThreads) {
                s_c1[q] = cc[q];
                s_c2[q] = cc[(o.ms - 1) + q];
            }
            if (nsp)
                for (uint32_t q = threadIdx.x; q < kTopStride; q += kPartThreads)
                    s_top[q] = o.top[(size_t)b * kTopStride + q];
            for (uint32_t q = threadIdx.x; q < (uint32_t)NW; q += kPartThreads) s_p0[q] = nsp ? spl[q] : 0ull;
        }
        for (uint32_t q = threadIdx.x; q <= nsp; q += kPartThreads) s_hist[q] = 0;
        __syncthreads();
        const uint64_t start = boff[b] + (uint64_t)(c - cb[b]) * kChunkRecs;
        const uint64_t end = mn<uint64_t>(start + kChunkRecs, boff[b + 1]);
        for (uint64_t p = start + threadIdx.x; p < end; p += kPartThreads) {
            uint32_t id = 0;
            if (nsp) {
                uint64_t k[NW];
                src.key(rec[p], k);
                id = locate_coarse<NW>(k, s_c1, s_c2, s_p0, nsp, L, spl, s_top);
            }
            sid[p] = (uint16_t)id;
            atomicAdd(&s_hist[id], 1u);
        }
        __syncthreads();
        for (uint32_t q = threadIdx.x; q <= nsp; q += kPartThreads)
            if (s_hist[q]) atomicAdd(&scount[(size_t)b * o.ms + q], s_hist[q]);
    }
}

// Per coarse range: slot offsets (absolute term positions, also the place
// pass's cursors) and the packing of consecutive slots into leaves of at
// most `cap` terms.  A slot of one repeated key, or one above cap, is a leaf
// of its own.  Leaves go to ldesc[b][..], their count to nleaf[b].
static __global__ void __launch_bounds__(1024) k_slot_offsets(const uint64_t* __restrict__ boff, uint32_t nbk,
                                                              uint32_t ms, const uint32_t* __restrict__ meta,
                                                              const uint32_t* __restrict__ scount,
                                                              const uint8_t* __restrict__ sflag, uint32_t cap,
                                                              uint64_t* soff, Leaf* ldesc, uint32_t* nleaf) {
    __shared__ uint32_t s_cnt[kMaxSlots];
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_ex[kMaxSlots];
    for (uint32_t b = blockIdx.x; b < nbk; b += gridDim.x) {
        const uint32_t ns = meta[2 * b] + 1;
        for (uint32_t q = threadIdx.x; q < ns; q += 1024) s_cnt[q] = scount[(size_t)b * ms + q];
        __syncthreads();
        // exclusive scan, four slots per thread
        const uint32_t q0 = 4 * threadIdx.x;
        uint32_t loc = 0;
        for (uint32_t q = q0; q < q0 + 4 && q < ns; ++q) loc += s_cnt[q];
        uint32_t tot;
        uint32_t ex = block_excl_scan<1024>(loc, s_warp, tot);
        for (uint32_t q = q0; q < q0 + 4 && q < ns; ++q) {
            s_ex[q] = ex;
            soff[(size_t)b * ms + q] = boff[b] + ex;
            ex += s_cnt[q];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            Leaf* ld = ldesc + (size_t)b * ms;
            uint32_t nl = 0, cn = 0;
            uint64_t co = 0;
            for (uint32_t q = 0; q < ns; ++q) {
                const uint32_t c = s_cnt[q];
                if (c == 0) continue;
                const uint32_t f = sflag[(size_t)b * ms + q];
                const uint64_t off = boff[b] + s_ex[q];
                if ((f & LF_UNIFORM) || c > cap) {
                    if (cn) ld[nl++] = Leaf{co, cn, 0u};
                    cn = 0;
                    ld[nl++] = Leaf{off, c, (f & LF_UNIFORM) ? LF_UNIFORM : LF_OVERSIZE};
                    continue;
                }
                if (cn + c > cap) {
                    ld[nl++] = Leaf{co, cn, 0u};
                    cn = 0;
                }
                if (cn == 0) co = off;
                cn += c;
            }
            if (cn) ld[nl++] = Leaf{co, cn, 0u};
            nleaf[b] = nl;
        }
        __syncthreads();
    }
}

// Leaf numbering in key order: lbase[b] = leaves before range b; lbase[nbk]
// is the total (single CTA).
static __global__ void __launch_bounds__(1024) k_slot_leafscan(const uint32_t* __restrict__ nleaf, uint32_t nbk,
                                                               uint32_t* lbase) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < nbk; base += 1024) {
        const uint32_t b = base + threadIdx.x;
        const uint32_t c = b < nbk ? nleaf[b] : 0u;
        uint32_t total;
        const uint32_t ex = block_excl_scan<1024>(c, s_warp, total);
        if (b < nbk) lbase[b] = s_carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) lbase[nbk] = s_carry;
}

static __global__ void k_slot_leafcopy(const Leaf* __restrict__ ldesc, const uint32_t* __restrict__ nleaf,
                                       const uint32_t* __restrict__ lbase, uint32_t nbk, uint32_t ms, Leaf* leaves) {
    for (uint32_t b = blockIdx.x; b < nbk; b += gridDim.x)
        for (uint32_t q = threadIdx.x; q < nleaf[b]; q += blockDim.x)
            leaves[lbase[b] + q] = ldesc[(size_t)b * ms + q];
}

__device__ __forceinline__ void store_cs(double2* p, double2 v) { __stcs(p, v); }
__device__ __forceinline__ void store_cs(float2* p, float2 v) { __stcs(p, v); }

// Forms every record's term (key, and coefficient with the phase folded in)
// once and writes it into its slot.  Per chunk: count the records of each
// slot, take each slot's places with one atomic per (chunk, slot), then place.
template <class Src, class VT>
__global__ void __launch_bounds__(kPartThreads, 2) k_slot_place(Src src, const uint32_t* __restrict__ rec,
                                                                const uint64_t* __restrict__ boff,
                                                                const uint32_t* __restrict__ cb, uint32_t nbk,
                                                                uint32_t ms, const uint32_t* __restrict__ meta,
                                                                const uint16_t* __restrict__ sid,
                                                                unsigned long long* cursor, uint64_t* tkeys,
                                                                VT* tvals) {
    constexpr int NW = Src::NW;
    __shared__ uint32_t s_cnt[kMaxSlots];
    __shared__ unsigned long long s_base[kMaxSlots];
    // chunks in range order across the grid: all CTAs fill the slots of the
    // same one or two ranges at a time, so every slot's partly written lines
    // stay in L2 until they are complete
    const uint32_t nch = cb[nbk];
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
        const uint32_t b = chunk_range(cb, nbk, c);
        const uint32_t ns = meta[2 * b] + 1;
        __syncthreads();
        for (uint32_t q = threadIdx.x; q < ns; q += kPartThreads) s_cnt[q] = 0;
        __syncthreads();
        const uint64_t start = boff[b] + (uint64_t)(c - cb[b]) * kChunkRecs;
        const uint64_t end = mn<uint64_t>(start + kChunkRecs, boff[b + 1]);
        for (uint64_t p = start + threadIdx.x; p < end; p += kPartThreads) atomicAdd(&s_cnt[sid[p]], 1u);
        __syncthreads();
        for (uint32_t q = threadIdx.x; q < ns; q += kPartThreads) {
            const uint32_t n = s_cnt[q];
            s_base[q] = n ? atomicAdd(cursor + (size_t)b * ms + q, (unsigned long long)n) : 0ull;
            s_cnt[q] = 0;
        }
        __syncthreads();
        for (uint64_t p = start + threadIdx.x; p < end; p += kPartThreads) {
            const uint32_t id = sid[p];
            const uint64_t d = s_base[id] + atomicAdd(&s_cnt[id], 1u);
            uint64_t k[NW];
            const VT v = src.value(rec[p], k);
            // evict-first stores: the 16*WP+16 bytes per record stream
            // through L2 without pushing out the factor tables the
            // gathers read
            ulonglong2* kp = reinterpret_cast<ulonglong2*>(tkeys + d * NW);
#pragma unroll
            for (int q = 0; q < NW / 2; ++q) __stcs(kp + q, make_ulonglong2(k[2 * q], k[2 * q + 1]));
            store_cs(tvals + d, v);
        }
    }
}


// ---------------------------------------------------------------- leaves

// Upper bound of one look-back wait: the leaves before this one are running
// on resident CTAs, so a longer wait means a fault elsewhere.
constexpr uint64_t kWaitNs = 4000000000ull;
constexpr uint32_t kMaxSpins = 1u << 26;

__device__ __forceinline__ void st_release(uint64_t* p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_acquire(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Decoupled look-back (warp 0): the number of merged terms of all leaves
// before leaf t.  Lane l reads the status of leaf g - l; aggregates are added
// until the nearest inclusive prefix.  Returns false when the wait runs out.
static __device__ bool look_back(const uint64_t* status, uint32_t t, uint64_t& excl) {
    const uint32_t lane = threadIdx.x & 31u;
    excl = 0;
    int64_t g = (int64_t)t - 1;
    const uint64_t t0 = gtimer();
    uint32_t spins = 0;
    while (g >= 0) {
        const int64_t idx = g - (int64_t)lane;
        uint64_t v = idx >= 0 ? ld_acquire(status + idx) : kIncl;
        while (__any_sync(0xffffffffu, v == 0ull)) {
            if (v == 0ull) v = ld_acquire(status + idx);
            if (((++spins) & 31u) == 0u) {
                const bool late = spins > kMaxSpins || gtimer() - t0 > kWaitNs;
                if (__any_sync(0xffffffffu, late)) return false;
                __nanosleep(128);
            }
        }
        const uint32_t im = __ballot_sync(0xffffffffu, (v & kIncl) != 0ull);
        uint64_t c = v & kValMask;
        if (im && lane > (uint32_t)(__ffs(im) - 1)) c = 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        excl += c;
        if (im) break;
        g -= 32;
    }
    return true;
}

template <int MODE>
__device__ Acc<MODE> block_reduce_acc(Acc<MODE> a, Acc<MODE>* s_acc) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a.shfl_merge(o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_acc[threadIdx.x >> 5] = a;
    __syncthreads();
    Acc<MODE> r;
    if (threadIdx.x == 0) {
        r = s_acc[0];
        for (uint32_t w = 1; w < blockDim.x / 32; ++w) r.merge(s_acc[w]);
    }
    return r;
}

// Shared-memory layout of a leaf CTA (two CTAs per SM).
template <int NW, int MODE>
struct LeafLayout {
    using VT = typename ValT<MODE>::T;
    static constexpr uint32_t CAP = cap<NW>();
    static constexpr uint32_t N2 = pow2_at_least(CAP);
    static constexpr size_t KEY = 0;
    static constexpr size_t VAL = KEY + (size_t)NW * CAP * 8;
    static constexpr size_t C2 = VAL + (((size_t)CAP * sizeof(VT) + 15) & ~(size_t)15);
    static constexpr size_t HSH = C2 + (size_t)CAP * 8;
    static constexpr size_t SRT = HSH + (size_t)CAP * 8;
    static constexpr size_t HD = SRT + (size_t)N2 * 8;
    static constexpr size_t SUB = HD + ((((size_t)CAP + 1) * 2 + 15) & ~(size_t)15);
    static constexpr size_t SUBF = SUB + (size_t)2 * kSubMax * NW * 8;
    static constexpr size_t BYTES = SUBF + 2 * kSubMax;
    static_assert(BYTES <= 111 * 1024, "two leaf CTAs per SM");
};

struct LeafMisc {
    OrderScratch o;
    uint32_t s_warp[32];
    uint32_t s_t, s_cnt, s_ok;
    uint64_t s_excl;
};

// Orders the n terms staged in shared memory (keys word-major, stride CAP)
// by full key and finds the runs of equal keys.  Leaves s_srt[0, n) ordered
// (element = code | index) and s_hd[r] = first sorted position of distinct
// key r, s_hd[D] = n.  Returns D.  An order the whole-key check rejects sets
// m.o.s_err.  Whole CTA.
template <int NW, int MODE>
__device__ uint32_t leaf_order(uint32_t n, const uint64_t* s_key, const OrdAux& aux, uint64_t* s_srt,
                               uint16_t* s_hd, LeafMisc& m) {
    using LL = LeafLayout<NW, MODE>;
    const SKeys sk{s_key, LL::CAP};
    const uint32_t P = order_keys<NW, kLeafThreads>(n, sk, s_srt, aux, m.o);
    return run_heads<NW, kLeafThreads>(n, sk, s_srt, (int)(P >> 6), s_hd, m.s_warp, &m.o.s_err);
}

// Writes merged term d (of D) at output position obase + d: the key of its
// first sorted element, the sum of the run's values in sorted order.
template <int NW, int MODE>
__device__ void leaf_write(uint32_t D, uint64_t obase, const uint64_t* s_key,
                           const typename ValT<MODE>::T* s_val, const uint64_t* s_srt, const uint16_t* s_hd,
                           uint64_t* okeys, double2* ocoef, uint8_t* opb) {
    using LL = LeafLayout<NW, MODE>;
    for (uint32_t d = threadIdx.x; d < D; d += kLeafThreads) {
        const uint32_t a = s_hd[d], e = s_hd[d + 1];
        Acc<MODE> acc;
        for (uint32_t p = a; p < e; ++p) acc.add(s_val[s_srt[p] & 0xffffu]);
        const uint32_t i0 = (uint32_t)(s_srt[a] & 0xffffu);
        uint64_t k[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) k[w] = s_key[(size_t)w * LL::CAP + i0];
        const uint64_t u = obase + d;
        key_store<NW>(okeys, u, k);
        ocoef[u] = acc.result();
        opb[u] = (uint8_t)normal_phase<NW / 2>(k, 0u);
    }
}

// Register key against word-major shared key j: -1, 0, 1.
template <int NW>
__device__ __forceinline__ int cmp_rs(const uint64_t (&k)[NW], const uint64_t* s, uint32_t stride, uint32_t j) {
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const uint64_t v = s[(size_t)w * stride + j];
        if (k[w] != v) return k[w] < v ? -1 : 1;
    }
    return 0;
}

// Leaves in key order, taken from a ticket counter.  A leaf of at most cap
// terms stages them in shared memory, orders them, publishes its distinct
// count D, learns the count before it by look-back, then writes its merged
// terms.  A leaf of one repeated key is reduced.  A larger leaf (one
// oversized slot) is ordered in sub-ranges chosen from a sample of its keys;
// it takes its offset first and publishes after its last write, and it needs
// its whole output to land below its own terms (else SE_OVERLAP and the host
// uses the range-sort pipeline).
template <int NW, int MODE>
__global__ void __launch_bounds__(kLeafThreads, 2) k_slot_leaf(const Leaf* __restrict__ leaves,
                                                               const uint32_t* __restrict__ nleaves_p,
                                                               uint32_t* ticket, uint64_t* status, uint64_t* keys,
                                                               const typename ValT<MODE>::T* vals, double2* ocoef,
                                                               uint8_t* opb, uint64_t* total, int32_t* err,
                                                               uint32_t capr) {
    using LL = LeafLayout<NW, MODE>;
    using VT = typename ValT<MODE>::T;
    constexpr uint32_t CAP = LL::CAP;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_key = reinterpret_cast<uint64_t*>(smem + LL::KEY);
    VT* s_val = reinterpret_cast<VT*>(smem + LL::VAL);
    uint64_t* s_srt = reinterpret_cast<uint64_t*>(smem + LL::SRT);
    uint16_t* s_hd = reinterpret_cast<uint16_t*>(smem + LL::HD);
    uint64_t* s_sub = reinterpret_cast<uint64_t*>(smem + LL::SUB);
    uint8_t* s_subf = smem + LL::SUBF;
    const OrdAux aux{reinterpret_cast<uint64_t*>(smem + LL::C2), reinterpret_cast<uint64_t*>(smem + LL::HSH)};
    __shared__ LeafMisc m;
    __shared__ Acc<MODE> s_acc[kLeafThreads / 32];
    __shared__ double2 s_red;
    const uint32_t nl = *nleaves_p;
    const bool lead = threadIdx.x < 32;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            m.s_t = atomicAdd(ticket, 1u);
            m.o.s_err = 0;
        }
        __syncthreads();
        const uint32_t t = m.s_t;
        if (t >= nl) break;
        const Leaf L = leaves[t];
        const uint64_t bound = L.off + L.n;  // a count no correct prefix can exceed
        uint64_t incl = bound;
        if (L.flags & LF_UNIFORM) {
            Acc<MODE> a;
            for (uint32_t i = threadIdx.x; i < L.n; i += kLeafThreads) a.add(vals[L.off + i]);
            a = block_reduce_acc<MODE>(a, s_acc);
            if (threadIdx.x < (uint32_t)NW) s_key[(size_t)threadIdx.x * CAP] = keys[L.off * NW + threadIdx.x];
            if (threadIdx.x == 0) s_red = a.result();
            __syncthreads();  // every read of this leaf's terms is done
            if (threadIdx.x == 0) st_release(status + t, kAgg | 1ull);
            if (lead) {
                uint64_t ex;
                const bool ok = look_back(status, t, ex);
                if (threadIdx.x == 0) {
                    m.s_ok = ok && ex + 1 <= bound;
                    if (!ok) atomicOr(err, SE_TIMEOUT);
                    else if (!m.s_ok) atomicOr(err, SE_BOUNDS);
                    m.s_excl = ex;
                    incl = m.s_ok ? ex + 1 : bound;
                    st_release(status + t, kIncl | incl);
                }
            }
            __syncthreads();
            if (threadIdx.x == 0 && m.s_ok) {
                uint64_t k[NW];
#pragma unroll
                for (int w = 0; w < NW; ++w) k[w] = s_key[(size_t)w * CAP];
                key_store<NW>(keys, m.s_excl, k);
                ocoef[m.s_excl] = s_red;
                opb[m.s_excl] = (uint8_t)normal_phase<NW / 2>(k, 0u);
            }
        } else if (L.n <= capr) {
            const uint32_t n = L.n;
            for (uint32_t i = threadIdx.x; i < n; i += kLeafThreads) {
                uint64_t k[NW];
                key_load_g<NW>(keys, L.off + i, k);
#pragma unroll
                for (int w = 0; w < NW; ++w) s_key[(size_t)w * CAP + i] = k[w];
                s_val[i] = vals[L.off + i];
            }
            __syncthreads();
            const uint32_t D = leaf_order<NW, MODE>(n, s_key, aux, s_srt, s_hd, m);
            if (threadIdx.x == 0 && m.o.s_err) atomicOr(err, SE_ORDER);
            if (threadIdx.x == 0) st_release(status + t, kAgg | D);
            if (lead) {
                uint64_t ex;
                const bool ok = look_back(status, t, ex);
                if (threadIdx.x == 0) {
                    m.s_ok = ok && ex + D <= bound;
                    if (!ok) atomicOr(err, SE_TIMEOUT);
                    else if (!m.s_ok) atomicOr(err, SE_BOUNDS);
                    m.s_excl = ex;
                    incl = m.s_ok ? ex + D : bound;
                    st_release(status + t, kIncl | incl);
                }
            }
            __syncthreads();
            if (m.s_ok) leaf_write<NW, MODE>(D, m.s_excl, s_key, s_val, s_srt, s_hd, keys, ocoef, opb);
        } else {
            // ---- one oversized slot: offset first, then sub-ranges
            const uint32_t n = L.n;
            if (lead) {
                uint64_t ex;
                const bool ok = look_back(status, t, ex);
                if (threadIdx.x == 0) {
                    m.s_ok = ok && ex + n <= L.off;  // the whole output stays below these terms
                    if (!ok) atomicOr(err, SE_TIMEOUT);
                    else if (!m.s_ok) atomicOr(err, SE_OVERLAP);
                    m.s_excl = ex;
                }
            }
            __syncthreads();
            uint64_t done = 0;
            bool good = m.s_ok;
            if (good) {
                // sample: capr keys at evenly spread positions, ordered
                const uint32_t ms = capr;
                for (uint32_t i = threadIdx.x; i < ms; i += kLeafThreads) {
                    uint64_t k[NW];
                    key_load_g<NW>(keys, L.off + (uint64_t)i * n / ms, k);
#pragma unroll
                    for (int w = 0; w < NW; ++w) s_key[(size_t)w * CAP + i] = k[w];
                }
                __syncthreads();
                const uint32_t Dm = leaf_order<NW, MODE>(ms, s_key, aux, s_srt, s_hd, m);
                const uint32_t q = (uint32_t)mn<uint64_t>(kSubMax, mn<uint64_t>(ms, (uint64_t)n * 4 / (3ull * capr) + 1));
                const uint32_t nsub = 2 * (q - 1);
                for (uint32_t j = threadIdx.x; j <= nsub; j += kLeafThreads) s_subf[j] = 0;
                __syncthreads();
                for (uint32_t t2 = 1 + threadIdx.x; t2 < q; t2 += kLeafThreads) {
                    const uint32_t tau = (uint32_t)(((uint64_t)t2 * ms) / q);
                    uint32_t lo = 0, len = Dm;  // run r with s_hd[r] <= tau < s_hd[r+1]
                    while (len > 0) {
                        const uint32_t half = len >> 1, mid = lo + half;
                        if (s_hd[mid] <= tau) {
                            lo = mid + 1;
                            len -= half + 1;
                        } else {
                            len = half;
                        }
                    }
                    const uint32_t r = lo - 1, a = s_hd[r], e = s_hd[r + 1];
                    const bool heavy = (uint64_t)(e - a) * q >= ms;
                    const uint32_t prev = (uint32_t)(((uint64_t)(t2 - 1) * ms) / q);
                    const bool repeat = heavy && t2 > 1 && prev >= a;
                    uint64_t k[NW], k2[NW];
                    const uint32_t i0 = (uint32_t)(s_srt[tau] & 0xffffu);
#pragma unroll
                    for (int w = 0; w < NW; ++w) k[w] = s_key[(size_t)w * CAP + i0];
                    const bool ok = heavy ? key_succ<NW>(k, k2) : true;
                    const uint32_t j0 = 2 * (t2 - 1);
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        const uint64_t lo_w = (heavy && ok && repeat) ? k2[w] : k[w];
                        const uint64_t hi_w = (heavy && ok) ? k2[w] : k[w];
                        s_sub[(size_t)w * 2 * kSubMax + j0] = lo_w;
                        s_sub[(size_t)w * 2 * kSubMax + j0 + 1] = hi_w;
                    }
                    if (heavy && ok && !repeat) s_subf[j0 + 1] = 1;
                    if (heavy && !ok) s_subf[nsub] = 1;
                }
                __syncthreads();
                constexpr uint32_t SS = 2 * kSubMax;
                for (uint32_t j = 0; j <= nsub && good; ++j) {
                    // sub-range j is [s_sub[j-1], s_sub[j]) (open at the ends)
                    const bool uni = s_subf[j] != 0;
                    __syncthreads();
                    if (threadIdx.x == 0) m.s_cnt = 0;
                    __syncthreads();
                    Acc<MODE> a;
                    for (uint32_t i = threadIdx.x; i < n; i += kLeafThreads) {
                        uint64_t k[NW];
                        key_load_g<NW>(keys, L.off + i, k);
                        const bool in = (j == 0 || cmp_rs<NW>(k, s_sub, SS, j - 1) >= 0) &&
                                        (j == nsub || cmp_rs<NW>(k, s_sub, SS, j) < 0);
                        if (!in) continue;
                        if (uni) {
                            a.add(vals[L.off + i]);
                            atomicAdd(&m.s_cnt, 1u);
                            continue;
                        }
                        const uint32_t c = atomicAdd(&m.s_cnt, 1u);
                        if (c < capr) {
#pragma unroll
                            for (int w = 0; w < NW; ++w) s_key[(size_t)w * CAP + c] = k[w];
                            s_val[c] = vals[L.off + i];
                        }
                    }
                    if (uni) {
                        a = block_reduce_acc<MODE>(a, s_acc);
                        const uint32_t c = m.s_cnt;
                        if (threadIdx.x == 0 && c) {
                            uint64_t k[NW];
#pragma unroll
                            for (int w = 0; w < NW; ++w) k[w] = s_sub[(size_t)w * SS + (j - 1)];
                            const uint64_t u = m.s_excl + done;
                            key_store<NW>(keys, u, k);
                            ocoef[u] = a.result();
                            opb[u] = (uint8_t)normal_phase<NW / 2>(k, 0u);
                        }
                        done += c ? 1 : 0;
                        __syncthreads();
                        continue;
                    }
                    __syncthreads();
                    const uint32_t c = m.s_cnt;
                    if (c > capr) {
                        good = false;
                        if (threadIdx.x == 0) atomicOr(err, SE_SUBRANGE);
                        break;
                    }
                    if (c == 0) continue;
                    const uint32_t Dj = leaf_order<NW, MODE>(c, s_key, aux, s_srt, s_hd, m);
                    leaf_write<NW, MODE>(Dj, m.s_excl + done, s_key, s_val, s_srt, s_hd, keys, ocoef, opb);
                    done += Dj;
                    __syncthreads();
                }
            }
            __syncthreads();
            if (threadIdx.x == 0 && m.o.s_err) atomicOr(err, SE_ORDER);
            incl = good ? m.s_excl + done : bound;
            if (threadIdx.x == 0) st_release(status + t, kIncl | incl);
        }
        if (t == nl - 1 && threadIdx.x == 0) *total = incl;
    }
}


}  // namespace slot

// ---------------------------------------------------------------- host

// Canonical form by slot sort.  Returns nullptr (after freeing what it made)
// when the device reports a case this method leaves to the range-sort
// pipeline: an oversized slot whose output could reach its own terms, a
// sub-range above a leaf, or an expired wait.
template <class Src, int MODE>
static paulib_sum* slot_canonical(const Src& src, uint32_t R, uint32_t nb_terms, int32_t n_qubits,
                                  cudaStream_t st) {
    using namespace slot;
    constexpr int NW = Src::NW;
    using VT = typename ValT<MODE>::T;
    const int sms = device_sm_count();
    const SlotTuning tn = slot_tuning_for(NW);
    const uint32_t capr = tn.leaf_cap > 0 ? std::min<uint32_t>((uint32_t)tn.leaf_cap, cap<NW>()) : cap<NW>();
    const uint32_t target = std::max<uint32_t>(1u, tn.target > 0 ? (uint32_t)tn.target : capr / 5u);
    const uint32_t ov = tn.oversample > 0 ? (uint32_t)tn.oversample : 8u;
    uint64_t Reff = R;
    if constexpr (IsProd<Src>::value) {
        if (src.sym) Reff = (uint64_t)src.na * (src.na + 1) / 2;
    }
    Scratch err(4, st);
    check_cuda(cudaMemsetAsync(err.p, 0, 4, st), "memset err");
    Scratch recA((size_t)Reff * 4, st), subid((size_t)R * 2, st);
    Scratch boff_s, bflags_s;
    const Tuning tune = tuning_for(NW);
    const uint64_t C1 = (uint64_t)target * 1024u;
    const uint32_t nbk = level1_partition<Src, MODE>(src, R, nb_terms, C1, 2048u, tune.oversample,
                                                     tune.count_ctas_per_sm, st, recA.as<uint32_t>(),
                                                     subid.as<uint16_t>(), boff_s, bflags_s, err.as<int32_t>());
    const uint64_t B1 = (nbk + 1) / 2;
    const uint64_t avg = (Reff + B1 - 1) / B1;
    const uint32_t fcap = (uint32_t)std::max<uint64_t>(
        2, std::min<uint64_t>(kFmax, 3 * ((avg + target - 1) / target) + 1));
    const uint32_t ms = 2 * fcap - 1;
    Scratch spl((size_t)nbk * (ms - 1) * NW * 8, st), codes((size_t)nbk * 2 * (ms - 1) * 8, st),
        meta((size_t)nbk * 8, st), top((size_t)nbk * kTopStride * 2, st), sflag((size_t)nbk * ms, st);
    SplitOut so{spl.as<uint64_t>(), codes.as<uint64_t>(), meta.as<uint32_t>(), top.as<uint16_t>(),
                sflag.as<uint8_t>(), ms};
    Scratch cb((size_t)(nbk + 1) * 4, st), scount((size_t)nbk * ms * 4, st);
    uint16_t* sid = subid.as<uint16_t>();  // level-1 ids are dead after the scatter
    {
        StageScope ss(ST_SPLIT, st);
        const unsigned gsplit = (unsigned)std::min<uint32_t>(nbk, (uint32_t)sms);
        Scratch skeys((size_t)gsplit * kSampleMax * (NW + 2) * 8, st);
        const size_t smem = (size_t)kSampleMax * 8 + (size_t)(kSampleMax + 8) * 2 + 16;
        auto ks = k_slot_split<Src>;
        smem_attr(ks, smem);
        note_launch(ST_SPLIT);
        ks<<<gsplit, kSplThreads, smem, st>>>(src, recA.as<uint32_t>(), boff_s.as<uint64_t>(),
                                              bflags_s.as<uint8_t>(), nbk, target, ov, fcap,
                                              g_sample_seed ^ 0x51075eedull, skeys.as<uint64_t>(), so,
                                              err.as<int32_t>());
        check_cuda(cudaGetLastError(), "k_slot_split");
        note_launch(ST_SPLIT);
        k_slot_chunks<<<1, 1024, 0, st>>>(boff_s.as<uint64_t>(), nbk, cb.as<uint32_t>());
        check_cuda(cudaMemsetAsync(scount.p, 0, (size_t)nbk * ms * 4, st), "memset slot counts");
        auto kl = k_slot_locate<Src>;
        smem_attr(kl, locate_smem<NW>());
        note_launch(ST_SPLIT);
        kl<<<(unsigned)sms * 2, kPartThreads, locate_smem<NW>(), st>>>(src, recA.as<uint32_t>(),
                                                                       boff_s.as<uint64_t>(), cb.as<uint32_t>(),
                                                                       nbk, so, sid, scount.as<uint32_t>());
        check_cuda(cudaGetLastError(), "k_slot_locate");
    }
    const uint64_t lcap = std::min<uint64_t>(Reff, (uint64_t)nbk * ms);
    Scratch soff((size_t)nbk * ms * 8, st), ldesc((size_t)nbk * ms * sizeof(Leaf), st),
        nleaf((size_t)nbk * 4, st), lbase((size_t)(nbk + 1) * 4, st), leaves((size_t)lcap * sizeof(Leaf), st);
    paulib_sum* out = sum_alloc(n_qubits, (int64_t)Reff, false, st);
    try {
        Scratch vf;
        VT* tvals;
        if constexpr (MODE == M_FP64) {
            tvals = out->coef;
        } else {
            vf = Scratch((size_t)Reff * sizeof(VT), st);
            tvals = vf.as<VT>();
        }
        {
            StageScope ss(ST_PLACE, st);
            note_launch(ST_PLACE);
            k_slot_offsets<<<std::min<uint32_t>(nbk, (uint32_t)sms * 2), 1024, 0, st>>>(
                boff_s.as<uint64_t>(), nbk, ms, meta.as<uint32_t>(), scount.as<uint32_t>(), sflag.as<uint8_t>(),
                capr, soff.as<uint64_t>(), ldesc.as<Leaf>(), nleaf.as<uint32_t>());
            note_launch(ST_PLACE);
            k_slot_leafscan<<<1, 1024, 0, st>>>(nleaf.as<uint32_t>(), nbk, lbase.as<uint32_t>());
            note_launch(ST_PLACE);
            k_slot_leafcopy<<<std::min<uint32_t>(nbk, (uint32_t)sms * 4), 256, 0, st>>>(
                ldesc.as<Leaf>(), nleaf.as<uint32_t>(), lbase.as<uint32_t>(), nbk, ms, leaves.as<Leaf>());
            note_launch(ST_PLACE);
            k_slot_place<Src, VT><<<(unsigned)sms * 2, kPartThreads, 0, st>>>(
                src, recA.as<uint32_t>(), boff_s.as<uint64_t>(), cb.as<uint32_t>(), nbk, ms, meta.as<uint32_t>(),
                sid, reinterpret_cast<unsigned long long*>(soff.as<uint64_t>()), out->keys, tvals);
            check_cuda(cudaGetLastError(), "slot placement");
        }
        Scratch status((size_t)lcap * 8, st), misc(16, st);
        check_cuda(cudaMemsetAsync(status.p, 0, (size_t)lcap * 8, st), "memset status");
        check_cuda(cudaMemsetAsync(misc.p, 0, 16, st), "memset ticket");
        {
            StageScope ss(ST_LEAF, st);
            using LL = LeafLayout<NW, MODE>;
            auto kf = k_slot_leaf<NW, MODE>;
            smem_attr(kf, LL::BYTES);
            note_launch(ST_LEAF);
            kf<<<(unsigned)sms * 2, slot::kLeafThreads, LL::BYTES, st>>>(
                leaves.as<Leaf>(), lbase.as<uint32_t>() + nbk, misc.as<uint32_t>(), status.as<uint64_t>(),
                out->keys, tvals, out->coef, out->pbase, misc.as<uint64_t>() + 1, err.as<int32_t>(), capr);
            check_cuda(cudaGetLastError(), "k_slot_leaf");
        }
        struct { uint64_t u; int32_t e; uint32_t nl; } h{};
        check_cuda(cudaMemcpyAsync(&h.u, misc.as<uint64_t>() + 1, 8, cudaMemcpyDeviceToHost, st), "U copy");
        check_cuda(cudaMemcpyAsync(&h.e, err.p, 4, cudaMemcpyDeviceToHost, st), "err copy");
        check_cuda(cudaMemcpyAsync(&h.nl, lbase.as<uint32_t>() + nbk, 4, cudaMemcpyDeviceToHost, st), "leaf count");
        check_cuda(cudaStreamSynchronize(st), "slot sort sync");
        note_canon_stats(nbk, ms, h.nl, capr, target);
        if (h.e & (SE_OVERLAP | SE_SUBRANGE | SE_TIMEOUT | SE_ORDER | SE_ORDER_SPLIT)) {
            sum_free(out, st);
            note_canon_method(1, h.e);
            return nullptr;
        }
        if (h.e) fail(PAULIB_ERR_INTERNAL, "slot sort failed on device (error word " + std::to_string(h.e) + ")");
        out->n_terms = (int64_t)h.u;
        out->is_canonical = 1;
        note_canon_method(0, 0);
        return out;
    } catch (...) {
        sum_free(out, st);
        throw;
    }
}

// Canonical form of the records of src: the slot sort, or the range-sort
// pipeline when tuning asks for it or the slot sort hands the case back.
template <class Src, int MODE>
static paulib_sum* finish_canonical(const Src& src, uint32_t R, uint32_t nb_terms, int32_t n_qubits,
                                    cudaStream_t st) {
    if (slot_tuning_for(Src::NW).method == 0) {
        paulib_sum* r = slot_canonical<Src, MODE>(src, R, nb_terms, n_qubits, st);
        if (r) return r;
    } else {
        note_canon_method(1, 0);
    }
    return finish<Src, MODE>(src, R, nb_terms, n_qubits, st);
}

template <int WP, int MODE>
static paulib_sum* product_mode(const paulib_sum* a, const paulib_sum* b, cudaStream_t st) {
    using Src = ProdSrc<WP, MODE>;
    using V = typename Src::V;
    const uint32_t R = (uint32_t)(a->n_terms * b->n_terms);
    Scratch fa, fb;
    const V* ac;
    const V* bc;
    if constexpr (MODE == M_FP64) {
        ac = reinterpret_cast<const V*>(a->coef);
        bc = reinterpret_cast<const V*>(b->coef);
    } else {
        fa = Scratch((size_t)a->n_terms * 8, st);
        fb = Scratch((size_t)b->n_terms * 8, st);
        StageScope ss(ST_CONVERT, st);
        k_to_f32<MODE><<<(unsigned)((a->n_terms + 255) / 256), 256, 0, st>>>(a->coef, fa.as<float2>(), a->n_terms);
        k_to_f32<MODE><<<(unsigned)((b->n_terms + 255) / 256), 256, 0, st>>>(b->coef, fb.as<float2>(), b->n_terms);
        note_launch(ST_CONVERT);
        note_launch(ST_CONVERT);
        check_cuda(cudaGetLastError(), "k_to_f32");
        ac = fa.as<V>();
        bc = fb.as<V>();
    }
    // the same sum on both sides: only i <= j pairs are generated
    Src src{a->keys, b->keys, a->pbase, b->pbase, ac, bc, (uint32_t)a->n_terms, a == b ? 1u : 0u,
            recip64((uint32_t)a->n_terms)};
    return finish_canonical<Src, MODE>(src, R, (uint32_t)b->n_terms, a->n_qubits, st);
}

template <int WP, int MODE>
static paulib_sum* terms_mode(const paulib_sum* in, cudaStream_t st) {
    using Src = TermSrc<WP, MODE>;
    using V = typename Src::V;
    Scratch f;
    const V* c;
    if constexpr (MODE == M_FP64) {
        c = reinterpret_cast<const V*>(in->coef);
    } else {
        f = Scratch((size_t)in->n_terms * 8, st);
        StageScope ss(ST_CONVERT, st);
        k_to_f32<MODE><<<(unsigned)((in->n_terms + 255) / 256), 256, 0, st>>>(in->coef, f.as<float2>(), in->n_terms);
        note_launch(ST_CONVERT);
        check_cuda(cudaGetLastError(), "k_to_f32");
        c = f.as<V>();
    }
    Src src{in->keys, in->phase, c};
    return finish_canonical<Src, MODE>(src, (uint32_t)in->n_terms, 0, in->n_qubits, st);
}

}  // namespace paulib
