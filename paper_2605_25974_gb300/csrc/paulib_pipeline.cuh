// paulib_pipeline.cuh -- canonical form of a Pauli-sum product (PauLIB Sec. III-H
// sort_and_combine, applied to the outer product of Sec. IV-C / V-C).
//
// The paper sorts an index array by the lexicographic key of the packed words
// and then merges equal neighbours in one linear scan.  This file computes the
// same result with a sample sort laid out for the GPU:
//
//   records   A record is a 32-bit index: a product (i, j) is r = j*|A| + i
//             (Sec. IV-C's raw index); a term of a sum is its position.  Keys
//             are never stored per product; they are recomputed from (i, j).
//   level 1   Sample records, sort the sample (recursively, with this same
//             pipeline), pick splitters, then count and scatter every record
//             into its coarse key range.  For products the counting kernel
//             walks the product space in tiles: left terms in registers, right
//             terms in shared memory read as warp broadcasts.
//   level 2   One CTA per coarse range keeps a worklist: a range larger than
//             the shared-memory leaf capacity is split again by splitters taken
//             from a sample of its own records; a leaf is gathered into shared
//             memory, sorted by (key, record) with a bitonic network, and its
//             equal-key runs are summed (Sec. III-H's merge).  A range whose
//             keys are all equal (one heavily repeated string) is reduced
//             without sorting.  Each coarse range writes its merged terms
//             densely to a staging buffer.
//   compact   Exclusive scan of the per-range term counts, then a copy into
//             the output sum.
//
// Every device loop is bounded; failures raise a device error word that the
// host turns into a status.
#pragma once
#include <algorithm>
#include <mutex>
#include <type_traits>
#include <vector>
#include "paulib_device.cuh"
#include "paulib_internal.h"

namespace paulib {

enum : int { M_FP64 = 0, M_F32_D64 = 1, M_F32_TWOSUM = 2 };
enum : int32_t { ERR_NONE = 0, ERR_STACK = 1, ERR_PROGRESS = 2, ERR_ITER = 4, ERR_LIST = 16 };

template <int MODE> struct ValT { using T = float2; };
template <> struct ValT<M_FP64> { using T = double2; };

__device__ __forceinline__ double2 rot_v(double2 c, uint32_t k) { return rot_ik(c, k); }
__device__ __forceinline__ float2 rot_v(float2 c, uint32_t k) { return rot_ikf(c, k); }
__device__ __forceinline__ double2 mul_v(double2 a, double2 b) { return cmul(a, b); }
__device__ __forceinline__ float2 mul_v(float2 a, float2 b) { return cmulf(a, b); }
template <class V> __device__ __forceinline__ V one_v();
template <> __device__ __forceinline__ double2 one_v<double2>() { return make_double2(1.0, 0.0); }
template <> __device__ __forceinline__ float2 one_v<float2>() { return make_float2(1.f, 0.f); }

// ---------------------------------------------------------------- record sources

// Products of two sums: record r = j*na + i stands for a_i * b_j.
//
// When both operands are the same sum (sym != 0, e.g. H*H) only records with
// i <= j exist.  P_a P_b and P_b P_a are the same string, and their phases
// differ by 2*[a,b] (the symplectic inner product, Sec. III-F), so the pair
// contributes i^k c_a c_b (1 + (-1)^[a,b]): twice one product when the
// strings commute, exactly zero when they anti-commute.  The string is kept
// either way, as in the ordered-pair form.
template <int WP_, int MODE>
struct ProdSrc {
    static constexpr int WP = WP_;
    static constexpr int NW = 2 * WP;
    using V = typename ValT<MODE>::T;
    const uint64_t* ak;
    const uint64_t* bk;
    const uint8_t* ap;
    const uint8_t* bp;
    const V* ac;
    const V* bc;
    uint32_t na;
    uint32_t sym = 0;
    uint64_t na_inv = 0;  // ceil(2^64 / na), or 0 when na = 1 (see recip64)
    // j = r / na by one high multiply: exact for every 32-bit r, because the
    // reciprocal's error adds less than 2^-32 while r / na's fractional part
    // stays at least 1 / na > 2^-32 away from the next integer.
    __device__ __forceinline__ void split(uint32_t r, uint32_t& i, uint32_t& j) const {
        j = na_inv ? (uint32_t)__umul64hi((uint64_t)r, na_inv) : r;
        i = r - j * na;
    }
    __device__ __forceinline__ void key(uint32_t r, uint64_t (&k)[NW]) const {
        uint32_t i, j;
        split(r, i, j);
        uint64_t a[NW], b[NW];
        key_load_g<NW>(ak, i, a);
        key_load_g<NW>(bk, j, b);
#pragma unroll
        for (int q = 0; q < NW; ++q) k[q] = a[q] ^ b[q];
    }
    // Product key, and the coefficient i^k c_a c_b in the mode's precision.
    __device__ __forceinline__ V value(uint32_t r, uint64_t (&k)[NW]) const {
        uint32_t i, j;
        split(r, i, j);
        uint64_t a[NW], b[NW];
        key_load_g<NW>(ak, i, a);
        key_load_g<NW>(bk, j, b);
        const uint32_t ph = sym_flags(i, j, a, b) | string_product<WP>(a, b, __ldg(ap + i), __ldg(bp + j), k);
        return apply(mul_v(ac[i], bc[j]), ph);
    }
    // Bit 2: the unordered pair cancels; bit 3: it counts twice.
    __device__ __forceinline__ uint32_t sym_flags(uint32_t i, uint32_t j, const uint64_t (&a)[NW],
                                                  const uint64_t (&b)[NW]) const {
        if (!sym || i == j) return 0u;
        uint64_t s = 0;
#pragma unroll
        for (int q = 0; q < WP; ++q) s ^= (a[q] & b[WP + q]) ^ (a[WP + q] & b[q]);
        return (__popcll(s) & 1) ? 4u : 8u;
    }
    __device__ __forceinline__ V apply(V v, uint32_t ph) const {
        if (ph & 4u) {
            V z;
            z.x = 0;
            z.y = 0;
            return z;
        }
        v = rot_v(v, ph & 3u);
        if (ph & 8u) {
            v.x += v.x;  // exact doubling
            v.y += v.y;
        }
        return v;
    }
    // Product key and phase exponent (plus the symmetric-pair bits) only.
    __device__ __forceinline__ uint32_t keyphase(uint32_t r, uint64_t (&k)[NW]) const {
        uint32_t i, j;
        split(r, i, j);
        uint64_t a[NW], b[NW];
        key_load_g<NW>(ak, i, a);
        key_load_g<NW>(bk, j, b);
        return sym_flags(i, j, a, b) | string_product<WP>(a, b, __ldg(ap + i), __ldg(bp + j), k);
    }
    // Coefficient of record r from its keyphase() bits.
    __device__ __forceinline__ V coefv(uint32_t r, uint32_t ph) const {
        uint32_t i, j;
        split(r, i, j);
        return apply(mul_v(ac[i], bc[j]), ph);
    }
};

inline uint64_t recip64(uint32_t d) { return d <= 1 ? 0ull : ~0ull / d + 1ull; }

// Terms of one sum: record r is term r; value i^phase * c (or 1 when c is
// null, which counts occurrences).
template <int WP_, int MODE>
struct TermSrc {
    static constexpr int WP = WP_;
    static constexpr int NW = 2 * WP;
    using V = typename ValT<MODE>::T;
    const uint64_t* keys;
    const uint8_t* phase;
    const V* c;
    __device__ __forceinline__ void key(uint32_t r, uint64_t (&k)[NW]) const { key_load_g<NW>(keys, r, k); }
    __device__ __forceinline__ V value(uint32_t r, uint64_t (&k)[NW]) const {
        key_load_g<NW>(keys, r, k);
        const V v = c ? c[r] : one_v<V>();
        return rot_v(v, phase ? (uint32_t)(__ldg(phase + r) & 3u) : 0u);
    }
    __device__ __forceinline__ uint32_t keyphase(uint32_t r, uint64_t (&k)[NW]) const {
        key_load_g<NW>(keys, r, k);
        return phase ? (uint32_t)(__ldg(phase + r) & 3u) : 0u;
    }
    __device__ __forceinline__ V coefv(uint32_t r, uint32_t ph) const {
        return rot_v(c ? c[r] : one_v<V>(), ph);
    }
};

// Opaque NW-word keys with value 1 each: sorting them with the pipeline
// yields the distinct keys and their multiplicities (used for splitters).
template <int NW_>
struct SampleSrc {
    static constexpr int NW = NW_;
    static constexpr int WP = NW_ / 2;
    using V = double2;
    const uint64_t* keys;
    __device__ __forceinline__ void key(uint32_t r, uint64_t (&k)[NW]) const { key_load_g<NW>(keys, r, k); }
    __device__ __forceinline__ V value(uint32_t r, uint64_t (&k)[NW]) const {
        key_load_g<NW>(keys, r, k);
        return make_double2(1.0, 0.0);
    }
    __device__ __forceinline__ uint32_t keyphase(uint32_t r, uint64_t (&k)[NW]) const {
        key_load_g<NW>(keys, r, k);
        return 0u;
    }
    __device__ __forceinline__ V coefv(uint32_t, uint32_t) const { return make_double2(1.0, 0.0); }
};

// ---------------------------------------------------------------- small helpers

template <int NW>
__device__ __forceinline__ bool key_succ(const uint64_t (&k)[NW], uint64_t (&o)[NW]) {
    bool carry = true;
#pragma unroll
    for (int q = NW - 1; q >= 0; --q) {
        o[q] = k[q] + (carry ? 1ull : 0ull);
        carry = carry && (o[q] == 0ull);
    }
    return !carry;  // false on overflow (k was the largest key)
}

// Number of splitters <= k among n sorted splitters at `spl` (upper bound).
template <int NW>
__device__ __forceinline__ uint32_t upper_bound_keys(const uint64_t* spl, uint32_t n,
                                                     const uint64_t (&k)[NW]) {
    uint32_t lo = 0, len = n;
    while (len > 0) {
        const uint32_t half = len >> 1;
        if (key_cmp_m<NW>(k, spl + (uint64_t)(lo + half) * NW) >= 0) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo;
}

// Keys held in shared memory are stored word-major: word w of key t at
// s[w * stride + t].  Lanes that touch different keys then touch different
// banks; a key-major layout (32- or 64-byte records) puts every lane on the
// same few banks.
template <int NW>
__device__ __forceinline__ void skey_store(uint64_t* s, uint32_t stride, uint32_t t, const uint64_t (&k)[NW]) {
#pragma unroll
    for (int w = 0; w < NW; ++w) s[(size_t)w * stride + t] = k[w];
}
template <int NW>
__device__ __forceinline__ void skey_load(const uint64_t* s, uint32_t stride, uint32_t t, uint64_t (&k)[NW]) {
#pragma unroll
    for (int w = 0; w < NW; ++w) k[w] = s[(size_t)w * stride + t];
}
template <int NW>
__device__ __forceinline__ int skey_cmp(const uint64_t* s, uint32_t stride, uint32_t a, uint32_t b) {
#pragma unroll 4
    for (int w = 0; w < NW; ++w) {
        const uint64_t u = s[(size_t)w * stride + a], v = s[(size_t)w * stride + b];
        if (u != v) return u < v ? -1 : 1;
    }
    return 0;
}
// skey_cmp over words w0..NW-1 only (the keys agree on the words before).
template <int NW>
__device__ __forceinline__ int skey_cmp_from(const uint64_t* s, uint32_t stride, uint32_t a, uint32_t b, int w0) {
    for (int w = w0; w < NW; ++w) {
        const uint64_t u = s[(size_t)w * stride + a], v = s[(size_t)w * stride + b];
        if (u != v) return u < v ? -1 : 1;
    }
    return 0;
}
template <int NW>
__device__ __forceinline__ int skey_cmp_r(const uint64_t (&k)[NW], const uint64_t* s, uint32_t stride, uint32_t b) {
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const uint64_t v = s[(size_t)w * stride + b];
        if (k[w] != v) return k[w] < v ? -1 : 1;
    }
    return 0;
}
// Number of splitters <= k among n sorted word-major splitters.
template <int NW>
__device__ __forceinline__ uint32_t upper_bound_skeys(const uint64_t* s, uint32_t stride, uint32_t n,
                                                      const uint64_t (&k)[NW]) {
    uint32_t lo = 0, len = n;
    while (len > 0) {
        const uint32_t half = len >> 1;
        if (skey_cmp_r<NW>(k, s, stride, lo + half) >= 0) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo;
}

template <int THREADS>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_warp, uint32_t& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < THREADS / 32 ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < THREADS / 32) s_warp[lane] = w;
    }
    __syncthreads();
    total = s_warp[THREADS / 32 - 1];
    const uint32_t before = wid ? s_warp[wid - 1] : 0u;
    __syncthreads();
    return before + x - v;
}

// ---------------------------------------------------------------- accumulators

template <int MODE> struct Acc;
template <> struct Acc<M_FP64> {
    double re = 0.0, im = 0.0;
    __device__ __forceinline__ Acc up(int o) const {
        Acc t;
        t.re = __shfl_up_sync(0xffffffffu, re, o);
        t.im = __shfl_up_sync(0xffffffffu, im, o);
        return t;
    }
    __device__ __forceinline__ Acc bcast(int l) const {
        Acc t;
        t.re = __shfl_sync(0xffffffffu, re, l);
        t.im = __shfl_sync(0xffffffffu, im, l);
        return t;
    }
    __device__ __forceinline__ void add(double2 v) { re += v.x; im += v.y; }
    __device__ __forceinline__ void merge(const Acc& o) { re += o.re; im += o.im; }
    __device__ __forceinline__ double2 result() const { return make_double2(re, im); }
    __device__ __forceinline__ void shfl_merge(int o) {
        Acc t;
        t.re = __shfl_down_sync(0xffffffffu, re, o);
        t.im = __shfl_down_sync(0xffffffffu, im, o);
        merge(t);
    }
};
template <> struct Acc<M_F32_D64> {
    double re = 0.0, im = 0.0;
    __device__ __forceinline__ Acc up(int o) const {
        Acc t;
        t.re = __shfl_up_sync(0xffffffffu, re, o);
        t.im = __shfl_up_sync(0xffffffffu, im, o);
        return t;
    }
    __device__ __forceinline__ Acc bcast(int l) const {
        Acc t;
        t.re = __shfl_sync(0xffffffffu, re, l);
        t.im = __shfl_sync(0xffffffffu, im, l);
        return t;
    }
    __device__ __forceinline__ void add(float2 v) { re += (double)v.x; im += (double)v.y; }
    __device__ __forceinline__ void merge(const Acc& o) { re += o.re; im += o.im; }
    __device__ __forceinline__ double2 result() const { return make_double2(re, im); }
    __device__ __forceinline__ void shfl_merge(int o) {
        Acc t;
        t.re = __shfl_down_sync(0xffffffffu, re, o);
        t.im = __shfl_down_sync(0xffffffffu, im, o);
        merge(t);
    }
};
// FP32 sum with TwoSum error terms (Ogita, Rump, Oishi 2005, Sum2): the
// rounding error of every addition is collected exactly and added back once.
template <> struct Acc<M_F32_TWOSUM> {
    float sr = 0.f, er = 0.f, si = 0.f, ei = 0.f;
    __device__ __forceinline__ Acc up(int o) const {
        Acc t;
        t.sr = __shfl_up_sync(0xffffffffu, sr, o);
        t.er = __shfl_up_sync(0xffffffffu, er, o);
        t.si = __shfl_up_sync(0xffffffffu, si, o);
        t.ei = __shfl_up_sync(0xffffffffu, ei, o);
        return t;
    }
    __device__ __forceinline__ Acc bcast(int l) const {
        Acc t;
        t.sr = __shfl_sync(0xffffffffu, sr, l);
        t.er = __shfl_sync(0xffffffffu, er, l);
        t.si = __shfl_sync(0xffffffffu, si, l);
        t.ei = __shfl_sync(0xffffffffu, ei, l);
        return t;
    }
    __device__ __forceinline__ void add(float2 v) {
        float s, e;
        two_sum(sr, v.x, s, e);
        sr = s;
        er = __fadd_rn(er, e);
        two_sum(si, v.y, s, e);
        si = s;
        ei = __fadd_rn(ei, e);
    }
    __device__ __forceinline__ void merge(const Acc& o) {
        float s, e;
        two_sum(sr, o.sr, s, e);
        sr = s;
        er = __fadd_rn(__fadd_rn(er, o.er), e);
        two_sum(si, o.si, s, e);
        si = s;
        ei = __fadd_rn(__fadd_rn(ei, o.ei), e);
    }
    __device__ __forceinline__ double2 result() const {
        return make_double2((double)sr + (double)er, (double)si + (double)ei);
    }
    __device__ __forceinline__ void shfl_merge(int o) {
        Acc t;
        t.sr = __shfl_down_sync(0xffffffffu, sr, o);
        t.er = __shfl_down_sync(0xffffffffu, er, o);
        t.si = __shfl_down_sync(0xffffffffu, si, o);
        t.ei = __shfl_down_sync(0xffffffffu, ei, o);
        merge(t);
    }
};

// ---------------------------------------------------------------- capacities

constexpr int kL2Threads = 512;
constexpr int kStackCap = 4096;
constexpr int kSmemBudget = 110 * 1024;

// Shared memory per sample slot of the range kernel: the key (8*NW bytes),
// two sort codes (16 bytes), two 16-bit slot arrays for the merge sort and a
// range flag (1 byte).  A block leaf slot adds the record number (4 bytes,
// the tie-break that makes the order of equal keys and so the summation
// order deterministic).  CAP is the sample capacity of the range kernel.
constexpr int kSplitRecBytes = 16 + 2 + 2 + 1;
constexpr int kBlockLeafRecBytes = kSplitRecBytes + 4;
template <int NW>
constexpr int leaf_cap() {
    int cap = 4096;
    while (cap > 64 && cap * (8 * NW + kSplitRecBytes) > kSmemBudget) cap >>= 1;
    return cap;
}
template <int NW>
constexpr size_t leaf_smem() {
    return (size_t)leaf_cap<NW>() * (8 * NW + kSplitRecBytes);
}

// Coarse (level 1) splitters live in shared memory of the counting kernel.
template <int NW>
constexpr int max_coarse_splitters() {
    return (128 * 1024) / (8 * NW) < 4094 ? (128 * 1024) / (8 * NW) : 4094;
}

// ---------------------------------------------------------------- sampling

template <class Src>
struct IsProdT : std::false_type {};
template <int WP, int MODE>
struct IsProdT<ProdSrc<WP, MODE>> : std::true_type {};

template <class Src>
__global__ void k_sample(Src src, uint32_t R, uint32_t S, uint64_t seed, uint64_t* out) {
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    uint32_t r;
    if (S >= R) r = s;
    else r = (uint32_t)(mix64(seed + s) % R);
    if constexpr (IsProdT<Src>::value) {
        if (src.sym) {  // fold onto the i <= j triangle
            const uint32_t j = r / src.na, i = r - j * src.na;
            if (i > j) r = i * src.na + j;
        }
    }
    uint64_t k[Src::NW];
    src.key(r, k);
    key_store<Src::NW>(out, s, k);
}

// One coarse range holding every record in order.
static __global__ void k_iota(uint32_t* rec, uint32_t n, uint64_t* boff, uint8_t* bflags) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) rec[t] = t;
    if (t == 0) {
        boff[0] = 0;
        boff[1] = n;
        bflags[0] = 0;
    }
}

// One coarse range holding the i <= j records of a symmetric product, in
// order: t -> (i, j) with j(j+1)/2 <= t < (j+1)(j+2)/2.
static __global__ void k_iota_tri(uint32_t* rec, uint32_t n, uint32_t na, uint64_t* boff, uint8_t* bflags) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        uint64_t j = (uint64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
        while (j * (j + 1) / 2 > t) --j;
        while ((j + 1) * (j + 2) / 2 <= t) ++j;
        const uint64_t i = t - j * (j + 1) / 2;
        rec[t] = (uint32_t)(j * na + i);
    }
    if (t == 0) {
        boff[0] = 0;
        boff[1] = n;
        bflags[0] = 0;
    }
}

// Splitter choice from the sorted, merged sample: keys dk[u] with occurrence
// counts dc[u].x.  For t = 1..B1-1 the key holding sample rank t*S/B1 gives
// a pair (key, succ(key)) when that key fills at least one whole coarse
// range (a uniform range), else (key, key) (an empty range).
template <int NW>
__global__ void __launch_bounds__(1024) k_select(const uint64_t* __restrict__ dk,
                                                 const double2* __restrict__ dc,
                                                 const uint64_t* __restrict__ u_dev, uint32_t S,
                                                 uint32_t B1, uint32_t* pref, uint64_t* spl,
                                                 uint8_t* bflags) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    const uint32_t U = (uint32_t)*u_dev;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < U; base += 1024) {
        const uint32_t u = base + threadIdx.x;
        const uint32_t c = u < U ? (uint32_t)dc[u].x : 0u;
        uint32_t total;
        const uint32_t ex = block_excl_scan<1024>(c, s_warp, total);
        if (u < U) pref[u] = s_carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += total;
        __syncthreads();
    }
    const uint32_t nb = 2 * B1 - 1;
    for (uint32_t b = threadIdx.x; b < nb; b += 1024) bflags[b] = 0;
    __syncthreads();
    const double full = (double)S / (double)B1;
    for (uint32_t t = 1 + threadIdx.x; t < B1; t += 1024) {
        const uint32_t tau = (uint32_t)(((uint64_t)t * S) / B1);
        // largest u with pref[u] <= tau
        uint32_t lo = 0, hi = U;  // pref[lo] <= tau invariant (pref[0] = 0)
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (pref[mid] <= tau) lo = mid; else hi = mid;
        }
        uint64_t k[NW], s2[NW];
        key_load_g<NW>(dk, lo, k);
        const bool heavy = dc[lo].x >= full;
        bool ok = true;
        if (heavy) ok = key_succ<NW>(k, s2);
        key_store<NW>(spl, 2 * (t - 1), k);
        if (heavy && ok) {
            key_store<NW>(spl, 2 * (t - 1) + 1, s2);
            bflags[2 * t - 1] = 1;
        } else {
            key_store<NW>(spl, 2 * (t - 1) + 1, k);
            if (heavy) bflags[nb - 1] = 1;  // the largest possible key: its range is the last one
        }
    }
}

// ---------------------------------------------------------------- level 1: count

// 64 bits of a register key starting at bit position P (word 0's top bit is
// position 0); zero beyond the key.
template <int NW>
__device__ __forceinline__ uint64_t reg_bits64(const uint64_t (&k)[NW], uint32_t P) {
    const uint32_t w = P >> 6, sh = P & 63u;
    uint64_t v = 0, nx = 0;
#pragma unroll
    for (int q = 0; q < NW; ++q) {  // masks rather than an index, so k stays in registers
        v |= k[q] & (0ull - (uint64_t)((uint32_t)q == w));
        nx |= k[q] & (0ull - (uint64_t)((uint32_t)q == w + 1u));
    }
    return sh ? (v << sh) | (nx >> (64u - sh)) : v;
}

// Compares bits [0, P) of a register key with those of word-major key 0.
template <int NW>
__device__ __forceinline__ int prefix_cmp(const uint64_t (&k)[NW], const uint64_t* s, uint32_t stride, uint32_t P) {
    int pc = 0;
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        if (pc == 0 && 64u * q < P) {
            uint64_t a = k[q], b = s[(size_t)q * stride];
            const uint32_t nb = P - 64u * q;
            if (nb < 64u) {
                const uint64_t m = ~0ull << (64u - nb);
                a &= m;
                b &= m;
            }
            if (a != b) pc = a < b ? -1 : 1;
        }
    }
    return pc;
}

constexpr int kCountThreads = 256;
constexpr int kCountCols = 64;
constexpr int kTopBits = 11;  // top-level table of the coarse splitter search: 2^11 + 1 entries

// Coarse splitters are located through a 128-bit window of their keys: all
// splitters share their first L bits (L is the first position where one of
// them differs from splitter 0), and code1/code2 are key bits [L, L+64) and
// [L+64, L+128).  A key whose first L bits differ from the shared prefix lies
// below or above every splitter; other keys compare by the window, and by the
// whole key (from the splitter table in global memory) only when the windows
// are equal.  The search then reads 16 bytes of shared memory per step
// instead of whole keys.
template <int NW>
__global__ void __launch_bounds__(1024) k_spl_codes(const uint64_t* __restrict__ spl, uint32_t nsp,
                                                    uint64_t* codes, uint32_t* meta) {
    __shared__ unsigned long long s_or[NW];
    __shared__ uint32_t s_L;
    for (int w = threadIdx.x; w < NW; w += blockDim.x) s_or[w] = 0ull;
    __syncthreads();
    uint64_t acc[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) acc[w] = 0;
    for (uint32_t t = threadIdx.x; t < nsp; t += blockDim.x) {
#pragma unroll
        for (int w = 0; w < NW; ++w) acc[w] |= spl[(size_t)t * NW + w] ^ spl[w];
    }
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        uint64_t v = acc[w];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicOr(&s_or[w], (unsigned long long)v);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t L = 64u * NW;
        for (int w = 0; w < NW; ++w)
            if (s_or[w]) { L = 64u * w + (uint32_t)__clzll((long long)s_or[w]); break; }
        s_L = L;
        meta[0] = L;
    }
    __syncthreads();
    const uint32_t L = s_L;
    for (uint32_t t = threadIdx.x; t < nsp; t += blockDim.x) {
        uint64_t k[NW];
        key_load_g<NW>(spl, t, k);
        codes[t] = reg_bits64<NW>(k, L);
        codes[nsp + t] = reg_bits64<NW>(k, L + 64u);
    }
}

// Number of splitters <= k (see k_spl_codes); p0 is splitter 0 (shared).
template <int NW>
__device__ __forceinline__ uint32_t locate_coarse(const uint64_t (&k)[NW], const uint64_t* s_c1,
                                                  const uint64_t* s_c2, const uint64_t* p0, uint32_t nsp,
                                                  uint32_t L, const uint64_t* __restrict__ spl,
                                                  const uint16_t* s_top) {
    // first L bits against the splitters' shared prefix
    int pc = 0;
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        if (pc == 0 && 64u * q < L) {
            uint64_t a = k[q], b = p0[q];
            const uint32_t nb = L - 64u * q;
            if (nb < 64u) {
                const uint64_t m = ~0ull << (64u - nb);
                a &= m;
                b &= m;
            }
            if (a != b) pc = a < b ? -1 : 1;
        }
    }
    if (pc) return pc < 0 ? 0u : nsp;
    const uint64_t c1 = reg_bits64<NW>(k, L), c2 = reg_bits64<NW>(k, L + 64u);
    // splitters are ordered by c1 first: those whose top bits of c1 are below
    // the key's are below it, those above are above it
    const uint32_t v = (uint32_t)(c1 >> (64 - kTopBits));
    uint32_t lo = s_top[v], len = (uint32_t)s_top[v + 1] - lo;
    while (len > 0) {
        const uint32_t half = len >> 1, mid = lo + half;
        const uint64_t s1 = s_c1[mid];
        bool ge;
        if (c1 != s1) {
            ge = c1 > s1;
        } else {
            const uint64_t s2 = s_c2[mid];
            ge = c2 != s2 ? c2 > s2 : key_cmp_m<NW>(k, spl + (size_t)mid * NW) >= 0;
        }
        if (ge) {
            lo = mid + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo;
}

// Shared-memory layout of the counting kernels: codes [2][nsp], splitter 0,
// then (products) one tile of right-hand keys, then the bucket histogram.
template <int NW>
__host__ __device__ constexpr size_t count_smem(uint32_t nsp, bool tile) {
    return (size_t)nsp * 16 + (size_t)NW * 8 + (tile ? (size_t)kCountCols * NW * 8 : 0) + (size_t)(nsp + 1) * 4 +
           (size_t)((1u << kTopBits) + 1) * 2;
}

// s_top[v] = number of splitters whose code c1 has its top kTopBits bits
// below v (v = 0 .. 2^kTopBits); c1 is sorted.  Narrows every search to the
// splitters sharing the key's top bits.
__device__ __forceinline__ void build_top(const uint64_t* s_c1, uint32_t nsp, uint16_t* s_top) {
    for (uint32_t v = threadIdx.x; v <= (1u << kTopBits); v += blockDim.x) {
        uint32_t lo = 0, len = nsp;
        while (len > 0) {
            const uint32_t half = len >> 1, mid = lo + half;
            if ((s_c1[mid] >> (64 - kTopBits)) < v) {
                lo = mid + 1;
                len -= half + 1;
            } else {
                len = half;
            }
        }
        s_top[v] = (uint16_t)lo;
    }
}

// Products: a tile is kCountThreads left terms x kCountCols right terms.
template <int WP, int MODE>
__global__ void __launch_bounds__(kCountThreads) k_count_prod(ProdSrc<WP, MODE> src, uint32_t nb_terms,
                                                               const uint64_t* __restrict__ spl,
                                                               const uint64_t* __restrict__ codes,
                                                               const uint32_t* __restrict__ meta,
                                                               uint32_t nsp, uint16_t* ids,
                                                               uint32_t* counts) {
    constexpr int NW = 2 * WP;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_c1 = reinterpret_cast<uint64_t*>(smem);
    uint64_t* s_c2 = s_c1 + nsp;
    uint64_t* s_p0 = s_c2 + nsp;
    uint64_t* s_b = s_p0 + NW;
    uint32_t* s_hist = reinterpret_cast<uint32_t*>(s_b + kCountCols * NW);
    const uint32_t nbk = nsp + 1;
    uint16_t* s_top = reinterpret_cast<uint16_t*>(s_hist + nbk);
    const uint32_t L = meta[0];
    for (uint32_t q = threadIdx.x; q < 2 * nsp; q += blockDim.x) s_c1[q] = codes[q];
    for (uint32_t q = threadIdx.x; q < (uint32_t)NW; q += blockDim.x) s_p0[q] = spl[q];
    for (uint32_t q = threadIdx.x; q < nbk; q += blockDim.x) s_hist[q] = 0;
    __syncthreads();
    build_top(s_c1, nsp, s_top);  // visible after the tile loop's first barrier
    const uint32_t na = src.na;
    const uint32_t ti_n = (na + kCountThreads - 1) / kCountThreads;
    const uint32_t tj_n = (nb_terms + kCountCols - 1) / kCountCols;
    const uint64_t ntiles = (uint64_t)ti_n * tj_n;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t ti = (uint32_t)(tile % ti_n), tj = (uint32_t)(tile / ti_n);
        const uint32_t j0 = tj * kCountCols;
        const uint32_t ncols = min((uint32_t)kCountCols, nb_terms - j0);
        __syncthreads();
        for (uint32_t q = threadIdx.x; q < ncols * NW; q += blockDim.x) s_b[q] = src.bk[(uint64_t)j0 * NW + q];
        __syncthreads();
        const uint32_t i = ti * kCountThreads + threadIdx.x;
        if (i < na) {
            uint64_t a[NW];
            key_load_g<NW>(src.ak, i, a);
            for (uint32_t c = 0; c < ncols; ++c) {
                if (src.sym && i > j0 + c) continue;  // the (j, i) record stands for both orders
                uint64_t k[NW];
                const uint64_t* bb = s_b + c * NW;
#pragma unroll
                for (int q = 0; q < NW; ++q) k[q] = a[q] ^ bb[q];
                const uint32_t bkt = locate_coarse<NW>(k, s_c1, s_c2, s_p0, nsp, L, spl, s_top);
                ids[(uint64_t)(j0 + c) * na + i] = (uint16_t)bkt;
                atomicAdd(&s_hist[bkt], 1u);
            }
        }
    }
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < nbk; q += blockDim.x)
        if (s_hist[q]) atomicAdd(&counts[q], s_hist[q]);
}

template <class Src>
__global__ void __launch_bounds__(kCountThreads) k_count_lin(Src src, uint32_t R,
                                                              const uint64_t* __restrict__ spl,
                                                              const uint64_t* __restrict__ codes,
                                                              const uint32_t* __restrict__ meta,
                                                              uint32_t nsp, uint16_t* ids,
                                                              uint32_t* counts) {
    constexpr int NW = Src::NW;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_c1 = reinterpret_cast<uint64_t*>(smem);
    uint64_t* s_c2 = s_c1 + nsp;
    uint64_t* s_p0 = s_c2 + nsp;
    uint32_t* s_hist = reinterpret_cast<uint32_t*>(s_p0 + NW);
    const uint32_t nbk = nsp + 1;
    uint16_t* s_top = reinterpret_cast<uint16_t*>(s_hist + nbk);
    const uint32_t L = meta[0];
    for (uint32_t q = threadIdx.x; q < 2 * nsp; q += blockDim.x) s_c1[q] = codes[q];
    for (uint32_t q = threadIdx.x; q < (uint32_t)NW; q += blockDim.x) s_p0[q] = spl[q];
    for (uint32_t q = threadIdx.x; q < nbk; q += blockDim.x) s_hist[q] = 0;
    __syncthreads();
    build_top(s_c1, nsp, s_top);
    __syncthreads();
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        uint64_t k[NW];
        src.key(r, k);
        const uint32_t bkt = locate_coarse<NW>(k, s_c1, s_c2, s_p0, nsp, L, spl, s_top);
        ids[r] = (uint16_t)bkt;
        atomicAdd(&s_hist[bkt], 1u);
    }
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < nbk; q += blockDim.x)
        if (s_hist[q]) atomicAdd(&counts[q], s_hist[q]);
}

// Exclusive scan of n 32-bit counts into 64-bit offsets (single CTA).
static __global__ void __launch_bounds__(1024) k_scan_counts(const uint32_t* __restrict__ cnt, uint32_t n,
                                                      uint64_t* off) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint64_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < n; base += 1024) {
        const uint32_t u = base + threadIdx.x;
        const uint32_t c = u < n ? cnt[u] : 0u;
        uint32_t total;
        const uint32_t ex = block_excl_scan<1024>(c, s_warp, total);
        if (u < n) off[u] = s_carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) off[n] = s_carry;
}

static __global__ void __launch_bounds__(1024) k_scan_u64(const uint64_t* __restrict__ cnt, uint32_t n,
                                                   uint64_t* off) {
    __shared__ uint64_t s_v[1024];
    __shared__ uint64_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < n; base += 1024) {
        const uint32_t u = base + threadIdx.x;
        uint64_t v = u < n ? cnt[u] : 0ull;
        s_v[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const uint64_t y = threadIdx.x >= (uint32_t)o ? s_v[threadIdx.x - o] : 0ull;
            __syncthreads();
            s_v[threadIdx.x] += y;
            __syncthreads();
        }
        if (u < n) off[u] = s_carry + s_v[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += s_v[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) off[n] = s_carry;
}

// ---------------------------------------------------------------- level 1: scatter

constexpr int kScatterThreads = 512;
constexpr uint32_t kScatterChunk = 16384;

// Reads the bucket ids of records r0 .. r0+7 (one 16-byte load when all
// eight are in range; r0 is a multiple of 8, so the load is aligned).
__device__ __forceinline__ void load_ids8(const uint16_t* __restrict__ ids, uint32_t r0, uint32_t end,
                                          uint32_t (&b)[8]) {
    if (r0 + 8u <= end) {
        const uint4 v = *reinterpret_cast<const uint4*>(ids + r0);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            b[2 * q] = w[q] & 0xffffu;
            b[2 * q + 1] = w[q] >> 16;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) b[q] = r0 + q < end ? ids[r0 + q] : 0u;
    }
}

// Scatter of records into their coarse ranges, one chunk of kScatterChunk
// records at a time: count per range, take each range's global slots with one
// atomic per (chunk, range), order the chunk's records by range in shared
// memory (a counting sort), then write each range's run contiguously so that
// the stores coalesce instead of landing 4 bytes at a time.
static __global__ void __launch_bounds__(kScatterThreads) k_scatter(const uint16_t* __restrict__ ids, uint32_t R,
                                                             uint32_t nbk, uint64_t* cursor,
                                                             uint32_t* rec, uint32_t sym_na) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem);                       // [nbk] counts, then cursors
    uint32_t* s_off = s_cnt + ((nbk + 1) & ~1u);                               // [nbk + 1] chunk-local offsets
    uint64_t* s_base = reinterpret_cast<uint64_t*>(s_off + ((nbk + 2) & ~1u)); // [nbk] global first slot
    uint32_t* s_rec = reinterpret_cast<uint32_t*>(s_base + nbk);               // [kScatterChunk] records by range
    uint16_t* s_bid = reinterpret_cast<uint16_t*>(s_rec + kScatterChunk);      // [kScatterChunk] their ranges
    __shared__ uint32_t s_warp[32];
    // a symmetric product has no record for i > j (r = j*na + i)
    auto live = [&](uint32_t r) { return !sym_na || r % sym_na <= r / sym_na; };
    for (uint64_t c0 = (uint64_t)blockIdx.x * kScatterChunk; c0 < R; c0 += (uint64_t)gridDim.x * kScatterChunk) {
        const uint32_t c1 = (uint32_t)mn<uint64_t>(R, c0 + kScatterChunk);
        __syncthreads();
        for (uint32_t q = threadIdx.x; q < nbk; q += blockDim.x) s_cnt[q] = 0;
        __syncthreads();
        for (uint32_t r0 = (uint32_t)c0 + 8u * threadIdx.x; r0 < c1; r0 += 8u * blockDim.x) {
            uint32_t b[8];
            load_ids8(ids, r0, c1, b);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (r0 + q < c1 && live(r0 + q)) atomicAdd(&s_cnt[b[q]], 1u);
        }
        __syncthreads();
        // chunk-local exclusive offsets of the ranges (block scan in slices)
        {
            const uint32_t per = (nbk + kScatterThreads - 1) / kScatterThreads;
            const uint32_t q0 = threadIdx.x * per;
            uint32_t loc = 0;
            for (uint32_t q = q0; q < q0 + per && q < nbk; ++q) loc += s_cnt[q];
            uint32_t tot;
            uint32_t ex = block_excl_scan<kScatterThreads>(loc, s_warp, tot);
            for (uint32_t q = q0; q < q0 + per && q < nbk; ++q) {
                const uint32_t c = s_cnt[q];
                s_off[q] = ex;
                s_base[q] = c ? atomicAdd(reinterpret_cast<unsigned long long*>(cursor + q), (unsigned long long)c)
                              : 0ull;
                s_cnt[q] = ex;  // becomes the placement cursor
                ex += c;
            }
            if (threadIdx.x == 0) s_off[nbk] = tot;
        }
        __syncthreads();
        for (uint32_t r0 = (uint32_t)c0 + 8u * threadIdx.x; r0 < c1; r0 += 8u * blockDim.x) {
            uint32_t b[8];
            load_ids8(ids, r0, c1, b);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const uint32_t r = r0 + q;
                if (r < c1 && live(r)) {
                    const uint32_t p = atomicAdd(&s_cnt[b[q]], 1u);
                    s_rec[p] = r;
                    s_bid[p] = (uint16_t)b[q];
                }
            }
        }
        __syncthreads();
        const uint32_t nloc = s_off[nbk];
        for (uint32_t p = threadIdx.x; p < nloc; p += blockDim.x) {
            const uint32_t b = s_bid[p];
            rec[s_base[b] + (p - s_off[b])] = s_rec[p];
        }
    }
}

// ---------------------------------------------------------------- level 2

struct StackEnt {
    uint32_t lo, hi, flags, pad;
};
enum : uint32_t { SF_UNIFORM = 1u, SF_INB = 2u };

template <class Src, int MODE>
struct L2Cfg {
    using V = typename Src::V;
    static constexpr int NW = Src::NW;
    static constexpr int CAP = leaf_cap<NW>();
    static constexpr size_t SMEM = leaf_smem<NW>();
    // block leaves: at most MCAP records, sorted by one small CTA
    static constexpr uint32_t MCAP = CAP < 512 ? (uint32_t)CAP : 512u;
    static constexpr size_t MSMEM = (size_t)MCAP * (8 * NW + kBlockLeafRecBytes);
};

// ---- leaf ordering
//
// A block leaf (or a split sample) is ordered through two 64-bit codes per
// slot, held as c1s[t] and c1s[CAP + t]: the 64 key bits from the first
// position L where keys of the range differ, and the 64 from the first
// position L2 >= L + 64 where they differ.  Keys agree on every position
// outside those windows up to L2 + 64, so equal code pairs rarely hide
// different keys; they fall back to the full keys and then to the record
// number, so the order is total and deterministic.  Slots >= n are padding
// that sorts last.

// w0: keys with equal codes agree on every word before w0 (the word holding
// position L2 + 64), so whole-key comparisons start there.
template <int NW, uint32_t CAP>
__device__ __forceinline__ bool slot_gt(uint32_t a, uint32_t b, const uint64_t* c1s, const uint64_t* keys_s,
                                        uint32_t n, const uint32_t* recs, int w0) {
    if (a >= n || b >= n) return a >= n && (b < n || a > b);
    const uint64_t ca = c1s[a], cb = c1s[b];
    if (ca != cb) return ca > cb;
    const uint64_t da = c1s[CAP + a], db = c1s[CAP + b];
    if (da != db) return da > db;
    const int c = skey_cmp_from<NW>(keys_s, CAP, a, b, w0);
    if (c) return c > 0;
    if (recs) return recs[a] > recs[b];
    return a > b;
}

template <int NW, uint32_t CAP>
__device__ __forceinline__ bool slot_key_neq(uint32_t a, uint32_t b, const uint64_t* c1s, const uint64_t* keys_s,
                                             int w0) {
    if (c1s[a] != c1s[b] || c1s[CAP + a] != c1s[CAP + b]) return true;
    return skey_cmp_from<NW>(keys_s, CAP, a, b, w0) != 0;
}

// 64 bits of key t starting at bit position P (word 0's top bit is position 0).
template <int NW, uint32_t CAP>
__device__ __forceinline__ uint64_t key_bits64(const uint64_t* keys_s, uint32_t t, uint32_t P) {
    const uint32_t w = P >> 6, sh = P & 63u;
    if (w >= (uint32_t)NW) return 0ull;
    uint64_t v = keys_s[(size_t)w * CAP + t] << sh;
    if (sh && w + 1 < (uint32_t)NW) v |= keys_s[(size_t)(w + 1) * CAP + t] >> (64u - sh);
    return v;
}

// Codes c1s[0..n) and c1s[CAP..CAP + n): the positions where keys differ
// come from an OR reduction of (key ^ key 0) over the range.
template <int NW, int T, uint32_t CAP>
__device__ void build_codes(uint64_t* c1s, const uint64_t* keys_s, uint32_t n, unsigned long long* s_or,
                            uint32_t* s_L) {
    for (int w = threadIdx.x; w < NW; w += T) s_or[w] = 0ull;
    __syncthreads();
    uint64_t acc[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) acc[w] = 0;
    for (uint32_t t = threadIdx.x; t < n; t += T) {
#pragma unroll
        for (int w = 0; w < NW; ++w) acc[w] |= keys_s[(size_t)w * CAP + t] ^ keys_s[(size_t)w * CAP];
    }
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        uint64_t v = acc[w];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicOr(&s_or[w], (unsigned long long)v);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t L = 64u * NW, L2 = 64u * NW;
        for (int w = 0; w < NW; ++w)
            if (s_or[w]) { L = 64u * w + (uint32_t)__clzll((long long)s_or[w]); break; }
        for (int w = 0; w < NW; ++w) {
            if (64u * w + 63u < L + 64u) continue;
            uint64_t mm = s_or[w];
            if (L + 64u > 64u * w) mm &= ~0ull >> (L + 64u - 64u * w);
            if (mm) { L2 = 64u * w + (uint32_t)__clzll((long long)mm); break; }
        }
        s_L[0] = L;
        s_L[1] = L2;
    }
    __syncthreads();
    const uint32_t L = s_L[0], L2 = s_L[1];
    for (uint32_t t = threadIdx.x; t < n; t += T) {
        c1s[t] = key_bits64<NW, CAP>(keys_s, t, L);
        c1s[CAP + t] = key_bits64<NW, CAP>(keys_s, t, L2);
    }
    __syncthreads();
}

// Stable merge sort of slots 0..n-1 (padded to size, a power of two <= CAP).
// Each thread first sorts a run of `em` slots by insertion; every following
// level merges pairs of runs with merge-path partitioning: a thread finds
// where its `em` outputs start by a binary search along the diagonal, then
// merges sequentially.  One barrier per level.  Returns the array holding
// the sorted slots (ord or tmp).
template <int NW, int T, uint32_t CAP>
__device__ uint16_t* merge_sort_slots(uint16_t* ord, uint16_t* tmp, const uint64_t* c1s, const uint64_t* keys_s,
                                      uint32_t n, uint32_t size, const uint32_t* recs, int w0) {
    constexpr uint32_t EMAX = CAP / (uint32_t)T >= 2u ? CAP / (uint32_t)T : 2u;
    const uint32_t em = size / (uint32_t)T >= 2u ? size / (uint32_t)T : 2u;
    const uint32_t nthr = size / em;
    for (uint32_t t = threadIdx.x; t < nthr; t += T) {
        uint32_t v[EMAX];
#pragma unroll
        for (uint32_t k = 0; k < EMAX; ++k) {
            if (k < em) {
                uint32_t x = t * em + k;
                uint32_t q = k;
                while (q > 0 && slot_gt<NW, CAP>(v[q - 1], x, c1s, keys_s, n, recs, w0)) {
                    v[q] = v[q - 1];
                    --q;
                }
                v[q] = x;
            }
        }
#pragma unroll
        for (uint32_t k = 0; k < EMAX; ++k)
            if (k < em) ord[t * em + k] = (uint16_t)v[k];
    }
    __syncthreads();
    uint16_t* src = ord;
    uint16_t* dst = tmp;
    for (uint32_t s = em; s < size; s <<= 1) {
        for (uint32_t t = threadIdx.x; t < nthr; t += T) {
            const uint32_t o = t * em;
            const uint32_t seg = o & ~(2 * s - 1);
            const uint32_t d = o - seg;  // output offset within the merged segment
            const uint16_t* A = src + seg;
            const uint16_t* B = src + seg + s;
            uint32_t lo = d > s ? d - s : 0u, hi = d < s ? d : s;
            while (lo < hi) {  // number of A elements among the first d outputs
                const uint32_t mid = (lo + hi) >> 1;
                if (slot_gt<NW, CAP>(A[mid], B[d - mid - 1], c1s, keys_s, n, recs, w0)) hi = mid;
                else lo = mid + 1;
            }
            uint32_t i = lo, j = d - lo;
            for (uint32_t k = 0; k < em; ++k) {
                bool takeA;
                if (i >= s) takeA = false;
                else if (j >= s) takeA = true;
                else takeA = !slot_gt<NW, CAP>(A[i], B[j], c1s, keys_s, n, recs, w0);
                dst[o + k] = takeA ? A[i++] : B[j++];
            }
        }
        __syncthreads();
        uint16_t* t2 = src;
        src = dst;
        dst = t2;
    }
    return src;
}

// Exclusive block scan of (run started here?, partial sum) pairs under
// (f1, a1) . (f2, a2) = (f1 | f2, f2 ? a2 : a1 + a2): the sum carried into a
// thread from the run that began before it.
template <int T, int MODE>
__device__ __forceinline__ Acc<MODE> block_seg_carry(bool flag, const Acc<MODE>& a, Acc<MODE>* s_acc,
                                                     uint32_t* s_flag) {
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    Acc<MODE> x = a;
    bool f = flag;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Acc<MODE> y = x.up(o);
        const bool fy = __shfl_up_sync(0xffffffffu, f, o);
        if (lane >= (uint32_t)o) {
            if (!f) {
                Acc<MODE> t = y;
                t.merge(x);
                x = t;
            }
            f = f || fy;
        }
    }
    // exclusive within the warp
    Acc<MODE> ex = x.up(1);
    bool fex = __shfl_up_sync(0xffffffffu, f, 1);
    if (lane == 0) {
        ex = Acc<MODE>();
        fex = false;
    }
    if (lane == 31) {
        s_acc[wid] = x;
        s_flag[wid] = f;
    }
    __syncthreads();
    if (wid == 0) {
        Acc<MODE> wx = lane < (uint32_t)(T / 32) ? s_acc[lane] : Acc<MODE>();
        bool wf = lane < (uint32_t)(T / 32) ? s_flag[lane] != 0 : false;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const Acc<MODE> y = wx.up(o);
            const bool fy = __shfl_up_sync(0xffffffffu, wf, o);
            if (lane >= (uint32_t)o) {
                if (!wf) {
                    Acc<MODE> t = y;
                    t.merge(wx);
                    wx = t;
                }
                wf = wf || fy;
            }
        }
        Acc<MODE> wex = wx.up(1);
        bool wfex = __shfl_up_sync(0xffffffffu, wf, 1);
        if (lane == 0) {
            wex = Acc<MODE>();
            wfex = false;
        }
        if (lane < (uint32_t)(T / 32)) {
            s_acc[lane] = wex;
            s_flag[lane] = wfex;
        }
    }
    __syncthreads();
    Acc<MODE> res = ex;
    if (!fex) {  // the warp prefix flows in unless a run started earlier in this warp
        Acc<MODE> t = s_acc[wid];
        t.merge(ex);
        res = t;
    }
    __syncthreads();
    return res;
}

// Key order of two slots (codes, then full keys); records are ignored.
template <int NW, uint32_t CAP>
__device__ __forceinline__ int slot_key_cmp(uint32_t a, uint32_t b, const uint64_t* c1s, const uint64_t* keys_s,
                                            int w0) {
    const uint64_t ca = c1s[a], cb = c1s[b];
    if (ca != cb) return ca < cb ? -1 : 1;
    const uint64_t da = c1s[CAP + a], db = c1s[CAP + b];
    if (da != db) return da < db ? -1 : 1;
    return skey_cmp_from<NW>(keys_s, CAP, a, b, w0);
}

// Block-wide scratch of the range and leaf kernels.
template <int MODE, int NW>
struct BlockShared {
    uint32_t warp[32];
    Acc<MODE> acc[32];
    uint32_t flag[32];
    unsigned long long orr[NW];
    uint32_t L[2];
};

// Device buffers of level 2.  Merged terms are written at the record
// position of the range they come from: a range [lo, hi) whose records hold
// U distinct keys writes its terms, in key order, to slots [lo, lo + U) of
// Tkeys/Tcoef and sets oflag there.  Ranges are disjoint and ordered by key,
// so the flagged slots, read in position order, are the canonical sum.
struct L2Bufs {
    uint32_t* recA;
    uint32_t* recB;
    uint16_t* subid;
    uint32_t* ctr;  // [0] coarse-range ticket, [1] small leaves, [2] medium leaves
    StackEnt* stacks;
    uint64_t* spl;
    uint64_t* Tkeys;
    double2* Tcoef;
    uint8_t* oflag;
    uint2* small;  // ranges for one warp: {lo, n | uniform << 30 | buffer << 31}
    uint2* med;    // leaves for one CTA
    uint32_t small_cap, med_cap;
    int32_t* err;
    // Test settings (paulib_set_debug): the warp leaves' key hashes are
    // and-ed with hash_mask (narrow masks force the hash-clash path), and a
    // range CTA's worklist holds stack_cap entries (at most kStackCap).
    uint64_t hash_mask = ~0ull;
    uint32_t stack_cap = (uint32_t)kStackCap;
};

// Applies the test settings of paulib_set_debug to a launch's buffers.
inline void apply_debug(L2Bufs& b) {
    const DebugSettings d = debug_settings();
    if (d.hash_bits > 0 && d.hash_bits < 64) b.hash_mask = (1ull << d.hash_bits) - 1ull;
    if (d.stack_cap > 0 && d.stack_cap < kStackCap) b.stack_cap = (uint32_t)d.stack_cap;
}

// ---- block leaf: one CTA orders a range of at most CAP records in shared
// memory and sums each run of equal keys with a block segmented scan.
template <class Src, int MODE, int T, uint32_t CAP>
__device__ void block_leaf(const Src& src, const uint32_t* cur, uint32_t lo, uint32_t n, unsigned char* smem,
                           BlockShared<MODE, Src::NW>& sh, uint64_t* Tkeys, double2* Tcoef, uint8_t* oflag) {
    using V = typename Src::V;
    constexpr int NW = Src::NW;
    constexpr uint32_t ACT = CAP < (uint32_t)T ? CAP : (uint32_t)T;
    constexpr uint32_t PP = CAP / ACT;  // sorted positions per active thread
    uint64_t* keys_s = reinterpret_cast<uint64_t*>(smem);        // [NW][CAP]
    uint64_t* c1s = keys_s + (size_t)CAP * NW;                   // [2][CAP] codes
    uint32_t* rec_s = reinterpret_cast<uint32_t*>(c1s + 2 * CAP);  // [CAP]
    uint16_t* ord_s = reinterpret_cast<uint16_t*>(rec_s + CAP);  // [CAP]
    uint16_t* tmp_s = ord_s + CAP;                               // [CAP]
    uint8_t* ph_s = reinterpret_cast<uint8_t*>(tmp_s + CAP);     // [CAP]
    const int tid = threadIdx.x;
    const bool act = (uint32_t)tid < ACT;
    for (uint32_t t = tid; t < n; t += T) {
        uint64_t k[NW];
        const uint32_t r = cur[lo + t];
        rec_s[t] = r;
        ph_s[t] = (uint8_t)src.keyphase(r, k);
        skey_store<NW>(keys_s, CAP, t, k);
    }
    uint32_t size = 64u;
    while (size < n) size <<= 1;
    __syncthreads();
    build_codes<NW, T, CAP>(c1s, keys_s, n, sh.orr, sh.L);
    const int w0 = (int)((sh.L[1] + 64u) >> 6);
    const uint16_t* srt = merge_sort_slots<NW, T, CAP>(ord_s, tmp_s, c1s, keys_s, n, size, rec_s, w0);
    const uint32_t p0 = (uint32_t)tid * PP;
    bool hd[PP];
    V v[PP];
    uint32_t sl[PP];
    uint32_t nh = 0;
#pragma unroll
    for (uint32_t q = 0; q < PP; ++q) {
        const uint32_t p = p0 + q;
        hd[q] = false;
        if (act && p < n) {
            sl[q] = srt[p];
            v[q] = src.coefv(rec_s[sl[q]], ph_s[sl[q]]);
            hd[q] = (p == 0) || slot_key_neq<NW, CAP>(sl[q], srt[p - 1], c1s, keys_s, w0);
            nh += hd[q] ? 1u : 0u;
        }
    }
    Acc<MODE> trail;
#pragma unroll
    for (uint32_t q = 0; q < PP; ++q) {
        if (act && p0 + q < n) {
            if (hd[q]) trail = Acc<MODE>();
            trail.add(v[q]);
        }
    }
    uint32_t total;
    const uint32_t hex = block_excl_scan<T>(nh, sh.warp, total);
    Acc<MODE> run = block_seg_carry<T, MODE>(nh > 0, trail, sh.acc, sh.flag);
    uint64_t oidx = (uint64_t)lo + hex - 1;  // slot of the run flowing in (if any)
#pragma unroll
    for (uint32_t q = 0; q < PP; ++q) {
        const uint32_t p = p0 + q;
        if (act && p < n) {
            if (hd[q]) {
                run = Acc<MODE>();
                ++oidx;
            }
            run.add(v[q]);
            bool last = p + 1 >= n;
            if (!last) {
                if (q + 1 < PP) last = hd[q + 1];
                else last = slot_key_neq<NW, CAP>(srt[p + 1], sl[q], c1s, keys_s, w0);
            }
            if (last) {
                uint64_t k[NW];
                skey_load<NW>(keys_s, CAP, sl[q], k);
                key_store<NW>(Tkeys, oidx, k);
                Tcoef[oidx] = run.result();
                oflag[oidx] = 1;
            }
        }
    }
    __syncthreads();
}

// ---- warp leaves
//
// A range of at most WL records is ordered and merged by one warp with no
// block barrier: the warp gathers its keys into a private shared-memory
// slice, builds 64-bit codes after the range's common prefix, sorts
// (code, slot) pairs with a register/shuffle bitonic network over WL
// positions (lane l holds positions e*32 + l), and sums equal-key runs with a
// segmented warp scan.  Outputs go to the staging slots [lo, lo + U) of the
// range and are marked in the output-flag array.

// A sort entry: one or two 64-bit codes and the slot it came from.
struct WE {
    uint64_t c, c2;
    uint32_t s;
};

// K: 1 = one code, 2 = two codes, 3 = two codes then the remaining words.
template <int K>
__device__ __forceinline__ WE we_shfl_xor(const WE& v, int m) {
    WE r;
    r.c = __shfl_xor_sync(0xffffffffu, v.c, m);
    r.c2 = K >= 2 ? __shfl_xor_sync(0xffffffffu, v.c2, m) : 0ull;
    r.s = __shfl_xor_sync(0xffffffffu, v.s, m);
    return r;
}
template <int K>
__device__ __forceinline__ WE we_shfl(const WE& v, int src) {
    WE r;
    r.c = __shfl_sync(0xffffffffu, v.c, src);
    r.c2 = K >= 2 ? __shfl_sync(0xffffffffu, v.c2, src) : 0ull;
    r.s = __shfl_sync(0xffffffffu, v.s, src);
    return r;
}
template <int K>
__device__ __forceinline__ WE we_shfl_up(const WE& v, int d) {
    WE r;
    r.c = __shfl_up_sync(0xffffffffu, v.c, d);
    r.c2 = K >= 2 ? __shfl_up_sync(0xffffffffu, v.c2, d) : 0ull;
    r.s = __shfl_up_sync(0xffffffffu, v.s, d);
    return r;
}

// Order of two sort entries: by the codes, then (K = 3) by the key words
// from w0 on, then by record number (phase-2 entries: padding last).
// Phase-1 and direct entries hold a slot in s; padding slots carry all-ones
// codes and record number 0xffffffff, so they sort after every real entry.
// Phase-2 entries hold (slot | position << 8) in s, with bit 31 marking
// padding; they are distinct keys and never tie.
template <int NW, uint32_t WL, int K, bool PH2>
__device__ __forceinline__ bool we_gt(const WE& a, const WE& b, const uint64_t* wk, const uint32_t* wr, int w0) {
    if (a.c != b.c) return a.c > b.c;
    if constexpr (K >= 2) {
        if (a.c2 != b.c2) return a.c2 > b.c2;
    }
    if constexpr (PH2) {
        const uint32_t pa = a.s >> 31, pb = b.s >> 31;
        if constexpr (K == 3) {
            if (!(pa | pb)) {
                const int c = skey_cmp_from<NW>(wk, WL, a.s & 0xffu, b.s & 0xffu, w0);
                if (c) return c > 0;
            }
        }
        return pa > pb;
    } else {
        const uint32_t ra = wr[a.s], rb = wr[b.s];
        if constexpr (K == 3) {
            if (ra != 0xffffffffu && rb != 0xffffffffu) {
                const int c = skey_cmp_from<NW>(wk, WL, a.s, b.s, w0);
                if (c) return c > 0;
            }
        }
        return ra > rb;
    }
}

// Compare-exchange of rows e and e | D (positions 32*D apart) in a
// bitonic stage of block size kk.
template <int NW, uint32_t WL, uint32_t EPL, uint32_t D, int K, bool PH2>
__device__ __forceinline__ void rows_cx(WE (&x)[EPL], uint32_t kk, uint32_t lane, const uint64_t* wk,
                                        const uint32_t* wr, int w0) {
#pragma unroll
    for (uint32_t e = 0; e < EPL; ++e) {
        if ((e & D) == 0 && (e | D) < EPL) {
            const uint32_t e2 = e | D;
            const bool up = ((e * 32u + lane) & kk) == 0;
            if (we_gt<NW, WL, K, PH2>(x[e], x[e2], wk, wr, w0) == up) {
                const WE t = x[e];
                x[e] = x[e2];
                x[e2] = t;
            }
        }
    }
}

// Bitonic network over 32*EPL positions g = e*32 + lane.  The stage loops
// stay rolled so that the code stays small.
template <int NW, uint32_t WL, uint32_t EPL, int K, bool PH2>
__device__ __forceinline__ void warp_sort(WE (&x)[EPL], uint32_t lane, const uint64_t* wk, const uint32_t* wr,
                                          int w0) {
#pragma unroll 1
    for (uint32_t kk = 2; kk <= 32u * EPL; kk <<= 1) {
#pragma unroll 1
        for (uint32_t jj = kk >> 1; jj > 0; jj >>= 1) {
            if (jj >= 32) {
                if constexpr (EPL >= 2) {
                    if (jj == 32) rows_cx<NW, WL, EPL, 1, K, PH2>(x, kk, lane, wk, wr, w0);
                }
                if constexpr (EPL >= 4) {
                    if (jj == 64) rows_cx<NW, WL, EPL, 2, K, PH2>(x, kk, lane, wk, wr, w0);
                }
            } else {
#pragma unroll
                for (uint32_t e = 0; e < EPL; ++e) {
                    const uint32_t g = e * 32u + lane;
                    const WE y = we_shfl_xor<K>(x[e], (int)jj);
                    const bool keep_min = ((lane & jj) == 0) == ((g & kk) == 0);
                    if (keep_min == we_gt<NW, WL, K, PH2>(x[e], y, wk, wr, w0)) x[e] = y;
                }
            }
        }
    }
}

// Run heads in position order: position g starts a run when its entry's
// codes (and for K = 3 its key words from w0 on) differ from position g-1's.
// With VERIFY (phase 1, K = 1 on key hashes), equal hashes are checked
// against the whole keys; the return value reports a mismatch.
template <int NW, uint32_t WL, uint32_t EPL, int K, bool VERIFY>
__device__ __forceinline__ bool warp_heads(const WE (&x)[EPL], bool (&hd)[EPL], uint32_t lane, uint32_t n,
                                           const uint64_t* wk, int w0) {
    bool bad = false;
#pragma unroll
    for (uint32_t e = 0; e < EPL; ++e) {
        WE prev = we_shfl_up<K>(x[e], 1);
        if (e > 0) {
            const WE last = we_shfl<K>(x[e - 1], 31);
            if (lane == 0) prev = last;
        }
        const uint32_t g = e * 32u + lane;
        bool h = false;
        if (g < n) {
            h = g == 0 || x[e].c != prev.c;
            if constexpr (K >= 2) h = h || x[e].c2 != prev.c2;
            if constexpr (K == 3) {
                if (!h) h = skey_cmp_from<NW>(wk, WL, x[e].s, prev.s, w0) != 0;
            }
            if constexpr (VERIFY) {
                if (!h && skey_cmp_from<NW>(wk, WL, x[e].s, prev.s, w0) != 0) bad = true;
            }
        }
        hd[e] = h;
    }
    if constexpr (VERIFY) return __any_sync(0xffffffffu, bad);
    return false;
}

// Value of slot s from the gather layout (slot t lives in row t/32 of lane
// t%32).  Called by all lanes.
template <class V, uint32_t EPL>
__device__ __forceinline__ V fetch_v(const V (&vr)[EPL], uint32_t s) {
    V out = vr[0];
    const int srcl = (int)(s & 31u);
#pragma unroll
    for (uint32_t r = 0; r < EPL; ++r) {
        V t;
        t.x = __shfl_sync(0xffffffffu, vr[r].x, srcl);
        t.y = __shfl_sync(0xffffffffu, vr[r].y, srcl);
        if (r == (s >> 5)) out = t;
    }
    return out;
}

// Segmented sums of the sorted entries' values over runs of equal keys.
// DIRECT writes each run's term to slot lo + (run index); otherwise the run
// total stays in acc[e] at the run's last position and repl[run index]
// records (slot | position << 8) of that position.  Returns the run count.
template <class Src, int MODE, int NW, uint32_t WL, uint32_t EPL, bool DIRECT>
__device__ __forceinline__ uint32_t warp_run_sums(const typename Src::V (&vr)[EPL], const WE (&x)[EPL],
                                                  const bool (&hd)[EPL], Acc<MODE> (&acc)[EPL], uint32_t lane,
                                                  uint32_t n, uint32_t lo, const uint64_t* wk, uint16_t* repl,
                                                  uint64_t* Tkeys, double2* Tcoef, uint8_t* oflag) {
    using V = typename Src::V;
    const uint32_t lt_mask = (1u << lane) - 1u;
    V vv[EPL];
    bool cont[EPL];  // position continues a run
#pragma unroll
    for (uint32_t e = 0; e < EPL; ++e) {
        vv[e] = fetch_v<V, EPL>(vr, x[e].s);
        cont[e] = e * 32u + lane < n && !hd[e];
    }
    // Fast path: every run holds one or two records (each string of H*H
    // typically arises from P_aP_b and P_bP_a), so a run's total is its last
    // value plus, for a two-record run, the value before it.
    bool longer = false;
#pragma unroll
    for (uint32_t e = 0; e < EPL; ++e) {
        bool pc = __shfl_up_sync(0xffffffffu, cont[e], 1);
        const bool pc_row = __shfl_sync(0xffffffffu, cont[e > 0 ? e - 1 : 0], 31);
        if (lane == 0) pc = e > 0 ? pc_row : false;
        longer = longer || (cont[e] && pc);
    }
    if (!__any_sync(0xffffffffu, longer)) {
        uint32_t heads = 0;
#pragma unroll
        for (uint32_t e = 0; e < EPL; ++e) {
            const uint32_t g = e * 32u + lane;
            const bool valid = g < n;
            V pv;
            pv.x = __shfl_up_sync(0xffffffffu, vv[e].x, 1);
            pv.y = __shfl_up_sync(0xffffffffu, vv[e].y, 1);
            const V& prow = vv[e > 0 ? e - 1 : 0];
            const auto px = __shfl_sync(0xffffffffu, prow.x, 31);
            const auto py = __shfl_sync(0xffffffffu, prow.y, 31);
            if (lane == 0) {
                pv.x = px;
                pv.y = py;
            }
            Acc<MODE> a;
            if (valid) {
                if (!hd[e]) a.add(pv);  // record order: the run's first value, then its second
                a.add(vv[e]);
            }
            const uint32_t hb = __ballot_sync(0xffffffffu, hd[e]);
            const uint32_t oidx = heads + __popc(hb & lt_mask) + (hd[e] ? 1u : 0u) - 1u;
            const bool nh_same = __shfl_down_sync(0xffffffffu, hd[e], 1);
            const bool nh_next = __shfl_sync(0xffffffffu, hd[e + 1 < EPL ? e + 1 : e], 0);
            const bool next_head = lane < 31 ? nh_same : (e + 1 < EPL ? nh_next : false);
            const bool last = valid && (g + 1 >= n || next_head);
            if (last) {
                if constexpr (DIRECT) {
                    uint64_t k[NW];
                    skey_load<NW>(wk, WL, x[e].s, k);
                    key_store<NW>(Tkeys, (uint64_t)lo + oidx, k);
                    Tcoef[(uint64_t)lo + oidx] = a.result();
                    oflag[(uint64_t)lo + oidx] = 1;
                } else {
                    repl[oidx] = (uint16_t)(x[e].s | (g << 8));
                }
            }
            acc[e] = a;
            heads += __popc(hb);
        }
        return heads;
    }
    Acc<MODE> carry;
    uint32_t heads_before = 0;
#pragma unroll
    for (uint32_t e = 0; e < EPL; ++e) {
        const uint32_t g = e * 32u + lane;
        const bool valid = g < n;
        Acc<MODE> a;
        if (valid) a.add(vv[e]);
        bool f = hd[e];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const Acc<MODE> y = a.up(o);
            const bool fy = __shfl_up_sync(0xffffffffu, f, o);
            if (lane >= (uint32_t)o) {
                if (!f) {
                    Acc<MODE> t2 = y;
                    t2.merge(a);
                    a = t2;
                }
                f = f || fy;
            }
        }
        if (!f) {  // no run starts at or before this lane in the row: the open run flows in
            Acc<MODE> t2 = carry;
            t2.merge(a);
            a = t2;
        }
        const uint32_t hb = __ballot_sync(0xffffffffu, hd[e]);
        const uint32_t oidx = heads_before + __popc(hb & lt_mask) + (hd[e] ? 1u : 0u) - 1u;
        bool next_head;
        {
            const bool nh_same = __shfl_down_sync(0xffffffffu, hd[e], 1);
            bool nh_next = false;
            if (e + 1 < EPL) nh_next = __shfl_sync(0xffffffffu, hd[e + 1 < EPL ? e + 1 : e], 0);
            next_head = lane < 31 ? nh_same : nh_next;
        }
        const bool last = valid && (g + 1 >= n || next_head);
        if (last) {
            if constexpr (DIRECT) {
                uint64_t k[NW];
                skey_load<NW>(wk, WL, x[e].s, k);
                key_store<NW>(Tkeys, (uint64_t)lo + oidx, k);
                Tcoef[(uint64_t)lo + oidx] = a.result();
                oflag[(uint64_t)lo + oidx] = 1;
            } else {
                repl[oidx] = (uint16_t)(x[e].s | (g << 8));
            }
        }
        acc[e] = a;
        carry = a.bcast(31);
        heads_before += __popc(hb);
    }
    return heads_before;
}

// Phase 2: the U distinct keys, ordered by their codes, written to slots
// lo .. lo + U - 1 with the run totals held by the phase-1 lanes.
template <class Src, int MODE, int NW, uint32_t WL, uint32_t EPL, uint32_t EPL2, int K>
__device__ __forceinline__ void warp_phase2(const Acc<MODE> (&acc)[EPL], uint32_t U, uint32_t lane, uint32_t lo,
                                            const uint64_t* wk, const uint16_t* repl, uint32_t L, uint32_t L2,
                                            int w0, uint64_t* Tkeys, double2* Tcoef, uint8_t* oflag) {
    WE y[EPL2];
#pragma unroll
    for (uint32_t e = 0; e < EPL2; ++e) {
        const uint32_t u = e * 32u + lane;
        if (u < U) {
            const uint32_t rv = repl[u];
            const uint32_t sl = rv & 0xffu;
            y[e] = WE{key_bits64<NW, WL>(wk, sl, L), K >= 2 ? key_bits64<NW, WL>(wk, sl, L2) : 0ull, rv};
        } else {
            y[e] = WE{~0ull, ~0ull, 0x80000000u | u};
        }
    }
    warp_sort<NW, WL, EPL2, K, true>(y, lane, wk, nullptr, w0);
#pragma unroll
    for (uint32_t e = 0; e < EPL2; ++e) {
        const uint32_t u = e * 32u + lane;
        const uint32_t rv = y[e].s;
        const uint32_t g = (rv >> 8) & 0xffu;
        Acc<MODE> v;
#pragma unroll
        for (uint32_t r = 0; r < EPL; ++r) {
            const Acc<MODE> t = acc[r].bcast((int)(g & 31u));
            if (r == (g >> 5)) v = t;
        }
        if (u < U) {
            uint64_t k[NW];
            skey_load<NW>(wk, WL, rv & 0xffu, k);
            key_store<NW>(Tkeys, (uint64_t)lo + u, k);
            Tcoef[(uint64_t)lo + u] = v.result();
            oflag[(uint64_t)lo + u] = 1;
        }
    }
}

template <class Src, int MODE, int NW, uint32_t WL, uint32_t EPL2, uint32_t EPL>
__device__ __forceinline__ void warp_phase2_k(int K, const Acc<MODE> (&acc)[EPL], uint32_t U, uint32_t lane,
                                              uint32_t lo, const uint64_t* wk, const uint16_t* repl, uint32_t L,
                                              uint32_t L2, int w0, uint64_t* Tkeys, double2* Tcoef,
                                              uint8_t* oflag) {
    if (K == 1) warp_phase2<Src, MODE, NW, WL, EPL, EPL2, 1>(acc, U, lane, lo, wk, repl, L, L2, w0, Tkeys, Tcoef, oflag);
    else if (K == 2) warp_phase2<Src, MODE, NW, WL, EPL, EPL2, 2>(acc, U, lane, lo, wk, repl, L, L2, w0, Tkeys, Tcoef, oflag);
    else warp_phase2<Src, MODE, NW, WL, EPL, EPL2, 3>(acc, U, lane, lo, wk, repl, L, L2, w0, Tkeys, Tcoef, oflag);
}

// First position >= P (word 0's top bit is position 0) where mask m has a
// set bit, or 64*NW.
template <int NW>
__device__ __forceinline__ uint32_t first_set_from(const uint64_t (&m)[NW], uint32_t P) {
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        if (64u * w + 63u < P) continue;
        uint64_t mm = m[w];
        if (P > 64u * w) mm &= ~0ull >> (P - 64u * w);
        if (mm) return 64u * w + (uint32_t)__clzll((long long)mm);
    }
    return 64u * NW;
}

// 64-bit hash of a key (multiply-xorshift per word); equal keys hash equal.
template <int NW>
__device__ __forceinline__ uint64_t key_hash(const uint64_t (&k)[NW]) {
    uint64_t h = 0x243f6a8885a308d3ull;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        h = (h ^ k[w]) * 0x9e3779b97f4a7c15ull;
        h ^= h >> 29;
    }
    return mix64(h);
}

// One warp leaf of n <= 32*EPL records.  Phase 1 sorts (key hash, record),
// so that equal keys meet (each meeting is checked against the whole keys),
// and sums each run; phase 2 orders the distinct keys by codes of their
// varying bits.  Equal keys are frequent (e.g. both orders of a commuting
// pair) and would otherwise be compared word by word at every step of the
// network.  A hash clash between different keys falls back to one sort by
// the whole key.
template <class Src, int MODE, int NW, uint32_t WL, uint32_t EPL>
__device__ void warp_leaf_rows(const Src& src, const uint32_t* cur, uint32_t lo, uint32_t n, unsigned char* wsm,
                               uint64_t* Tkeys, double2* Tcoef, uint8_t* oflag, uint64_t hmask) {
    static_assert(EPL * 32 <= WL && WL <= 128, "network fits the slice");
    using V = typename Src::V;
    uint64_t* wk = reinterpret_cast<uint64_t*>(wsm);                   // [NW][WL]
    uint32_t* wr = reinterpret_cast<uint32_t*>(wk + (size_t)NW * WL);  // [WL]
    uint16_t* repl = reinterpret_cast<uint16_t*>(wr + WL);             // [WL]
    const uint32_t lane = threadIdx.x & 31u;
    uint64_t hh[EPL];
    V vr[EPL];  // each record's value, in the gather layout
#pragma unroll
    for (uint32_t e = 0; e < EPL; ++e) {
        const uint32_t t = e * 32u + lane;
        hh[e] = ~0ull;
        vr[e].x = 0;
        vr[e].y = 0;
        if (t < n) {
            uint64_t k[NW];
            const uint32_t r = cur[lo + t];
            wr[t] = r;
            vr[e] = src.value(r, k);
            skey_store<NW>(wk, WL, t, k);
            hh[e] = key_hash<NW>(k) & hmask;
        } else {
            wr[t] = 0xffffffffu;
        }
    }
    __syncwarp();
    // Variation mask: the positions where some key differs from key 0.  The
    // first code holds the 64 positions from the first varying one, L; the
    // second the 64 from the first varying position L2 >= L + 64.  Keys agree
    // everywhere else, up to the first varying position after L2 + 64.
    uint64_t m[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        uint64_t v = 0;
#pragma unroll
        for (uint32_t e = 0; e < EPL; ++e) {
            const uint32_t t = e * 32u + lane;
            if (t < n) v |= wk[(size_t)w * WL + t] ^ wk[(size_t)w * WL];
        }
        const uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(v >> 32));
        const uint32_t lo32 = __reduce_or_sync(0xffffffffu, (uint32_t)v);
        m[w] = ((uint64_t)hi << 32) | lo32;
    }
    const uint32_t L = first_set_from<NW>(m, 0u);
    const uint32_t L2 = L + 64u < 64u * NW ? first_set_from<NW>(m, L + 64u) : 64u * NW;
    const bool more = L2 + 64u < 64u * NW && first_set_from<NW>(m, L2 + 64u) < 64u * NW;
    const int K = L2 >= 64u * NW ? 1 : (more ? 3 : 2);
    const int w0 = (int)((L2 + 64u) >> 6);
    const int wl0 = (int)(L >> 6);  // first word where keys can differ
    WE x[EPL];
    bool hd[EPL];
    Acc<MODE> acc[EPL];
#pragma unroll
    for (uint32_t e = 0; e < EPL; ++e) {
        const uint32_t t = e * 32u + lane;
        x[e] = WE{hh[e], 0ull, t};
    }
    warp_sort<NW, WL, EPL, 1, false>(x, lane, wk, wr, 0);
    if (!warp_heads<NW, WL, EPL, 1, true>(x, hd, lane, n, wk, wl0)) {
        const uint32_t U = warp_run_sums<Src, MODE, NW, WL, EPL, false>(vr, x, hd, acc, lane, n, lo, wk, repl,
                                                                         Tkeys, Tcoef, oflag);
        __syncwarp();
        if (U <= 32u) {
            warp_phase2_k<Src, MODE, NW, WL, 1, EPL>(K, acc, U, lane, lo, wk, repl, L, L2, w0, Tkeys, Tcoef, oflag);
        } else if constexpr (EPL >= 2) {
            if (U <= 64u) {
                warp_phase2_k<Src, MODE, NW, WL, 2, EPL>(K, acc, U, lane, lo, wk, repl, L, L2, w0, Tkeys, Tcoef,
                                                         oflag);
            } else if constexpr (EPL >= 4) {
                warp_phase2_k<Src, MODE, NW, WL, 4, EPL>(K, acc, U, lane, lo, wk, repl, L, L2, w0, Tkeys, Tcoef,
                                                         oflag);
            }
        }
        __syncwarp();
        return;
    }
    // a hash clash: one sort by codes and the whole key, then direct sums
#pragma unroll
    for (uint32_t e = 0; e < EPL; ++e) {
        const uint32_t t = e * 32u + lane;
        x[e] = t < n ? WE{key_bits64<NW, WL>(wk, t, L), key_bits64<NW, WL>(wk, t, L2), t} : WE{~0ull, ~0ull, t};
    }
    warp_sort<NW, WL, EPL, 3, false>(x, lane, wk, wr, w0);
    warp_heads<NW, WL, EPL, 3, false>(x, hd, lane, n, wk, w0);
    warp_run_sums<Src, MODE, NW, WL, EPL, true>(vr, x, hd, acc, lane, n, lo, wk, repl, Tkeys, Tcoef, oflag);
    __syncwarp();
}

// A warp leaf sorts with the smallest network that holds its n records.
template <class Src, int MODE, int NW, uint32_t WL>
__device__ __forceinline__ void warp_leaf(const Src& src, const uint32_t* cur, uint32_t lo, uint32_t n,
                                          unsigned char* wsm, uint64_t* Tkeys, double2* Tcoef, uint8_t* oflag,
                                          uint64_t hmask) {
    if (n <= 32) {
        warp_leaf_rows<Src, MODE, NW, WL, 1>(src, cur, lo, n, wsm, Tkeys, Tcoef, oflag, hmask);
        return;
    }
    if constexpr (WL >= 64) {
        if (n <= 64) {
            warp_leaf_rows<Src, MODE, NW, WL, 2>(src, cur, lo, n, wsm, Tkeys, Tcoef, oflag, hmask);
            return;
        }
        if constexpr (WL >= 128)
            warp_leaf_rows<Src, MODE, NW, WL, 4>(src, cur, lo, n, wsm, Tkeys, Tcoef, oflag, hmask);
    }
}

// A range whose records all share one key, summed by one warp.
template <class Src, int MODE>
__device__ void warp_uniform(const Src& src, const uint32_t* cur, uint32_t lo, uint32_t n, uint64_t* Tkeys,
                             double2* Tcoef, uint8_t* oflag) {
    constexpr int NW = Src::NW;
    const uint32_t lane = threadIdx.x & 31u;
    Acc<MODE> acc;
    for (uint32_t t = lane; t < n; t += 32u) {
        uint64_t k[NW];
        acc.add(src.value(cur[lo + t], k));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc.shfl_merge(o);
    if (lane == 0) {
        uint64_t k[NW];
        src.key(cur[lo], k);
        key_store<NW>(Tkeys, lo, k);
        Tcoef[lo] = acc.result();
        oflag[lo] = 1;
    }
}

constexpr int kLeafThreads = 128;   // threads of the block-leaf kernel
constexpr uint32_t kUniformWarpMax = 4096;  // longest all-equal range summed by one warp
constexpr int kWarpLeafWarps = 8;   // warps per CTA of the warp-leaf kernel

// Warp-leaf capacity: up to 128 records, with each warp's slice of shared
// memory (keys, record numbers, run list) kept within 5.5 KB so that many warps
// stay resident (the leaf is bound by latency, not bandwidth).
template <int NW>
constexpr uint32_t warp_leaf_cap() {
    uint32_t wl = 128;
    while (wl > 32 && wl * (8u * NW + 6u) > 5632u) wl >>= 1;
    return wl;
}
template <int NW>
constexpr size_t warp_leaf_bytes() {
    return ((size_t)warp_leaf_cap<NW>() * (8 * NW + 6) + 15) & ~(size_t)15;
}

template <class Src, int MODE>
__global__ void __launch_bounds__(kLeafThreads) k_leaf_block(Src src, L2Bufs b) {
    using Cfg = L2Cfg<Src, MODE>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BlockShared<MODE, Cfg::NW> sh;
    const uint32_t cnt = mn<uint32_t>(b.ctr[2], b.med_cap);
    for (uint32_t e = blockIdx.x; e < cnt; e += gridDim.x) {
        const uint2 en = b.med[e];
        const uint32_t* cur = (en.y >> 31) ? b.recB : b.recA;
        block_leaf<Src, MODE, kLeafThreads, Cfg::MCAP>(src, cur, en.x, en.y & 0x7fffffffu, smem, sh, b.Tkeys,
                                                     b.Tcoef, b.oflag);
    }
}

template <class Src, int MODE>
__global__ void __launch_bounds__(kWarpLeafWarps * 32) k_leaf_warp(Src src, L2Bufs b) {
    constexpr int NW = Src::NW;
    constexpr uint32_t WL = warp_leaf_cap<NW>();
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t w = threadIdx.x >> 5;
    unsigned char* wsm = smem + (size_t)w * warp_leaf_bytes<NW>();
    const uint32_t cnt = mn<uint32_t>(b.ctr[1], b.small_cap);
    const uint32_t nwarp = gridDim.x * kWarpLeafWarps;
    for (uint32_t e = blockIdx.x * kWarpLeafWarps + w; e < cnt; e += nwarp) {
        const uint2 en = b.small[e];
        const uint32_t* cur = (en.y >> 31) ? b.recB : b.recA;
        const uint32_t n = en.y & 0x3fffffffu;
        if (en.y & 0x40000000u) warp_uniform<Src, MODE>(src, cur, en.x, n, b.Tkeys, b.Tcoef, b.oflag);
        else warp_leaf<Src, MODE, NW, WL>(src, cur, en.x, n, wsm, b.Tkeys, b.Tcoef, b.oflag, b.hash_mask);
    }
}

// ---- routing: a range that needs no split at this point goes to the leaf
// lists (or is emitted at once when it holds one record); a range to split,
// or one whose keys are all equal, goes on the CTA's stack.  Called by all
// 32 lanes of a warp; `valid` marks the lanes that hold a range.
template <class Src, int MODE, uint32_t WL, uint32_t MCAP>
__device__ __forceinline__ void route_range(const Src& src, const L2Bufs& b, bool valid, uint32_t lo, uint32_t n,
                                            uint32_t fl, StackEnt* stack, uint32_t* s_sp) {
    constexpr int NW = Src::NW;
    const uint32_t lane = threadIdx.x & 31u;
    int kind = -1;  // 0 one record, 1 warp list, 2 block leaf, 3 stack
    if (valid && n > 0) {
        if (n == 1) kind = 0;
        else if (fl & SF_UNIFORM) kind = n <= kUniformWarpMax ? 1 : 3;
        else if (n <= WL) kind = 1;
        else if (n <= MCAP) kind = 2;
        else kind = 3;
    }
    const uint32_t bufbit = ((fl & SF_INB) ? 0x80000000u : 0u) | ((fl & SF_UNIFORM) ? 0x40000000u : 0u);
    if (kind == 0) {
        const uint32_t* cur = (fl & SF_INB) ? b.recB : b.recA;
        uint64_t k[NW];
        Acc<MODE> a;
        a.add(src.value(cur[lo], k));
        key_store<NW>(b.Tkeys, lo, k);
        b.Tcoef[lo] = a.result();
        b.oflag[lo] = 1;
    }
#pragma unroll
    for (int list = 1; list <= 2; ++list) {
        const uint32_t m = __ballot_sync(0xffffffffu, kind == list);
        if (m) {
            const uint32_t leader = (uint32_t)__ffs(m) - 1u;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(&b.ctr[list], (uint32_t)__popc(m));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (kind == list) {
                const uint32_t idx = base + (uint32_t)__popc(m & ((1u << lane) - 1u));
                const uint32_t cap = list == 1 ? b.small_cap : b.med_cap;
                uint2* dst = list == 1 ? b.small : b.med;
                if (idx < cap) dst[idx] = make_uint2(lo, n | bufbit);
                else atomicOr(b.err, ERR_LIST);
            }
        }
    }
    if (kind == 3) {
        const uint32_t p = atomicAdd(s_sp, 1u);
        if (p < b.stack_cap) stack[p] = StackEnt{lo, lo + n, fl, 0u};
        else atomicOr(b.err, ERR_STACK);
    }
}

// ---- level 2: one CTA per coarse range (taken from a ticket counter) splits
// it until every piece fits a leaf.  Splitters come from a sorted sample of
// the range's own records; a key that fills a large share of the sample gets
// a range of its own, which is reduced here without sorting.
template <class Src, int MODE>
__global__ void __launch_bounds__(kL2Threads, 2) k_level2(Src src, uint32_t nbk, const uint64_t* __restrict__ boff,
                                                       const uint8_t* __restrict__ bflags, L2Bufs b,
                                                       uint32_t child_target) {
    using Cfg = L2Cfg<Src, MODE>;
    constexpr int NW = Cfg::NW;
    constexpr uint32_t CAP = Cfg::CAP;
    constexpr uint32_t WL = warp_leaf_cap<NW>();
    constexpr int T = kL2Threads;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* keys_s = reinterpret_cast<uint64_t*>(smem);        // [NW][CAP]
    uint64_t* c1s = keys_s + (size_t)CAP * NW;                   // [2][CAP] codes
    uint16_t* ord_s = reinterpret_cast<uint16_t*>(c1s + 2 * CAP);  // [CAP]
    uint16_t* tmp_s = ord_s + CAP;                               // [CAP]
    uint8_t* fl_s = reinterpret_cast<uint8_t*>(tmp_s + CAP);     // [CAP]: flag of range p+1 follows splitter p
    __shared__ BlockShared<MODE, NW> sh;
    __shared__ uint32_t s_bucket, s_lo, s_hi, s_fl, s_sp, s_done, s_bad;

    StackEnt* stack = b.stacks + (size_t)blockIdx.x * kStackCap;
    uint64_t* my_spl = b.spl + (size_t)blockIdx.x * (CAP / 2) * NW;
    const int tid = threadIdx.x;

    for (;;) {
        if (tid == 0) {
            s_bucket = atomicAdd(&b.ctr[0], 1u);
            s_sp = 0;
            s_bad = 0;
        }
        __syncthreads();
        const uint32_t c = s_bucket;
        if (c >= nbk) break;
        if (tid < 32) {
            const uint64_t base0 = boff[c], end0 = boff[c + 1];
            route_range<Src, MODE, WL, Cfg::MCAP>(src, b, tid == 0, (uint32_t)base0, (uint32_t)(end0 - base0),
                                            bflags[c] ? SF_UNIFORM : 0u, stack, &s_sp);
        }
        __syncthreads();
        uint32_t iters = 0;
        for (;;) {
            if (tid == 0) {
                if (s_sp == 0 || s_bad || s_sp > b.stack_cap) {
                    s_done = 1;
                } else {
                    const StackEnt e = stack[--s_sp];
                    s_lo = e.lo;
                    s_hi = e.hi;
                    s_fl = e.flags;
                    s_done = 0;
                }
            }
            __syncthreads();
            if (s_done) break;
            if (++iters > (1u << 24)) {
                if (tid == 0) atomicOr(b.err, ERR_ITER);
                break;
            }
            const uint32_t lo = s_lo, hi = s_hi, fl = s_fl;
            const uint32_t n = hi - lo;
            uint32_t* cur = (fl & SF_INB) ? b.recB : b.recA;
            uint32_t* oth = (fl & SF_INB) ? b.recA : b.recB;

            if (fl & SF_UNIFORM) {
                // ---- every record in the range has the same key
                Acc<MODE> acc;
                for (uint32_t t = tid; t < n; t += T) {
                    uint64_t k[NW];
                    acc.add(src.value(cur[lo + t], k));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc.shfl_merge(o);
                if ((tid & 31) == 0) sh.acc[tid >> 5] = acc;
                __syncthreads();
                if (tid < 32) {
                    Acc<MODE> a2;
                    if (tid < T / 32) a2 = sh.acc[tid];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) a2.shfl_merge(o);
                    if (tid == 0) {
                        uint64_t k[NW];
                        src.key(cur[lo], k);
                        key_store<NW>(b.Tkeys, lo, k);
                        b.Tcoef[lo] = a2.result();
                        b.oflag[lo] = 1;
                    }
                }
                __syncthreads();
                continue;
            }
            // ---- split: splitters from a sorted sample of this range
            static_assert(CAP / 4 <= (uint32_t)T, "one splitter candidate per thread");
            const uint32_t want = (uint32_t)mn<uint64_t>(
                CAP / 4, ((uint64_t)n + child_target - 1) / child_target > 2 ? ((uint64_t)n + child_target - 1) / child_target : 2);
            uint32_t S = 64;
            while (S < 16u * want && S < CAP) S <<= 1;
            for (uint32_t t = tid; t < S; t += T) {
                const uint32_t pos = lo + (uint32_t)(((uint64_t)t * n) / S);
                uint64_t k[NW];
                src.key(cur[pos], k);
                skey_store<NW>(keys_s, CAP, t, k);
            }
            __syncthreads();
            build_codes<NW, T, CAP>(c1s, keys_s, S, sh.orr, sh.L);
            const int w0 = (int)((sh.L[1] + 64u) >> 6);
            const uint16_t* srt = merge_sort_slots<NW, T, CAP>(ord_s, tmp_s, c1s, keys_s, S, S, nullptr, w0);
            // Candidate t (1 <= t < want) is the key at sample rank t*S/want.
            // A candidate equal to the one before it adds nothing; a key whose
            // run in the sample covers half a target range or more is heavy and
            // adds the pair (key, successor), so that it gets a range of its own.
            {
                const uint32_t heavy_min = mn<uint32_t>(S, S / (2u * want) > 2u ? S / (2u * want) : 2u);
                const uint32_t t = (uint32_t)tid + 1u;
                uint32_t emit = 0;
                bool heavy = false, has_succ = false;
                uint64_t k[NW], s2[NW];
                if (t < want) {
                    const uint32_t rho = (uint32_t)(((uint64_t)t * S) / want);
                    const uint32_t ci = srt[rho];
                    const uint32_t rp = (uint32_t)(((uint64_t)(t - 1) * S) / want);
                    if (t == 1 || slot_key_cmp<NW, CAP>(srt[rp], ci, c1s, keys_s, w0) != 0) {
                        skey_load<NW>(keys_s, CAP, ci, k);
                        uint32_t a0 = 0, a1 = rho;  // first sample rank holding this key
                        while (a0 < a1) {
                            const uint32_t mid = (a0 + a1) >> 1;
                            if (slot_key_cmp<NW, CAP>(srt[mid], ci, c1s, keys_s, w0) < 0) a0 = mid + 1;
                            else a1 = mid;
                        }
                        uint32_t b0 = rho, b1 = S - 1;  // last sample rank holding it
                        while (b0 < b1) {
                            const uint32_t mid = (b0 + b1 + 1) >> 1;
                            if (slot_key_cmp<NW, CAP>(srt[mid], ci, c1s, keys_s, w0) > 0) b1 = mid - 1;
                            else b0 = mid;
                        }
                        heavy = b0 - a0 + 1 >= heavy_min;
                        has_succ = heavy && key_succ<NW>(k, s2);
                        emit = has_succ ? 2u : 1u;
                    }
                }
                uint32_t nsp_total;
                const uint32_t pos = block_excl_scan<T>(emit, sh.warp, nsp_total);
                if (emit) {
                    key_store<NW>(my_spl, pos, k);
                    fl_s[pos + 1] = heavy ? 1u : 0u;  // [key, next splitter) holds only this key
                    if (has_succ) {
                        key_store<NW>(my_spl, pos + 1, s2);
                        fl_s[pos + 2] = 0;
                    }
                }
                if (tid == 0) {
                    fl_s[0] = 0;
                    s_done = nsp_total;  // splitter count, read after the barrier
                }
            }
            __syncthreads();
            const uint32_t nsp = s_done;
            const uint32_t nbs = nsp + 1;
            for (uint32_t q = tid; q < nsp * NW; q += T) keys_s[(q % NW) * (CAP / 2) + q / NW] = my_spl[q];
            uint32_t* cnt = reinterpret_cast<uint32_t*>(c1s);    // [CAP / 2]
            uint32_t* cpos = cnt + CAP / 2;                      // [CAP / 2]
            uint64_t* sc = reinterpret_cast<uint64_t*>(cpos + CAP / 2);  // [CAP / 2] splitter codes
            for (uint32_t q = tid; q < nbs; q += T) {
                cnt[q] = 0;
                cpos[q] = 0;
            }
            __syncthreads();
            // The splitters share their first Ls bits.  A key whose first Ls
            // bits differ from theirs lies below or above all of them; other
            // keys are located by the 64 bits that follow (their code), with
            // the whole key deciding only when a code equals a splitter's.
            uint32_t Ls = 64u * NW;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const uint64_t d = keys_s[(size_t)w * (CAP / 2)] ^ keys_s[(size_t)w * (CAP / 2) + nsp - 1];
                if (d) {
                    Ls = 64u * w + (uint32_t)__clzll((long long)d);
                    break;
                }
            }
            for (uint32_t q = tid; q < nsp; q += T) sc[q] = key_bits64<NW, CAP / 2>(keys_s, q, Ls);
            __syncthreads();
            for (uint32_t idx = lo + tid; idx < hi; idx += T) {
                uint64_t k[NW];
                src.key(cur[idx], k);
                uint32_t bb;
                const int pc = prefix_cmp<NW>(k, keys_s, CAP / 2, Ls);
                if (pc != 0) {
                    bb = pc < 0 ? 0u : nsp;
                } else {
                    const uint64_t code = reg_bits64<NW>(k, Ls);
                    uint32_t l2 = 0, len = nsp;
                    while (len > 0) {
                        const uint32_t half = len >> 1, mid = l2 + half;
                        const uint64_t sv = sc[mid];
                        const bool ge = code != sv ? code > sv : skey_cmp_r<NW>(k, keys_s, CAP / 2, mid) >= 0;
                        if (ge) {
                            l2 = mid + 1;
                            len -= half + 1;
                        } else {
                            len = half;
                        }
                    }
                    bb = l2;
                }
                b.subid[idx] = (uint16_t)bb;
                atomicAdd(&cnt[bb], 1u);
            }
            __syncthreads();
            {  // exclusive scan of the child counts, in place; a child that got
               // every record without being uniform means no progress
                const uint32_t per = (nbs + T - 1) / T;
                const uint32_t q0 = (uint32_t)tid * per;
                uint32_t loc = 0;
                for (uint32_t q = q0; q < q0 + per && q < nbs; ++q) {
                    const uint32_t cb = cnt[q];
                    if (cb == n && !(fl_s[q] & 1u)) s_bad = 1;
                    loc += cb;
                }
                uint32_t tot;
                uint32_t ex = block_excl_scan<T>(loc, sh.warp, tot);
                for (uint32_t q = q0; q < q0 + per && q < nbs; ++q) {
                    const uint32_t cb = cnt[q];
                    cnt[q] = ex;
                    ex += cb;
                }
            }
            __syncthreads();
            if (s_bad) {
                if (tid == 0) atomicOr(b.err, ERR_PROGRESS);
                continue;
            }
            for (uint32_t idx = lo + tid; idx < hi; idx += T) {
                const uint32_t bb = b.subid[idx];
                const uint32_t p = atomicAdd(&cpos[bb], 1u);
                oth[lo + cnt[bb] + p] = cur[idx];
            }
            __syncthreads();
            const uint32_t inb = (fl & SF_INB) ? 0u : SF_INB;  // children live in the other buffer
            for (uint32_t q0 = 0; q0 < nbs; q0 += T) {
                const uint32_t q = q0 + tid;
                const bool valid = q < nbs;
                uint32_t s0 = 0, s1 = 0, cf = 0;
                if (valid) {
                    s0 = cnt[q];
                    s1 = q + 1 < nbs ? cnt[q + 1] : n;
                    cf = ((fl_s[q] & 1u) ? SF_UNIFORM : 0u) | inb;
                }
                route_range<Src, MODE, WL, Cfg::MCAP>(src, b, valid, lo + s0, s1 - s0, cf, stack, &s_sp);
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------- compaction
//
// The flagged staging slots, in position order, are the merged terms.  The
// flag array is split into chunks of kChunk slots; a count pass and a scan
// give each chunk its first output index, and the copy kernels walk a chunk
// with one block scan.

constexpr uint32_t kChunk = 8192;  // 256 threads x 32 flags
constexpr int kChunkThreads = 256;

static __global__ void __launch_bounds__(kChunkThreads) k_flag_count(const uint8_t* __restrict__ oflag, uint32_t nch,
                                                              uint32_t* cnt) {
    __shared__ uint32_t s_w[kChunkThreads / 32];
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
        const uint4* f = reinterpret_cast<const uint4*>(oflag + (size_t)c * kChunk + (size_t)threadIdx.x * 32u);
        const uint4 a = f[0], b2 = f[1];
        // flags are 0 or 1 bytes: the bit count of a word is its flag count
        uint32_t v = __popc(a.x) + __popc(a.y) + __popc(a.z) + __popc(a.w) + __popc(b2.x) + __popc(b2.y) +
                     __popc(b2.z) + __popc(b2.w);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t s = 0;
            for (int w = 0; w < kChunkThreads / 32; ++w) s += s_w[w];
            cnt[c] = s;
        }
        __syncthreads();
    }
}

// Calls f(slot, output index) for every flagged slot of chunk c.  Warp w
// walks slots [c*kChunk + 1024w, +1024) in rows of 32 consecutive slots, so
// that reads of the staging arrays and writes of the output are coalesced.
// Called by the whole CTA.
template <class F>
__device__ __forceinline__ void for_each_flagged(uint32_t c, const uint8_t* __restrict__ oflag,
                                                 const uint64_t* __restrict__ coff, uint32_t* s_warp, F&& f) {
    static_assert(kChunk == 1024u * (kChunkThreads / 32), "one 1024-slot segment per warp");
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const uint64_t base = (uint64_t)c * kChunk + (uint64_t)w * 1024u;
    uint32_t mask = 0;  // bit i: slot base + 32i + lane is flagged
#pragma unroll
    for (int i = 0; i < 32; ++i) mask |= (uint32_t)(oflag[base + (uint64_t)i * 32u + lane] != 0) << i;
    const uint32_t wtot = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(mask));
    __syncthreads();  // s_warp may still be read for the previous chunk
    if (lane == 0) s_warp[w] = wtot;
    __syncthreads();
    uint32_t wbase = 0;
    for (uint32_t q = 0; q < w; ++q) wbase += s_warp[q];
    uint64_t r = coff[c] + wbase;
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll 4
    for (int i = 0; i < 32; ++i) {
        const bool fl = (mask >> i) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, fl);
        if (fl) f(base + (uint64_t)i * 32u + lane, r + (uint32_t)__popc(bal & lt));
        r += (uint32_t)__popc(bal);
    }
}

template <int WP>
__global__ void __launch_bounds__(kChunkThreads) k_compact(uint32_t nch, const uint8_t* __restrict__ oflag,
                                                         const uint64_t* __restrict__ coff,
                                                         const uint64_t* __restrict__ Tkeys,
                                                         const double2* __restrict__ Tcoef, uint64_t* okeys,
                                                         double2* ocoef, uint8_t* opb) {
    constexpr int NW = 2 * WP;
    __shared__ uint32_t s_warp[32];
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
        for_each_flagged(c, oflag, coff, s_warp, [&](uint64_t p, uint64_t d) {
            uint64_t k[NW];
            key_load_g<NW>(Tkeys, p, k);
            key_store<NW>(okeys, d, k);
            ocoef[d] = Tcoef[p];
            opb[d] = (uint8_t)normal_phase<WP>(k, 0u);
        });
    }
}

// Copies the merged (key, coefficient) pairs into dense arrays (the merged
// sample inside splitter selection).
template <int NW>
__global__ void __launch_bounds__(kChunkThreads) k_compact_plain(uint32_t nch, const uint8_t* __restrict__ oflag,
                                                               const uint64_t* __restrict__ coff,
                                                               const uint64_t* __restrict__ Tkeys,
                                                               const double2* __restrict__ Tcoef, uint64_t* okeys,
                                                               double2* ocoef) {
    __shared__ uint32_t s_warp[32];
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
        for_each_flagged(c, oflag, coff, s_warp, [&](uint64_t p, uint64_t d) {
            uint64_t k[NW];
            key_load_g<NW>(Tkeys, p, k);
            key_store<NW>(okeys, d, k);
            ocoef[d] = Tcoef[p];
        });
    }
}

template <int MODE>
__global__ void k_to_f32(const double2* __restrict__ in, float2* out, int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = make_float2(__double2float_rn(in[t].x), __double2float_rn(in[t].y));
}

// ---------------------------------------------------------------- host pipeline

// Opt a kernel into more than 48 KB of dynamic shared memory.  Attributes
// persist, so a capture-safe (replayed) launch skips the call.
template <class F>
static void smem_attr(F* kern, size_t bytes) {
    if (capture_safe()) return;
    check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes), "attr");
}

static __global__ void k_or_err(const int32_t* inner, int32_t* outer) {
    if (threadIdx.x == 0 && *inner) atomicOr(outer, *inner);
}

struct Staged {
    // merged terms at the flagged slots of Tkeys/Tcoef; the flagged slots of
    // chunk c start at output index coff[c], and coff[nch] is their count
    Scratch Tkeys, Tcoef, oflag, coff, err;
    uint32_t nch = 0;
};

// Level 2, both leaf kernels, and the chunk offsets of the flagged slots.
// b.oflag (nch * kChunk bytes), b.ctr (3 words) and b.err start at zero.
template <class Src, int MODE>
static void launch_level2(const Src& src, uint32_t nbk, const uint64_t* boff, const uint8_t* bflags, const L2Bufs& b,
                          unsigned grid2, uint32_t nch, uint32_t* ccount, uint64_t* coff, cudaStream_t st) {
    using Cfg = L2Cfg<Src, MODE>;
    constexpr int NW = Src::NW;
    constexpr uint32_t WL = warp_leaf_cap<NW>();
    const int sms = device_sm_count();
    {
        StageScope ss(ST_LEVEL2, st);
        auto k2 = k_level2<Src, MODE>;
        smem_attr(k2, Cfg::SMEM);
        note_launch(ST_LEVEL2);
        k2<<<grid2, kL2Threads, Cfg::SMEM, st>>>(src, nbk, boff, bflags, b, (WL * 5) / 8);
        check_cuda(cudaGetLastError(), "k_level2");
    }
    {
        StageScope ss(ST_LEAF, st);
        auto kb = k_leaf_block<Src, MODE>;
        smem_attr(kb, Cfg::MSMEM);
        const unsigned per_sm_b = (unsigned)std::max<size_t>(1, std::min<size_t>(8, (200u * 1024u) / Cfg::MSMEM));
        note_launch(ST_LEAF);
        kb<<<(unsigned)sms * per_sm_b, kLeafThreads, Cfg::MSMEM, st>>>(src, b);
        check_cuda(cudaGetLastError(), "k_leaf_block");
        auto kw = k_leaf_warp<Src, MODE>;
        const size_t wsm = (size_t)kWarpLeafWarps * warp_leaf_bytes<NW>();
        smem_attr(kw, wsm);
        const unsigned per_sm = (unsigned)std::max<size_t>(1, std::min<size_t>(8, (200u * 1024u) / wsm));
        note_launch(ST_LEAF);
        kw<<<(unsigned)sms * per_sm, kWarpLeafWarps * 32, wsm, st>>>(src, b);
        check_cuda(cudaGetLastError(), "k_leaf_warp");
    }
    StageScope ss(ST_COMPACT, st);
    note_launch(ST_COMPACT);
    note_launch(ST_COMPACT);
    k_flag_count<<<std::max<uint32_t>(1, std::min<uint32_t>(nch, (uint32_t)sms * 8)), kChunkThreads, 0, st>>>(
        b.oflag, nch, ccount);
    k_scan_counts<<<1, 1024, 0, st>>>(ccount, nch, coff);
    check_cuda(cudaGetLastError(), "flag scan");
}

template <class Src>
struct IsProd : std::false_type {};
template <int WP, int MODE>
struct IsProd<ProdSrc<WP, MODE>> : std::true_type {};

static uint64_t g_sample_seed = 0x5eed5eedull;

template <class Src, int MODE>
static void run_pipeline(const Src& src, uint32_t R, uint32_t nb_terms, cudaStream_t st, Staged& out);

// Sorted distinct sample keys with their multiplicities.
template <int NW>
static void sorted_sample(const uint64_t* samp, uint32_t S, cudaStream_t st, Scratch& dk, Scratch& dc,
                          Scratch& du, int32_t* outer_err) {
    SampleSrc<NW> ts{samp};
    Staged sg;
    run_pipeline<SampleSrc<NW>, M_FP64>(ts, S, 0, st, sg);
    dk = Scratch((size_t)S * NW * 8, st);
    dc = Scratch((size_t)S * 16, st);
    du = Scratch(8, st);
    note_launch(ST_SAMPLE);
    k_compact_plain<NW><<<std::min<uint32_t>(sg.nch, 1024), kChunkThreads, 0, st>>>(
        sg.nch, sg.oflag.as<uint8_t>(), sg.coff.as<uint64_t>(), sg.Tkeys.as<uint64_t>(), sg.Tcoef.as<double2>(),
        dk.as<uint64_t>(), dc.as<double2>());
    check_cuda(cudaMemcpyAsync(du.p, sg.coff.as<uint64_t>() + sg.nch, 8, cudaMemcpyDeviceToDevice, st),
               "sample count copy");
    check_cuda(cudaGetLastError(), "sample compaction");
    // the inner pipeline's error word joins the caller's (no host sync)
    k_or_err<<<1, 32, 0, st>>>(sg.err.as<int32_t>(), outer_err);
    check_cuda(cudaGetLastError(), "k_or_err");
}

// Level 1: every record is placed in its coarse key range.  Fills rec (the
// records grouped by range), boff (nbk + 1 range offsets) and bflags (1 for a
// range holding one repeated key); subid is scratch for the per-record range
// ids.  With Reff <= C1 there is one range holding every record in order.
// Returns nbk.  Device errors of the sample sort are or-ed into err.
// bmax caps the number of coarse ranges (the counting kernel keeps two 8-byte
// codes per splitter in shared memory: at most 2 * (bmax - 1) <= 4094).
template <class Src, int MODE>
static uint32_t level1_partition(const Src& src, uint32_t R, uint32_t nb_terms, uint64_t C1, uint32_t bmax,
                                 int oversample, int count_ctas_per_sm, cudaStream_t st, uint32_t* rec,
                                 uint16_t* subid, Scratch& boff_s, Scratch& bflags_s, int32_t* err) {
    constexpr int NW = Src::NW;
    constexpr int WP = Src::WP;
    const int sms = device_sm_count();
    uint32_t sym_na = 0;
    uint64_t Reff = R;
    if constexpr (IsProd<Src>::value) {
        if (src.sym) {
            sym_na = src.na;
            Reff = (uint64_t)src.na * (src.na + 1) / 2;
        }
    }
    if (Reff <= C1) {
        StageScope ss(ST_SCATTER, st);
        boff_s = Scratch(16, st);
        bflags_s = Scratch(1, st);
        if (sym_na)
            k_iota_tri<<<(unsigned)((Reff + 255) / 256), 256, 0, st>>>(rec, (uint32_t)Reff, sym_na,
                                                                     boff_s.as<uint64_t>(), bflags_s.as<uint8_t>());
        else
            k_iota<<<(R + 255) / 256, 256, 0, st>>>(rec, R, boff_s.as<uint64_t>(), bflags_s.as<uint8_t>());
        note_launch(ST_SCATTER);
        check_cuda(cudaGetLastError(), "k_iota");
        return 1;
    }
    const uint32_t B1 = (uint32_t)std::max<uint64_t>(2, std::min<uint64_t>(bmax, (Reff + C1 - 1) / C1));
    const uint32_t S = (uint32_t)std::min<uint64_t>(Reff, (uint64_t)B1 * (uint64_t)oversample);
    Scratch samp((size_t)S * NW * 8, st);
    const uint32_t nsp = 2 * (B1 - 1);
    const uint32_t nbk = nsp + 1;
    Scratch spl((size_t)nsp * NW * 8, st), pref((size_t)S * 4, st);
    bflags_s = Scratch(nbk, st);
    {
        StageScope ss(ST_SAMPLE, st);
        k_sample<Src><<<(S + 255) / 256, 256, 0, st>>>(src, R, S, g_sample_seed, samp.as<uint64_t>());
        note_launch(ST_SAMPLE);
        check_cuda(cudaGetLastError(), "k_sample");
        Scratch dk, dc, du;
        sorted_sample<NW>(samp.as<uint64_t>(), S, st, dk, dc, du, err);
        k_select<NW><<<1, 1024, 0, st>>>(dk.as<uint64_t>(), dc.as<double2>(), du.as<uint64_t>(), S, B1,
                                         pref.as<uint32_t>(), spl.as<uint64_t>(), bflags_s.as<uint8_t>());
        note_launch(ST_SAMPLE);
        check_cuda(cudaGetLastError(), "k_select");
    }
    Scratch cnt_s((size_t)nbk * 4, st);
    check_cuda(cudaMemsetAsync(cnt_s.p, 0, (size_t)nbk * 4, st), "memset");
    {
        StageScope ssc(ST_COUNT, st);
        Scratch codes((size_t)nsp * 16, st), meta(16, st);
        k_spl_codes<NW><<<1, 1024, 0, st>>>(spl.as<uint64_t>(), nsp, codes.as<uint64_t>(), meta.as<uint32_t>());
        note_launch(ST_COUNT);
        if constexpr (IsProd<Src>::value) {
            const size_t sm = count_smem<NW>(nsp, true);
            auto kern = k_count_prod<WP, MODE>;
            smem_attr(kern, sm);
            const uint64_t tiles = (uint64_t)((src.na + kCountThreads - 1) / kCountThreads) *
                                   ((nb_terms + kCountCols - 1) / kCountCols);
            const unsigned grid = (unsigned)std::max<uint64_t>(
                1, std::min<uint64_t>(tiles, (uint64_t)sms * (uint64_t)count_ctas_per_sm));
            kern<<<grid, kCountThreads, sm, st>>>(src, nb_terms, spl.as<uint64_t>(), codes.as<uint64_t>(),
                                                 meta.as<uint32_t>(), nsp, subid, cnt_s.as<uint32_t>());
        } else {
            const size_t sm = count_smem<NW>(nsp, false);
            auto kern = k_count_lin<Src>;
            smem_attr(kern, sm);
            const unsigned grid = (unsigned)std::max<uint64_t>(
                1, std::min<uint64_t>(((uint64_t)R + kCountThreads - 1) / kCountThreads,
                                      (uint64_t)sms * (uint64_t)count_ctas_per_sm));
            kern<<<grid, kCountThreads, sm, st>>>(src, R, spl.as<uint64_t>(), codes.as<uint64_t>(),
                                                 meta.as<uint32_t>(), nsp, subid, cnt_s.as<uint32_t>());
        }
        note_launch(ST_COUNT);
        check_cuda(cudaGetLastError(), "k_count");
    }
    StageScope ssx(ST_SCATTER, st);
    boff_s = Scratch((size_t)(nbk + 1) * 8, st);
    k_scan_counts<<<1, 1024, 0, st>>>(cnt_s.as<uint32_t>(), nbk, boff_s.as<uint64_t>());
    note_launch(ST_SCATTER);
    Scratch cursor((size_t)nbk * 8, st);
    check_cuda(cudaMemcpyAsync(cursor.p, boff_s.p, (size_t)nbk * 8, cudaMemcpyDeviceToDevice, st), "cursor");
    const size_t sm = (size_t)((nbk + 1) & ~1u) * 4 + (size_t)((nbk + 2) & ~1u) * 4 + (size_t)nbk * 8 +
                      (size_t)kScatterChunk * 6;
    smem_attr(k_scatter, sm);
    const uint64_t per_sm = std::max<uint64_t>(1, (220u * 1024u) / (sm + 1024u));
    const unsigned grid = (unsigned)std::max<uint64_t>(
        1, std::min<uint64_t>(((uint64_t)R + kScatterChunk - 1) / kScatterChunk, (uint64_t)sms * per_sm));
    k_scatter<<<grid, kScatterThreads, sm, st>>>(subid, R, nbk, cursor.as<uint64_t>(), rec, sym_na);
    note_launch(ST_SCATTER);
    check_cuda(cudaGetLastError(), "k_scatter");
    return nbk;
}

template <class Src, int MODE>
static void run_pipeline(const Src& src, uint32_t R, uint32_t nb_terms, cudaStream_t st, Staged& out) {
    constexpr int NW = Src::NW;
    using Cfg = L2Cfg<Src, MODE>;
    constexpr uint32_t CAP = Cfg::CAP;
    const int sms = device_sm_count();

    out.err = Scratch(4, st);
    check_cuda(cudaMemsetAsync(out.err.p, 0, 4, st), "memset err");
    // R indexes the record space; Reff records exist (fewer for a symmetric product)
    uint64_t Reff = R;
    if constexpr (IsProd<Src>::value) {
        if (src.sym) Reff = (uint64_t)src.na * (src.na + 1) / 2;
    }
    Scratch recA((size_t)Reff * 4, st), recB((size_t)Reff * 4, st), subid((size_t)R * 2, st);
    Scratch bflags_s, boff_s;
    const Tuning tune = tuning_for(NW);
    const uint64_t C1 = (uint64_t)CAP * (uint64_t)tune.coarse_factor;
    const uint32_t nbk = level1_partition<Src, MODE>(src, R, nb_terms, C1,
                                                     (uint32_t)(max_coarse_splitters<NW>() / 2 + 1), tune.oversample,
                                                     tune.count_ctas_per_sm, st, recA.as<uint32_t>(),
                                                     subid.as<uint16_t>(), boff_s, bflags_s, out.err.as<int32_t>());

    // level 2 and the leaves
    constexpr uint32_t WL = warp_leaf_cap<NW>();
    out.Tkeys = Scratch((size_t)Reff * NW * 8, st);
    out.Tcoef = Scratch((size_t)Reff * 16, st);
    out.nch = (uint32_t)((Reff + kChunk - 1) / kChunk);
    out.oflag = Scratch((size_t)out.nch * kChunk, st);
    out.coff = Scratch((size_t)(out.nch + 1) * 8, st);
    Scratch ctr(16, st), ccount((size_t)out.nch * 4, st);
    check_cuda(cudaMemsetAsync(out.oflag.p, 0, (size_t)out.nch * kChunk, st), "memset flags");
    check_cuda(cudaMemsetAsync(ctr.p, 0, 16, st), "memset counters");
    // every listed leaf holds at least two records (block leaves more than WL)
    const uint32_t small_cap = (uint32_t)(Reff / 2 + 1), med_cap = (uint32_t)(Reff / (WL + 1) + 1);
    Scratch lists(((size_t)small_cap + med_cap) * 8, st);
    const unsigned grid2 =
        (unsigned)std::max<uint32_t>(1, std::min<uint32_t>(nbk, (uint32_t)sms * (uint32_t)tune.range_ctas_per_sm));
    Scratch stacks((size_t)grid2 * kStackCap * sizeof(StackEnt), st);
    Scratch splscr((size_t)grid2 * (CAP / 2) * NW * 8, st);
    L2Bufs b{recA.as<uint32_t>(), recB.as<uint32_t>(), subid.as<uint16_t>(), ctr.as<uint32_t>(),
             stacks.as<StackEnt>(), splscr.as<uint64_t>(), out.Tkeys.as<uint64_t>(), out.Tcoef.as<double2>(),
             out.oflag.as<uint8_t>(), lists.as<uint2>(), lists.as<uint2>() + small_cap, small_cap, med_cap,
             out.err.as<int32_t>()};
    apply_debug(b);
    launch_level2<Src, MODE>(src, nbk, boff_s.as<uint64_t>(), bflags_s.as<uint8_t>(), b, grid2, out.nch,
                             ccount.as<uint32_t>(), out.coff.as<uint64_t>(), st);
}

// Runs the pipeline and builds the output sum (one host synchronisation).
template <class Src, int MODE>
static paulib_sum* finish(const Src& src, uint32_t R, uint32_t nb_terms, int32_t n_qubits, cudaStream_t st) {
    constexpr int WP = Src::WP;
    Staged sg;
    run_pipeline<Src, MODE>(src, R, nb_terms, st, sg);
    struct { uint64_t u; int32_t e; } h{};
    check_cuda(cudaMemcpyAsync(&h.u, sg.coff.as<uint64_t>() + sg.nch, 8, cudaMemcpyDeviceToHost, st), "U copy");
    check_cuda(cudaMemcpyAsync(&h.e, sg.err.p, 4, cudaMemcpyDeviceToHost, st), "err copy");
    check_cuda(cudaStreamSynchronize(st), "canonical sync");
    if (h.e) fail(PAULIB_ERR_INTERNAL, "canonicalisation failed on device (error word " + std::to_string(h.e) + ")");
    paulib_sum* out = sum_alloc(n_qubits, (int64_t)h.u, false, st);
    out->is_canonical = 1;
    if (h.u > 0) {
        StageScope ss(ST_COMPACT, st);
        note_launch(ST_COMPACT);
        const unsigned grid = std::max<uint32_t>(1, std::min<uint32_t>(sg.nch, (uint32_t)device_sm_count() * 8));
        k_compact<WP><<<grid, kChunkThreads, 0, st>>>(sg.nch, sg.oflag.as<uint8_t>(), sg.coff.as<uint64_t>(),
                                                     sg.Tkeys.as<uint64_t>(), sg.Tcoef.as<double2>(), out->keys,
                                                     out->coef, out->pbase);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            sum_free(out, st);
            check_cuda(e, "k_compact");
        }
    }
    return out;
}

static paulib_sum* empty_canonical(int32_t n_qubits, cudaStream_t st) {
    paulib_sum* out = sum_alloc(n_qubits, 0, false, st);
    out->is_canonical = 1;
    return out;
}

}  // namespace paulib
