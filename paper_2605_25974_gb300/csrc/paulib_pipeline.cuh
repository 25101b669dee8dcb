// paulib_pipeline.cuh -- canonical form of a Pauli-sum product (PauLIB Sec. III-G
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
//             equal-key runs are summed (Sec. III-G's merge).  A range whose
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
enum : int32_t { ERR_NONE = 0, ERR_STACK = 1, ERR_PROGRESS = 2, ERR_ITER = 4 };

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
// differ by 2*[a,b] (the symplectic inner product, Sec. III-D), so the pair
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
    __device__ __forceinline__ void split(uint32_t r, uint32_t& i, uint32_t& j) const {
        j = r / na;
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

// Shared memory per leaf record: the product key (8*NW bytes), a sort code
// (8 bytes), the record number (4 bytes, the tie-break that makes the order
// of equal keys and so the summation order deterministic), two 16-bit slot
// arrays for the merge sort and the product's phase exponent (1 byte).
constexpr int kLeafRecBytes = 8 + 4 + 2 + 2 + 1;
template <int NW>
constexpr int leaf_cap() {
    int cap = 4096;
    while (cap > 64 && cap * (8 * NW + kLeafRecBytes) > kSmemBudget) cap >>= 1;
    return cap;
}
template <int NW>
constexpr size_t leaf_smem() {
    return (size_t)leaf_cap<NW>() * (8 * NW + kLeafRecBytes);
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

constexpr int kCountThreads = 256;
constexpr int kCountCols = 64;

// Products: a tile is kCountThreads left terms x kCountCols right terms.
template <int WP, int MODE>
__global__ void __launch_bounds__(kCountThreads) k_count_prod(ProdSrc<WP, MODE> src, uint32_t nb_terms,
                                                               const uint64_t* __restrict__ spl,
                                                               uint32_t nsp, uint16_t* ids,
                                                               uint32_t* counts) {
    constexpr int NW = 2 * WP;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_spl = reinterpret_cast<uint64_t*>(smem);
    uint64_t* s_b = s_spl + (size_t)nsp * NW;
    uint32_t* s_hist = reinterpret_cast<uint32_t*>(s_b + kCountCols * NW);
    const uint32_t nbk = nsp + 1;
    for (uint32_t q = threadIdx.x; q < nsp * NW; q += blockDim.x) s_spl[(q % NW) * nsp + q / NW] = spl[q];
    for (uint32_t q = threadIdx.x; q < nbk; q += blockDim.x) s_hist[q] = 0;
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
                const uint32_t bkt = upper_bound_skeys<NW>(s_spl, nsp, nsp, k);
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
                                                              uint32_t nsp, uint16_t* ids,
                                                              uint32_t* counts) {
    constexpr int NW = Src::NW;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_spl = reinterpret_cast<uint64_t*>(smem);
    uint32_t* s_hist = reinterpret_cast<uint32_t*>(s_spl + (size_t)nsp * NW);
    const uint32_t nbk = nsp + 1;
    for (uint32_t q = threadIdx.x; q < nsp * NW; q += blockDim.x) s_spl[(q % NW) * nsp + q / NW] = spl[q];
    for (uint32_t q = threadIdx.x; q < nbk; q += blockDim.x) s_hist[q] = 0;
    __syncthreads();
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        uint64_t k[NW];
        src.key(r, k);
        const uint32_t bkt = upper_bound_skeys<NW>(s_spl, nsp, nsp, k);
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
constexpr uint32_t kScatterChunk = 32768;

static __global__ void __launch_bounds__(kScatterThreads) k_scatter(const uint16_t* __restrict__ ids, uint32_t R,
                                                             uint32_t nbk, uint64_t* cursor,
                                                             uint32_t* rec, uint32_t sym_na) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem);
    uint64_t* s_base = reinterpret_cast<uint64_t*>(s_cnt + ((nbk + 1) & ~1u));
    for (uint64_t c0 = (uint64_t)blockIdx.x * kScatterChunk; c0 < R; c0 += (uint64_t)gridDim.x * kScatterChunk) {
        const uint32_t c1 = (uint32_t)mn<uint64_t>(R, c0 + kScatterChunk);
        __syncthreads();
        for (uint32_t q = threadIdx.x; q < nbk; q += blockDim.x) s_cnt[q] = 0;
        __syncthreads();
        for (uint32_t r = (uint32_t)c0 + threadIdx.x; r < c1; r += blockDim.x) {
            if (sym_na && r % sym_na > r / sym_na) continue;  // no record for i > j
            atomicAdd(&s_cnt[ids[r]], 1u);
        }
        __syncthreads();
        for (uint32_t q = threadIdx.x; q < nbk; q += blockDim.x) {
            const uint32_t c = s_cnt[q];
            s_base[q] = c ? atomicAdd(reinterpret_cast<unsigned long long*>(cursor + q), (unsigned long long)c) : 0ull;
            s_cnt[q] = 0;
        }
        __syncthreads();
        for (uint32_t r = (uint32_t)c0 + threadIdx.x; r < c1; r += blockDim.x) {
            if (sym_na && r % sym_na > r / sym_na) continue;
            const uint32_t b = ids[r];
            const uint32_t p = atomicAdd(&s_cnt[b], 1u);
            rec[s_base[b] + p] = r;
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
};

// ---- leaf ordering
//
// A leaf (or a split sample) is ordered through one 64-bit code per slot:
// the key bits that follow the common prefix L of every key in the range.
// Equal codes fall back to the full keys and then to the record number, so
// the order is total and deterministic.  Slots >= n are padding that sorts
// last.

template <int NW, uint32_t CAP>
__device__ __forceinline__ bool slot_gt(uint32_t a, uint32_t b, const uint64_t* c1s, const uint64_t* keys_s,
                                        uint32_t n, const uint32_t* recs) {
    if (a >= n || b >= n) return a >= n && (b < n || a > b);
    const uint64_t ca = c1s[a], cb = c1s[b];
    if (ca != cb) return ca > cb;
    const int c = skey_cmp<NW>(keys_s, CAP, a, b);
    if (c) return c > 0;
    if (recs) return recs[a] > recs[b];
    return a > b;
}

template <int NW, uint32_t CAP>
__device__ __forceinline__ bool slot_key_neq(uint32_t a, uint32_t b, const uint64_t* c1s, const uint64_t* keys_s) {
    if (c1s[a] != c1s[b]) return true;
    return skey_cmp<NW>(keys_s, CAP, a, b) != 0;
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

// Codes c1s[0..n): the first bit L where any key differs from key 0 comes
// from an OR reduction of (key ^ key 0) over the range.
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
        uint32_t L = 64u * NW;
        for (int w = 0; w < NW; ++w)
            if (s_or[w]) { L = 64u * w + (uint32_t)__clzll((long long)s_or[w]); break; }
        *s_L = L;
    }
    __syncthreads();
    const uint32_t L = *s_L;
    for (uint32_t t = threadIdx.x; t < n; t += T) c1s[t] = key_bits64<NW, CAP>(keys_s, t, L);
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
                                      uint32_t n, uint32_t size, const uint32_t* recs) {
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
                while (q > 0 && slot_gt<NW, CAP>(v[q - 1], x, c1s, keys_s, n, recs)) {
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
                if (slot_gt<NW, CAP>(A[mid], B[d - mid - 1], c1s, keys_s, n, recs)) hi = mid;
                else lo = mid + 1;
            }
            uint32_t i = lo, j = d - lo;
            for (uint32_t k = 0; k < em; ++k) {
                bool takeA;
                if (i >= s) takeA = false;
                else if (j >= s) takeA = true;
                else takeA = !slot_gt<NW, CAP>(A[i], B[j], c1s, keys_s, n, recs);
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

template <class Src, int MODE>
__global__ void __launch_bounds__(kL2Threads) k_level2(
    Src src, uint32_t nbk, const uint64_t* __restrict__ boff, const uint8_t* __restrict__ bflags,
    uint32_t* recA, uint32_t* recB, uint16_t* subid, uint32_t* ticket, StackEnt* stacks,
    uint64_t* spl_scratch, uint64_t* Tkeys, double2* Tcoef, uint64_t* ucount, int32_t* err) {
    using Cfg = L2Cfg<Src, MODE>;
    using V = typename Cfg::V;
    constexpr int NW = Cfg::NW;
    constexpr uint32_t CAP = Cfg::CAP;
    constexpr int T = kL2Threads;
    constexpr uint32_t ACT = CAP < (uint32_t)T ? CAP : (uint32_t)T;
    constexpr uint32_t PP = CAP / ACT;  // sorted positions per active thread in the merge
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* keys_s = reinterpret_cast<uint64_t*>(smem);                     // [NW][CAP]
    uint64_t* c1s = keys_s + (size_t)CAP * NW;                                // [CAP]
    uint32_t* rec_s = reinterpret_cast<uint32_t*>(c1s + CAP);                 // [CAP]
    uint16_t* ord_s = reinterpret_cast<uint16_t*>(rec_s + CAP);               // [CAP]
    uint16_t* tmp_s = ord_s + CAP;                                            // [CAP]
    uint8_t* ph_s = reinterpret_cast<uint8_t*>(tmp_s + CAP);                  // [CAP]
    __shared__ uint32_t s_warp[32];
    __shared__ Acc<MODE> s_acc[32];
    __shared__ uint32_t s_flag[32];
    __shared__ unsigned long long s_or[NW];
    __shared__ uint32_t s_bucket, s_lo, s_hi, s_fl, s_sp, s_done, s_nsp, s_bad, s_L;
    __shared__ uint64_t s_u, s_tbase;

    StackEnt* stack = stacks + (size_t)blockIdx.x * kStackCap;
    uint64_t* my_spl = spl_scratch + (size_t)blockIdx.x * (CAP / 2) * NW;
    const int tid = threadIdx.x;
    const bool act = (uint32_t)tid < ACT;

    for (;;) {
        if (tid == 0) s_bucket = atomicAdd(ticket, 1u);
        __syncthreads();
        const uint32_t c = s_bucket;
        if (c >= nbk) break;
        const uint64_t base0 = boff[c];
        const uint64_t end0 = boff[c + 1];
        if (tid == 0) {
            s_u = 0;
            s_tbase = base0;
            s_bad = 0;
            s_sp = 0;
            if (end0 > base0) {
                stack[0] = StackEnt{(uint32_t)base0, (uint32_t)end0, bflags[c] ? SF_UNIFORM : 0u, 0u};
                s_sp = 1;
            }
        }
        __syncthreads();
        uint32_t iters = 0;
        for (;;) {
            if (tid == 0) {
                if (s_sp == 0 || s_bad) {
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
                if (tid == 0) { atomicOr(err, ERR_ITER); s_bad = 1; }
                __syncthreads();
                break;
            }
            const uint32_t lo = s_lo, hi = s_hi, fl = s_fl;
            const uint32_t n = hi - lo;
            const uint64_t tout = s_tbase + s_u;
            uint32_t* cur = (fl & SF_INB) ? recB : recA;
            uint32_t* oth = (fl & SF_INB) ? recA : recB;

            if (fl & SF_UNIFORM) {
                // ---- every record in the range has the same key
                Acc<MODE> acc;
                for (uint32_t t = tid; t < n; t += T) {
                    uint64_t k[NW];
                    acc.add(src.value(cur[lo + t], k));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc.shfl_merge(o);
                if ((tid & 31) == 0) s_acc[tid >> 5] = acc;
                __syncthreads();
                if (tid < 32) {
                    Acc<MODE> a2;
                    if (tid < T / 32) a2 = s_acc[tid];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) a2.shfl_merge(o);
                    if (tid == 0) {
                        uint64_t k[NW];
                        src.key(cur[lo], k);
                        key_store<NW>(Tkeys, tout, k);
                        Tcoef[tout] = a2.result();
                        s_u += 1;
                    }
                }
                __syncthreads();
            } else if (n <= CAP) {
                // ---- leaf: keys and phases into shared memory, sort, then sum
                // each run of equal keys with a block segmented scan
                for (uint32_t t = tid; t < n; t += T) {
                    uint64_t k[NW];
                    const uint32_t r = cur[lo + t];
                    rec_s[t] = r;
                    ph_s[t] = (uint8_t)src.keyphase(r, k);
                    skey_store<NW>(keys_s, CAP, t, k);
                }
                uint32_t size = 2u * (uint32_t)T >= 64u ? 64u : 2u * (uint32_t)T;
                while (size < n) size <<= 1;
                __syncthreads();
                build_codes<NW, T, CAP>(c1s, keys_s, n, s_or, &s_L);
                const uint16_t* srt = merge_sort_slots<NW, T, CAP>(ord_s, tmp_s, c1s, keys_s, n, size, rec_s);
                // positions [p0, p0 + PP) of this thread, in sorted order
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
                        hd[q] = (p == 0) || slot_key_neq<NW, CAP>(sl[q], srt[p - 1], c1s, keys_s);
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
                const uint32_t hex = block_excl_scan<T>(nh, s_warp, total);
                Acc<MODE> run = block_seg_carry<T, MODE>(nh > 0, trail, s_acc, s_flag);
                uint64_t oidx = (uint64_t)hex - 1;  // index of the run flowing in (if any)
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
                            else last = slot_key_neq<NW, CAP>(srt[p + 1], sl[q], c1s, keys_s);
                        }
                        if (last) {
                            uint64_t k[NW];
                            skey_load<NW>(keys_s, CAP, sl[q], k);
                            key_store<NW>(Tkeys, tout + oidx, k);
                            Tcoef[tout + oidx] = run.result();
                        }
                    }
                }
                __syncthreads();
                if (tid == 0) s_u += total;
                __syncthreads();
            } else {
                // ---- split: splitters from a sorted sample of this range
                const uint32_t want = (uint32_t)mn<uint64_t>(CAP / 4, ((uint64_t)n + CAP / 2 - 1) / (CAP / 2));
                uint32_t S = 64;
                while (S < 16u * want && S < CAP) S <<= 1;
                for (uint32_t t = tid; t < S; t += T) {
                    const uint32_t pos = lo + (uint32_t)(((uint64_t)t * n) / S);
                    uint64_t k[NW];
                    src.key(cur[pos], k);
                    skey_store<NW>(keys_s, CAP, t, k);
                }
                __syncthreads();
                build_codes<NW, T, CAP>(c1s, keys_s, S, s_or, &s_L);
                const uint16_t* srt = merge_sort_slots<NW, T, CAP>(ord_s, tmp_s, c1s, keys_s, S, S, nullptr);
                uint8_t* fl_s = ph_s;  // flag of range b+1 follows splitter b
                if (tid == 0) {
                    uint32_t nsp = 0;
                    fl_s[0] = 0;
                    bool stop = false;
                    // a key fills a uniform range when it covers half a target range of the sample
                    const uint32_t heavy_min = mn<uint32_t>(S, S / (2u * want) > 2u ? S / (2u * want) : 2u);
                    for (uint32_t t = 1; t < want && !stop; ++t) {
                        const uint32_t rho = (uint32_t)(((uint64_t)t * S) / want);
                        const uint32_t ci = srt[rho];
                        uint64_t k[NW], s2[NW];
                        skey_load<NW>(keys_s, CAP, ci, k);
                        if (nsp > 0 && key_cmp_m<NW>(k, my_spl + (size_t)(nsp - 1) * NW) <= 0) continue;
                        uint32_t r0 = rho, r1 = rho;
                        while (r0 > 0 && !slot_key_neq<NW, CAP>(srt[r0 - 1], ci, c1s, keys_s)) --r0;
                        while (r1 + 1 < S && !slot_key_neq<NW, CAP>(srt[r1 + 1], ci, c1s, keys_s)) ++r1;
                        const bool heavy = r1 - r0 + 1 >= heavy_min;
                        key_store<NW>(my_spl, nsp, k);
                        ++nsp;
                        fl_s[nsp] = heavy ? 1u : 0u;
                        if (heavy) {
                            if (key_succ<NW>(k, s2)) {
                                key_store<NW>(my_spl, nsp, s2);
                                ++nsp;
                                fl_s[nsp] = 0;
                            } else {
                                stop = true;  // nothing sorts after the largest key
                            }
                        }
                    }
                    s_nsp = nsp;
                }
                __syncthreads();
                const uint32_t nsp = s_nsp;
                const uint32_t nbs = nsp + 1;
                for (uint32_t q = tid; q < nsp * NW; q += T) keys_s[(q % NW) * (CAP / 2) + q / NW] = my_spl[q];
                uint32_t* cnt = reinterpret_cast<uint32_t*>(c1s);  // [nbs]
                uint32_t* cpos = cnt + CAP / 2;                      // [nbs]
                for (uint32_t q = tid; q < nbs; q += T) { cnt[q] = 0; cpos[q] = 0; }
                __syncthreads();
                for (uint32_t idx = lo + tid; idx < hi; idx += T) {
                    uint64_t k[NW];
                    src.key(cur[idx], k);
                    const uint32_t b = upper_bound_skeys<NW>(keys_s, CAP / 2, nsp, k);
                    subid[idx] = (uint16_t)b;
                    atomicAdd(&cnt[b], 1u);
                }
                __syncthreads();
                if (tid == 0) {
                    uint32_t runc = 0;
                    uint32_t bad = 0;
                    for (uint32_t b = 0; b < nbs; ++b) {
                        const uint32_t cb = cnt[b];
                        if (cb == n && !(fl_s[b] & 1u)) bad = 1;  // no progress
                        cnt[b] = runc;
                        runc += cb;
                    }
                    if (bad) { atomicOr(err, ERR_PROGRESS); s_bad = 1; }
                    else if (s_sp + nbs > (uint32_t)kStackCap) { atomicOr(err, ERR_STACK); s_bad = 1; }
                }
                __syncthreads();
                if (!s_bad) {
                    for (uint32_t idx = lo + tid; idx < hi; idx += T) {
                        const uint32_t b = subid[idx];
                        const uint32_t p = atomicAdd(&cpos[b], 1u);
                        oth[lo + cnt[b] + p] = cur[idx];
                    }
                    __syncthreads();
                    if (tid == 0) {
                        const uint32_t inb = (fl & SF_INB) ? 0u : SF_INB;  // children live in the other buffer
                        for (int b = (int)nbs - 1; b >= 0; --b) {
                            const uint32_t s0 = cnt[b];
                            const uint32_t s1 = (b + 1 < (int)nbs) ? cnt[b + 1] : n;
                            if (s1 > s0)
                                stack[s_sp++] = StackEnt{lo + s0, lo + s1, ((fl_s[b] & 1u) ? SF_UNIFORM : 0u) | inb, 0u};
                        }
                    }
                }
                __syncthreads();
            }
        }
        if (tid == 0) ucount[c] = s_u;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- compaction

template <int WP>
__global__ void __launch_bounds__(256) k_compact(uint32_t nbk, const uint64_t* __restrict__ boff,
                                                 const uint64_t* __restrict__ uoff,
                                                 const uint64_t* __restrict__ Tkeys,
                                                 const double2* __restrict__ Tcoef, uint64_t* okeys,
                                                 double2* ocoef, uint8_t* opb) {
    constexpr int NW = 2 * WP;
    for (uint32_t c = blockIdx.x; c < nbk; c += gridDim.x) {
        const uint64_t src0 = boff[c];
        const uint64_t dst0 = uoff[c];
        const uint64_t cnt = uoff[c + 1] - dst0;
        for (uint64_t t = threadIdx.x; t < cnt; t += blockDim.x) {
            uint64_t k[NW];
            key_load_g<NW>(Tkeys, src0 + t, k);
            key_store<NW>(okeys, dst0 + t, k);
            ocoef[dst0 + t] = Tcoef[src0 + t];
            opb[dst0 + t] = (uint8_t)normal_phase<WP>(k, 0u);
        }
    }
}

// Copies compacted (key, coefficient) pairs into dense scratch arrays (used
// for the merged sample inside splitter selection).
template <int NW>
__global__ void k_compact_plain(uint32_t nbk, const uint64_t* __restrict__ boff,
                                const uint64_t* __restrict__ uoff, const uint64_t* __restrict__ Tkeys,
                                const double2* __restrict__ Tcoef, uint64_t* okeys, double2* ocoef) {
    for (uint32_t c = blockIdx.x; c < nbk; c += gridDim.x) {
        const uint64_t src0 = boff[c];
        const uint64_t dst0 = uoff[c];
        const uint64_t cnt = uoff[c + 1] - dst0;
        for (uint64_t t = threadIdx.x; t < cnt; t += blockDim.x) {
            uint64_t k[NW];
            key_load_g<NW>(Tkeys, src0 + t, k);
            key_store<NW>(okeys, dst0 + t, k);
            ocoef[dst0 + t] = Tcoef[src0 + t];
        }
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
    // merged terms of every coarse range, dense within [boff[c], boff[c] + U_c)
    Scratch Tkeys, Tcoef, boff, uoff, err;
    uint32_t nbk = 0;
};

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
    k_compact_plain<NW><<<std::min<uint32_t>(sg.nbk, 1024), 256, 0, st>>>(
        sg.nbk, sg.boff.as<uint64_t>(), sg.uoff.as<uint64_t>(), sg.Tkeys.as<uint64_t>(),
        sg.Tcoef.as<double2>(), dk.as<uint64_t>(), dc.as<double2>());
    check_cuda(cudaMemcpyAsync(du.p, sg.uoff.as<uint64_t>() + sg.nbk, 8, cudaMemcpyDeviceToDevice, st),
               "sample count copy");
    check_cuda(cudaGetLastError(), "sample compaction");
    // the inner pipeline's error word joins the caller's (no host sync)
    k_or_err<<<1, 32, 0, st>>>(sg.err.as<int32_t>(), outer_err);
    check_cuda(cudaGetLastError(), "k_or_err");
}

template <class Src, int MODE>
static void run_pipeline(const Src& src, uint32_t R, uint32_t nb_terms, cudaStream_t st, Staged& out) {
    constexpr int NW = Src::NW;
    constexpr int WP = Src::WP;
    using Cfg = L2Cfg<Src, MODE>;
    constexpr uint32_t CAP = Cfg::CAP;
    const int sms = device_sm_count();

    out.err = Scratch(4, st);
    check_cuda(cudaMemsetAsync(out.err.p, 0, 4, st), "memset err");
    // R indexes the record space; Reff records exist (fewer for a symmetric product)
    uint32_t sym_na = 0;
    uint64_t Reff = R;
    if constexpr (IsProd<Src>::value) {
        if (src.sym) {
            sym_na = src.na;
            Reff = (uint64_t)src.na * (src.na + 1) / 2;
        }
    }
    Scratch recA((size_t)Reff * 4, st), recB((size_t)Reff * 4, st), subid((size_t)R * 2, st);
    Scratch bflags_s, cnt_s;
    uint32_t nbk = 1;
    const Tuning tune = tuning_for(NW);
    const uint64_t C1 = (uint64_t)CAP * (uint64_t)tune.coarse_factor;

    if (Reff <= C1) {
        StageScope ss(ST_SCATTER, st);
        out.boff = Scratch(16, st);
        bflags_s = Scratch(1, st);
        if (sym_na)
            k_iota_tri<<<(unsigned)((Reff + 255) / 256), 256, 0, st>>>(recA.as<uint32_t>(), (uint32_t)Reff, sym_na,
                                                                     out.boff.as<uint64_t>(), bflags_s.as<uint8_t>());
        else
            k_iota<<<(R + 255) / 256, 256, 0, st>>>(recA.as<uint32_t>(), R, out.boff.as<uint64_t>(),
                                                    bflags_s.as<uint8_t>());
        note_launch(ST_SCATTER);
        check_cuda(cudaGetLastError(), "k_iota");
    } else {
        const uint32_t bmax = (uint32_t)(max_coarse_splitters<NW>() / 2 + 1);
        const uint32_t B1 = (uint32_t)std::max<uint64_t>(2, std::min<uint64_t>(bmax, (Reff + C1 - 1) / C1));
        const uint32_t S = (uint32_t)std::min<uint64_t>(Reff, (uint64_t)B1 * (uint64_t)tune.oversample);
        Scratch samp((size_t)S * NW * 8, st);
        const uint32_t nsp = 2 * (B1 - 1);
        nbk = nsp + 1;
        Scratch spl((size_t)nsp * NW * 8, st), pref((size_t)S * 4, st);
        bflags_s = Scratch(nbk, st);
        {
            StageScope ss(ST_SAMPLE, st);
            k_sample<Src><<<(S + 255) / 256, 256, 0, st>>>(src, R, S, g_sample_seed, samp.as<uint64_t>());
            note_launch(ST_SAMPLE);
            check_cuda(cudaGetLastError(), "k_sample");
            Scratch dk, dc, du;
            sorted_sample<NW>(samp.as<uint64_t>(), S, st, dk, dc, du, out.err.as<int32_t>());
            k_select<NW><<<1, 1024, 0, st>>>(dk.as<uint64_t>(), dc.as<double2>(), du.as<uint64_t>(), S, B1,
                                             pref.as<uint32_t>(), spl.as<uint64_t>(), bflags_s.as<uint8_t>());
            note_launch(ST_SAMPLE);
            check_cuda(cudaGetLastError(), "k_select");
        }
        cnt_s = Scratch((size_t)nbk * 4, st);
        check_cuda(cudaMemsetAsync(cnt_s.p, 0, (size_t)nbk * 4, st), "memset");
        {
        StageScope ssc(ST_COUNT, st);
        if constexpr (IsProd<Src>::value) {
            const size_t sm = (size_t)nsp * NW * 8 + (size_t)kCountCols * NW * 8 + (size_t)nbk * 4;
            auto kern = k_count_prod<WP, MODE>;
            smem_attr(kern, sm);
            const uint64_t tiles = (uint64_t)((src.na + kCountThreads - 1) / kCountThreads) *
                                   ((nb_terms + kCountCols - 1) / kCountCols);
            const unsigned grid = (unsigned)std::max<uint64_t>(
                1, std::min<uint64_t>(tiles, (uint64_t)sms * (uint64_t)tune.count_ctas_per_sm));
            kern<<<grid, kCountThreads, sm, st>>>(src, nb_terms, spl.as<uint64_t>(), nsp, subid.as<uint16_t>(),
                                                 cnt_s.as<uint32_t>());
        } else {
            const size_t sm = (size_t)nsp * NW * 8 + (size_t)nbk * 4;
            auto kern = k_count_lin<Src>;
            smem_attr(kern, sm);
            const unsigned grid = (unsigned)std::max<uint64_t>(
                1, std::min<uint64_t>(((uint64_t)R + kCountThreads - 1) / kCountThreads,
                                      (uint64_t)sms * (uint64_t)tune.count_ctas_per_sm));
            kern<<<grid, kCountThreads, sm, st>>>(src, R, spl.as<uint64_t>(), nsp, subid.as<uint16_t>(),
                                                 cnt_s.as<uint32_t>());
        }
        note_launch(ST_COUNT);
        check_cuda(cudaGetLastError(), "k_count");
        }
        StageScope ssx(ST_SCATTER, st);
        out.boff = Scratch((size_t)(nbk + 1) * 8, st);
        k_scan_counts<<<1, 1024, 0, st>>>(cnt_s.as<uint32_t>(), nbk, out.boff.as<uint64_t>());
        note_launch(ST_SCATTER);
        Scratch cursor((size_t)nbk * 8, st);
        check_cuda(cudaMemcpyAsync(cursor.p, out.boff.p, (size_t)nbk * 8, cudaMemcpyDeviceToDevice, st), "cursor");
        const size_t sm = (size_t)((nbk + 1) & ~1u) * 4 + (size_t)nbk * 8;
        smem_attr(k_scatter, sm);
        const unsigned grid = (unsigned)std::max<uint64_t>(
            1, std::min<uint64_t>(((uint64_t)R + kScatterChunk - 1) / kScatterChunk, (uint64_t)sms * 2));
        k_scatter<<<grid, kScatterThreads, sm, st>>>(subid.as<uint16_t>(), R, nbk, cursor.as<uint64_t>(),
                                                    recA.as<uint32_t>(), sym_na);
        note_launch(ST_SCATTER);
        check_cuda(cudaGetLastError(), "k_scatter");
    }

    // level 2
    out.nbk = nbk;
    out.Tkeys = Scratch((size_t)Reff * NW * 8, st);
    out.Tcoef = Scratch((size_t)Reff * 16, st);
    Scratch ucount((size_t)nbk * 8, st), ticket(4, st);
    check_cuda(cudaMemsetAsync(ticket.p, 0, 4, st), "memset");
    const unsigned grid2 =
        (unsigned)std::max<uint32_t>(1, std::min<uint32_t>(nbk, (uint32_t)sms * (uint32_t)tune.range_ctas_per_sm));
    Scratch stacks((size_t)grid2 * kStackCap * sizeof(StackEnt), st);
    Scratch splscr((size_t)grid2 * (CAP / 2) * NW * 8, st);
    auto k2 = k_level2<Src, MODE>;
    smem_attr(k2, Cfg::SMEM);
    StageScope ss2(ST_LEVEL2, st);
    note_launch(ST_LEVEL2);
    note_launch(ST_LEVEL2);  // k_level2 and the scan below
    k2<<<grid2, kL2Threads, Cfg::SMEM, st>>>(src, nbk, out.boff.as<uint64_t>(), bflags_s.as<uint8_t>(),
                                            recA.as<uint32_t>(), recB.as<uint32_t>(), subid.as<uint16_t>(),
                                            ticket.as<uint32_t>(), stacks.as<StackEnt>(), splscr.as<uint64_t>(),
                                            out.Tkeys.as<uint64_t>(), out.Tcoef.as<double2>(),
                                            ucount.as<uint64_t>(), out.err.as<int32_t>());
    check_cuda(cudaGetLastError(), "k_level2");
    out.uoff = Scratch((size_t)(nbk + 1) * 8, st);
    k_scan_u64<<<1, 1024, 0, st>>>(ucount.as<uint64_t>(), nbk, out.uoff.as<uint64_t>());
    check_cuda(cudaGetLastError(), "k_scan_u64");
}

// Runs the pipeline and builds the output sum (one host synchronisation).
template <class Src, int MODE>
static paulib_sum* finish(const Src& src, uint32_t R, uint32_t nb_terms, int32_t n_qubits, cudaStream_t st) {
    constexpr int WP = Src::WP;
    Staged sg;
    run_pipeline<Src, MODE>(src, R, nb_terms, st, sg);
    struct { uint64_t u; int32_t e; } h{};
    check_cuda(cudaMemcpyAsync(&h.u, sg.uoff.as<uint64_t>() + sg.nbk, 8, cudaMemcpyDeviceToHost, st), "U copy");
    check_cuda(cudaMemcpyAsync(&h.e, sg.err.p, 4, cudaMemcpyDeviceToHost, st), "err copy");
    check_cuda(cudaStreamSynchronize(st), "canonical sync");
    if (h.e) fail(PAULIB_ERR_INTERNAL, "canonicalisation failed on device (error word " + std::to_string(h.e) + ")");
    paulib_sum* out = sum_alloc(n_qubits, (int64_t)h.u, false, st);
    out->is_canonical = 1;
    if (h.u > 0) {
        StageScope ss(ST_COMPACT, st);
        note_launch(ST_COMPACT);
        const unsigned grid = std::max<uint32_t>(1, std::min<uint32_t>(sg.nbk, (uint32_t)device_sm_count() * 8));
        k_compact<WP><<<grid, 256, 0, st>>>(sg.nbk, sg.boff.as<uint64_t>(), sg.uoff.as<uint64_t>(),
                                           sg.Tkeys.as<uint64_t>(), sg.Tcoef.as<double2>(), out->keys, out->coef,
                                           out->pbase);
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
    Src src{a->keys, b->keys, a->pbase, b->pbase, ac, bc, (uint32_t)a->n_terms, a == b ? 1u : 0u};
    return finish<Src, MODE>(src, R, (uint32_t)b->n_terms, a->n_qubits, st);
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
    return finish<Src, MODE>(src, (uint32_t)in->n_terms, 0, in->n_qubits, st);
}

}  // namespace paulib
