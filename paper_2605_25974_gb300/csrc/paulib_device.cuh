// paulib_device.cuh -- device primitives: packed symplectic keys, the string
// product with its exact phase, complex coefficient arithmetic in the three
// precision modes, and block-level sort/scan helpers.
//
// Key layout in device memory (one term): 2*WP 64-bit words
//   [x_0 .. x_{WP-1}, z_0 .. z_{WP-1}]
// WP is the padded word count (1, 2, 4, 8, 16 >= ceil(n/64)); padding words
// are zero, which leaves the lexicographic order of the real words unchanged
// (PauLIB Sec. III-H orders terms by a lexicographic key of the packed words).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace paulib {

// ------------------------------------------------------------------ keys

template <int NW>
__device__ __forceinline__ void key_load_g(const uint64_t* __restrict__ base, uint64_t t,
                                           uint64_t (&k)[NW]) {
    static_assert(NW % 2 == 0, "keys are whole 16-byte pairs");
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(base + t * NW);
#pragma unroll
    for (int q = 0; q < NW / 2; ++q) {
        ulonglong2 v = __ldg(p + q);
        k[2 * q] = v.x;
        k[2 * q + 1] = v.y;
    }
}

template <int NW>
__device__ __forceinline__ void key_store(uint64_t* base, uint64_t t, const uint64_t (&k)[NW]) {
    ulonglong2* p = reinterpret_cast<ulonglong2*>(base + t * NW);
#pragma unroll
    for (int q = 0; q < NW / 2; ++q) p[q] = make_ulonglong2(k[2 * q], k[2 * q + 1]);
}

template <int NW>
__device__ __forceinline__ void key_load_s(const uint64_t* base, uint32_t t, uint64_t (&k)[NW]) {
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(base + (uint64_t)t * NW);
#pragma unroll
    for (int q = 0; q < NW / 2; ++q) {
        ulonglong2 v = p[q];
        k[2 * q] = v.x;
        k[2 * q + 1] = v.y;
    }
}

// Lexicographic comparison, word 0 most significant, unsigned words.
template <int NW>
__device__ __forceinline__ int key_cmp(const uint64_t (&a)[NW], const uint64_t (&b)[NW]) {
#pragma unroll
    for (int q = 0; q < NW; ++q)
        if (a[q] != b[q]) return a[q] < b[q] ? -1 : 1;
    return 0;
}

// Compare a register key with a key in memory (shared or global).
template <int NW>
__device__ __forceinline__ int key_cmp_m(const uint64_t (&a)[NW], const uint64_t* b) {
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        uint64_t v = b[q];
        if (a[q] != v) return a[q] < v ? -1 : 1;
    }
    return 0;
}

template <int NW>
__device__ __forceinline__ int key_cmp_mm(const uint64_t* a, const uint64_t* b) {
#pragma unroll 4
    for (int q = 0; q < NW; ++q) {
        uint64_t u = a[q], v = b[q];
        if (u != v) return u < v ? -1 : 1;
    }
    return 0;
}

// ------------------------------------------------------------------ string product

// P(x,z) = i^{|x&z|} X^x Z^z per qubit (Y = iXZ, Sec. III-A).  `pa`, `pb` are
// the terms' exponents in that normal form, (|x&z| + own phase) mod 4.  Then
//   (i^pa X^xa Z^za)(i^pb X^xb Z^zb) = i^{pa+pb} (-1)^{|za&xb|} X^x Z^z
//                                    = i^{pa+pb+2|za&xb|-|x&z|} P(x, z)
// with x = xa^xb, z = za^zb (Sec. III-E: XOR of the words, phase from
// popcounts).  |x&z| mod 4 is accumulated bit-sliced (a two-bit counter per
// bit position across words) so only two popcounts are needed for any WP.
template <int WP>
__device__ __forceinline__ uint32_t string_product(const uint64_t (&a)[2 * WP],
                                                   const uint64_t (&b)[2 * WP], uint32_t pa,
                                                   uint32_t pb, uint64_t (&o)[2 * WP]) {
    uint64_t ones = 0, twos = 0, fold = 0;
#pragma unroll
    for (int q = 0; q < WP; ++q) {
        const uint64_t x = a[q] ^ b[q];
        const uint64_t z = a[WP + q] ^ b[WP + q];
        o[q] = x;
        o[WP + q] = z;
        const uint64_t v = x & z;
        twos ^= ones & v;
        ones ^= v;
        fold ^= a[WP + q] & b[q];
    }
    // |x&z| mod 4 = |ones| + 2|twos| (mod 4), so
    // k = pa + pb - |ones| + 2(|za&xb| + |twos|) and the factor-2 part only
    // needs the parity of |za&xb| + |twos| = parity of |fold ^ twos|.
    const uint32_t par = (uint32_t)__popcll(fold ^ twos) & 1u;
    return (pa + pb + 2u * par - (uint32_t)__popcll(ones)) & 3u;
}

// Exponent of a single term in the X^x Z^z normal form.
template <int WP>
__device__ __forceinline__ uint32_t normal_phase(const uint64_t (&k)[2 * WP], uint32_t own) {
    uint32_t c = 0;
#pragma unroll
    for (int q = 0; q < WP; ++q) c += (uint32_t)__popcll(k[q] & k[WP + q]);
    return (c + own) & 3u;
}

// ------------------------------------------------------------------ coefficients

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Multiply by i^k exactly: a swap and sign-bit flips done with integer ops,
// so the FP64 pipe is not used and no rounding happens.
__device__ __forceinline__ double2 rot_ik(double2 c, uint32_t k) {
    const bool sw = k & 1u;
    double re = sw ? c.y : c.x;
    double im = sw ? c.x : c.y;
    const uint64_t sre = ((k + 1u) & 2u) ? 0x8000000000000000ull : 0ull;  // k = 1, 2
    const uint64_t sim = (k & 2u) ? 0x8000000000000000ull : 0ull;         // k = 2, 3
    re = __longlong_as_double(__double_as_longlong(re) ^ sre);
    im = __longlong_as_double(__double_as_longlong(im) ^ sim);
    return make_double2(re, im);
}

__device__ __forceinline__ float2 rot_ikf(float2 c, uint32_t k) {
    const bool sw = k & 1u;
    float re = sw ? c.y : c.x;
    float im = sw ? c.x : c.y;
    const uint32_t sre = ((k + 1u) & 2u) ? 0x80000000u : 0u;
    const uint32_t sim = (k & 2u) ? 0x80000000u : 0u;
    re = __uint_as_float(__float_as_uint(re) ^ sre);
    im = __uint_as_float(__float_as_uint(im) ^ sim);
    return make_float2(re, im);
}

// Knuth's TwoSum: s + e == a + b exactly (round-to-nearest, no overflow).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// ------------------------------------------------------------------ misc

template <class T>
__host__ __device__ __forceinline__ T mn(T a, T b) { return a < b ? a : b; }

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    // SplitMix64 finaliser (Steele, Lea, Flood 2014), used to spread sample
    // positions; it is not part of the Pauli arithmetic.
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

}  // namespace paulib
