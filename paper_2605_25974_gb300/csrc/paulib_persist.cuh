// paulib_persist.cuh -- batched canonical products in one persistent kernel:
// PauLIB's sort_and_combine (Sec. III-H) applied at once to many independent
// outer products (Sec. IV-C), shaped like the many small products of a
// Pauli-propagation step (Sec. III-B).
//
// CTAs take problems from a device ticket, largest first, and own a problem
// until its last merged term is written:
//   * a problem of at most persist_leaf_cap<NW>() products (a smaller
//     capacity may be set for tests) is one shared-memory leaf;
//   * a larger one is split into key ranges: splitters are order-preserving
//     64-bit codes of a sorted sample of its records (the first nonzero
//     64-bit key window after a position before which the range's keys
//     agree, and where that window lies), so children stay balanced however
//     sparse the keys; a code frequent in the sample gets a child of its
//     own, and each child learns how far its keys agree.  A split that
//     separates nothing falls back to the range's exact first varying
//     position and the kPDigitBits bits there (which always separate), and a
//     range of one key is summed.  Children live in ping-pong record buffers
//     in global memory; the CTA walks them depth first, in key order, and
//     splits a child larger than a leaf again;
//   * a leaf gathers its records' whole keys into shared memory once and
//     sorts a permutation by (64-bit window from the leaf's first varying
//     position, whole key, record number), comparing whole keys only where
//     windows tie.  Each run of one key is summed in record order and its
//     merged term is written straight into the problem's output sum.
// Splits by sample happen only in the first kPSampleDepth levels; each later
// split consumes kPDigitBits key bits, so the walk's depth is bounded and its
// per-CTA level stack cannot overflow.  No CTA ever waits for another.
#pragma once
#include "paulib_pipeline.cuh"

namespace paulib {

constexpr int kPThreads = 256;                  // threads of a persistent CTA
constexpr uint32_t kPNB = 64;                   // most terms of a right operand
constexpr uint32_t kPDigitBits = 8;             // key bits of a digit split
constexpr uint32_t kPFan = 1u << kPDigitBits;   // most children of a split
constexpr uint32_t kPSample = 1024;             // most sampled codes per sample split
constexpr uint32_t kPSampleDepth = 6;           // levels that may split by sample
constexpr int kPU = 4;                          // records per thread in flight
static_assert(kPFan == (uint32_t)kPThreads, "one child per thread");

// Leaf capacity: whole keys of 64 KB at most (1,024 records up to 8-word
// keys, 512 for 16-word keys, 256 for 32-word keys).
template <int NW>
constexpr uint32_t persist_leaf_cap() {
    return (65536u / (8u * NW)) < 1024u ? (65536u / (8u * NW)) : 1024u;
}

// Problem b: left operand A_b (na terms), right operand B_b (nb terms).
struct ProbDesc {
    const uint64_t* ak;
    const uint64_t* bk;
    const uint8_t* ap;
    const uint8_t* bp;
    const void* ac;
    const void* bc;
    uint32_t na, nb;
    uint64_t na_inv;  // recip64(na): j = r / na by one high multiply
};
static_assert(sizeof(ProbDesc) == 64, "descriptor is one 64-byte record");

struct OutDesc {
    uint64_t* keys;
    double2* coef;
    uint8_t* pbase;
    uint64_t pad;
};

// One level of the depth-first walk: the split range's first record, the
// buffer its children live in, the next child to visit, the children's
// offsets (start[d] .. start[d + 1]) and, per child, a position before which
// all of its keys agree.
struct PLevel {
    uint32_t lo, buf, next, pad;
    uint32_t start[kPFan + 1];
    uint16_t D[kPFan];
};
template <int NW>
constexpr uint32_t persist_depth() {
    return kPSampleDepth + (64u * NW) / kPDigitBits + 1u;
}

// Shared-memory layout of a persistent CTA: the right operand and the
// leaf's arrays (a split uses the key area for its sample and splitters).
template <int WP, int MODE>
struct PLayout {
    static constexpr int NW = 2 * WP;
    static constexpr uint32_t CAP = persist_leaf_cap<NW>();
    using V = typename ValT<MODE>::T;
    static constexpr size_t BK = 0;                                // u64 [kPNB][NW]  B's keys
    static constexpr size_t BC = BK + (size_t)kPNB * NW * 8;       // V   [kPNB]      B's coefficients
    static constexpr size_t BP = BC + (size_t)kPNB * sizeof(V);    // u8  [kPNB]      B's phases
    static constexpr size_t KEYS = BP + kPNB;                      // u64 [NW][CAP]   whole keys, word-major
    static constexpr size_t C1 = KEYS + (size_t)NW * CAP * 8;      // u64 [CAP]       sort windows
    static constexpr size_t VAL = C1 + (size_t)CAP * 8;            // V   [CAP]       contributions
    static constexpr size_t RR = VAL + (size_t)CAP * sizeof(V);    // u32 [CAP]       record numbers
    static constexpr size_t IDX = RR + (size_t)CAP * 4;            // u16 [CAP]       slot at each position
    static constexpr size_t SEG = IDX + (size_t)CAP * 2;           // u16 [CAP]       run rank
    static constexpr size_t HD = SEG + (size_t)CAP * 2;            // u8  [CAP]       run heads
    static constexpr size_t BYTES = HD + CAP;
    static_assert(KEYS % 16 == 0 && C1 % 16 == 0 && VAL % 16 == 0, "aligned arrays");
    static_assert((size_t)NW * CAP * 8 >= (size_t)(kPSample + kPFan) * 8, "split sample fits the key area");
};

template <int NW, int MODE>
struct PShared {
    unsigned long long mask[NW];
    unsigned long long mand[NW];
    uint32_t warp[32];
    uint32_t hist[kPFan];
    uint32_t curs[kPFan];
    Acc<MODE> acc[kPThreads / 32];
    uint32_t prob, out, depth, next, full;
};

// The current problem, as seen by every thread of the CTA.
template <int WP, int MODE>
struct PCtx {
    static constexpr int NW = 2 * WP;
    using V = typename ValT<MODE>::T;
    const uint64_t* ak;
    const uint8_t* ap;
    const V* ac;
    const uint64_t* sbk;
    const uint8_t* sbp;
    const V* sbc;
    uint32_t na;
    uint64_t na_inv;
    // record r = j * na + i stands for a_i * b_j (Sec. IV-C's raw index)
    __device__ __forceinline__ void split(uint32_t r, uint32_t& i, uint32_t& j) const {
        j = na_inv ? (uint32_t)__umul64hi((uint64_t)r, na_inv) : r;
        i = r - j * na;
    }
    __device__ __forceinline__ void key(uint32_t r, uint64_t (&k)[NW]) const {
        uint32_t i, j;
        split(r, i, j);
        uint64_t a[NW], b[NW];
        key_load_g<NW>(ak, i, a);
        key_load_s<NW>(sbk, j, b);
#pragma unroll
        for (int q = 0; q < NW; ++q) k[q] = a[q] ^ b[q];
    }
    // Product key and its contribution i^k c_a c_b (Sec. III-E).
    __device__ __forceinline__ V value(uint32_t r, uint64_t (&k)[NW]) const {
        uint32_t i, j;
        split(r, i, j);
        uint64_t a[NW], b[NW];
        key_load_g<NW>(ak, i, a);
        key_load_s<NW>(sbk, j, b);
        const uint32_t ph = string_product<WP>(a, b, __ldg(ap + i), sbp[j], k);
        return rot_v(mul_v(ac[i], sbc[j]), ph);
    }
    // Skip-zero code: an order-preserving 64-bit code of record r's key bits
    // from position P that skips zero 64-bit windows.  With v_j the window of
    // bits [P + 64j, P + 64j + 64), K windows, j1 the first nonzero one and
    // F = K - j1 (0 when every window is zero), the code is F in the top 6
    // bits and the top 58 bits of v_j1.  For keys equal before P, a larger
    // code means a larger or equal key: at the first window where two keys
    // differ either one of them is zero there (its F is smaller) or both are
    // nonzero at the same index.  Keys that are zero in many windows get codes
    // spread like their first nonzero windows.  Only the windows up to the
    // first nonzero one are read.
    __device__ __forceinline__ uint64_t skip(uint32_t r, uint32_t P) const {
        constexpr uint32_t end = 64u * NW;
        if (P >= end) return 0ull;
        const uint32_t K = (end - P + 63u) >> 6;
        for (uint32_t j = 0; j < K; ++j) {
            const uint64_t v = window(r, P + 64u * j);
            if (v) return ((uint64_t)(K - j) << 58) | (v >> 6);
        }
        return 0ull;
    }
    // Key bits [P, P + 64) of record r (zero beyond the key), from the two
    // words that hold them.
    __device__ __forceinline__ uint64_t window(uint32_t r, uint32_t P) const {
        if (P >= 64u * NW) return 0ull;
        uint32_t i, j;
        split(r, i, j);
        const uint32_t w = P >> 6, sh = P & 63u;
        const uint64_t* pa = ak + (size_t)i * NW;
        const uint64_t* pb = sbk + (size_t)j * NW;
        uint64_t v = __ldg(pa + w) ^ pb[w];
        if (sh) {
            const uint64_t nx = w + 1u < (uint32_t)NW ? (__ldg(pa + w + 1) ^ pb[w + 1]) : 0ull;
            v = (v << sh) | (nx >> (64u - sh));
        }
        return v;
    }
};

// First set position >= P of a shared mask (word 0's top bit is position
// 0), or 64 * NW when there is none; with `and_` given, of the mask
// m ^ and_ (the OR and AND of a set of keys: where some of them differ).
template <int NW>
__device__ __forceinline__ uint32_t pmask_first(const unsigned long long* m, uint32_t P = 0,
                                                const unsigned long long* and_ = nullptr) {
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        if (64u * w + 63u < P) continue;
        uint64_t v = and_ ? (m[w] ^ and_[w]) : m[w];
        if (P > 64u * w) v &= ~0ull >> (P - 64u * w);
        if (v) return 64u * w + (uint32_t)__clzll((long long)v);
    }
    return 64u * NW;
}

// OR of every thread's mo into s_or and AND of its ma into s_and (set to 0
// and all-ones by the caller before the barrier that precedes this call).
template <int NW>
__device__ __forceinline__ void pmask_reduce(const uint64_t (&mo)[NW], const uint64_t (&ma)[NW],
                                             unsigned long long* s_or, unsigned long long* s_and) {
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const uint32_t oh = __reduce_or_sync(0xffffffffu, (uint32_t)(mo[w] >> 32));
        const uint32_t ol = __reduce_or_sync(0xffffffffu, (uint32_t)mo[w]);
        const uint32_t ah = __reduce_and_sync(0xffffffffu, (uint32_t)(ma[w] >> 32));
        const uint32_t al = __reduce_and_sync(0xffffffffu, (uint32_t)ma[w]);
        if ((threadIdx.x & 31u) == 0) {
            atomicOr(s_or + w, ((unsigned long long)oh << 32) | ol);
            atomicAnd(s_and + w, ((unsigned long long)ah << 32) | al);
        }
    }
}

// The positions where some keys differ, OR ^ AND of the keys, into s_or
// (after the barrier that follows pmask_reduce; ends with a barrier).
template <int NW>
__device__ __forceinline__ void pmask_finish(unsigned long long* s_or, const unsigned long long* s_and) {
    uint64_t v = 0;
    if (threadIdx.x < (uint32_t)NW) v = s_or[threadIdx.x] ^ s_and[threadIdx.x];
    __syncthreads();
    if (threadIdx.x < (uint32_t)NW) s_or[threadIdx.x] = v;
    __syncthreads();
}

// Sum of the CTA's accumulators in a fixed order (threads, then warps).
template <int MODE>
__device__ __forceinline__ Acc<MODE> pblock_sum(Acc<MODE> a, Acc<MODE>* s_acc) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a.shfl_merge(o);
    if ((threadIdx.x & 31u) == 0) s_acc[threadIdx.x >> 5] = a;
    __syncthreads();
    Acc<MODE> t = s_acc[0];
#pragma unroll
    for (int w = 1; w < kPThreads / 32; ++w) t.merge(s_acc[w]);
    __syncthreads();
    return t;
}

// Writes merged term `pos` of the problem's output.
template <int WP>
__device__ __forceinline__ void pemit(const OutDesc& o, uint32_t pos, const uint64_t (&k)[2 * WP], double2 c) {
    key_store<2 * WP>(o.keys, pos, k);
    o.coef[pos] = c;
    o.pbase[pos] = (uint8_t)normal_phase<WP>(k, 0u);
}

// Bitonic sort of npow shared 64-bit values (a split's sample).
__device__ __forceinline__ void psort_codes(uint64_t* c, uint32_t npow) {
    for (uint32_t k = 2; k <= npow; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t q = threadIdx.x; q < npow / 2; q += kPThreads) {
                const uint32_t i = ((q & ~(j - 1u)) << 1) | (q & (j - 1u));
                const uint32_t l = i | j;
                const uint64_t a = c[i], b = c[l];
                if ((a > b) == ((i & k) == 0)) {
                    c[i] = b;
                    c[l] = a;
                }
            }
            __syncthreads();
        }
    }
}

// Exclusive scan of the head flags over positions [0, n) in blocked chunks;
// writes each position's run rank to seg and returns the number of runs.
// Ends with a barrier: callers read ranks written by other threads.
__device__ __forceinline__ uint32_t prank_heads(const uint8_t* hd, uint16_t* seg, uint32_t n, uint32_t* s_warp) {
    const uint32_t per = (n + kPThreads - 1) / kPThreads;
    const uint32_t q0 = threadIdx.x * per;
    uint32_t c = 0;
    for (uint32_t q = q0; q < q0 + per && q < n; ++q) c += hd[q];
    uint32_t tot;
    uint32_t ex = block_excl_scan<kPThreads>(c, s_warp, tot);
    for (uint32_t q = q0; q < q0 + per && q < n; ++q) {
        ex += hd[q];
        seg[q] = (uint16_t)(ex - 1u);
    }
    __syncthreads();
    return tot;
}

// Key order of the leaf entries at positions p and q (slots idx[p], idx[q];
// a slot >= n is padding and sorts last): by window, then by the whole keys
// from word w0 on (all keys of the leaf agree before it).  -1, 0 or 1.
template <int NW, uint32_t CAP>
__device__ __forceinline__ int pleaf_cmp(const uint64_t* keys, const uint64_t* c1, const uint16_t* idx,
                                         uint32_t p, uint32_t q, uint32_t n, uint32_t w0) {
    const uint32_t a = idx[p], b = idx[q];
    const bool pa = a >= n, pb = b >= n;
    if (pa | pb) return pa == pb ? 0 : (pa ? 1 : -1);
    const uint64_t ca = c1[p], cb = c1[q];
    if (ca != cb) return ca < cb ? -1 : 1;
    for (uint32_t w = w0; w < (uint32_t)NW; ++w) {
        const uint64_t ka = keys[(size_t)w * CAP + a], kb = keys[(size_t)w * CAP + b];
        if (ka != kb) return ka < kb ? -1 : 1;
    }
    return 0;
}

// A leaf sort entry: window and slot.
struct PE {
    uint64_t c;
    uint32_t s;
};

// Strict order of two leaf entries: padding (slot >= n) last, then by
// window, by whole key from word w0 on, by record number and by slot.
template <int NW, uint32_t CAP>
__device__ __forceinline__ bool pe_gt(const PE& a, const PE& b, const uint64_t* keys, const uint32_t* rr, uint32_t n,
                                      uint32_t w0) {
    const bool pa = a.s >= n, pb = b.s >= n;
    if (pa || pb) return pa && (!pb || a.s > b.s);
    if (a.c != b.c) return a.c > b.c;
    for (uint32_t w = w0; w < (uint32_t)NW; ++w) {
        const uint64_t ka = keys[(size_t)w * CAP + a.s], kb = keys[(size_t)w * CAP + b.s];
        if (ka != kb) return ka > kb;
    }
    const uint32_t ra = rr[a.s], rb = rr[b.s];
    return ra != rb ? ra > rb : a.s > b.s;
}

// Bitonic sort of the first np positions (a power of two, 32 .. 256E) held
// in registers: position g = warp * 32E + e * 32 + lane.  Partners closer
// than 32 are exchanged by shuffles, partners 32 .. 16E apart between a
// thread's own rows, the rest through shared memory (sc, si), so only the
// stages that cross warps need barriers.  Positions >= np never meet a
// position below np and stay where they are.
template <int NW, uint32_t CAP, uint32_t E>
__device__ __forceinline__ void psort_reg(PE (&x)[E], uint32_t np, uint64_t* sc, uint16_t* si, const uint64_t* keys,
                                          const uint32_t* rr, uint32_t n, uint32_t w0) {
    const uint32_t lane = threadIdx.x & 31u, wb = (threadIdx.x >> 5) * 32u * E;
    const bool active = wb < np;  // whole warps lie below np or at or above it
#pragma unroll 1
    for (uint32_t k = 2; k <= np; k <<= 1) {
#pragma unroll 1
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32u * E) {
#pragma unroll
                for (uint32_t e = 0; e < E; ++e) {
                    const uint32_t g = wb + e * 32u + lane;
                    if (g < np) {
                        sc[g] = x[e].c;
                        si[g] = (uint16_t)x[e].s;
                    }
                }
                __syncthreads();
#pragma unroll
                for (uint32_t e = 0; e < E; ++e) {
                    const uint32_t g = wb + e * 32u + lane, p = g ^ j;
                    if (g < np) {
                        const PE y{sc[p], si[p]};
                        const bool keep_min = ((g & j) == 0) == ((g & k) == 0);
                        if (keep_min == pe_gt<NW, CAP>(x[e], y, keys, rr, n, w0)) x[e] = y;
                    }
                }
                __syncthreads();
            } else if (active) {
                if (j >= 32u) {
                    const uint32_t d = j >> 5;
#pragma unroll
                    for (uint32_t e = 0; e < E; ++e) {
                        if ((e & d) == 0 && (e | d) < E) {
                            const uint32_t e2 = e | d;
                            const uint32_t g = wb + e * 32u + lane;
                            if (g < np && pe_gt<NW, CAP>(x[e], x[e2], keys, rr, n, w0) == ((g & k) == 0)) {
                                const PE t = x[e];
                                x[e] = x[e2];
                                x[e2] = t;
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (uint32_t e = 0; e < E; ++e) {
                        const uint32_t g = wb + e * 32u + lane;
                        PE y;
                        y.c = __shfl_xor_sync(0xffffffffu, x[e].c, (int)j);
                        y.s = __shfl_xor_sync(0xffffffffu, x[e].s, (int)j);
                        const bool keep_min = ((lane & j) == 0) == ((g & k) == 0);
                        if (g < np && keep_min == pe_gt<NW, CAP>(x[e], y, keys, rr, n, w0)) x[e] = y;
                    }
                }
            }
        }
    }
}

// Loads the leaf's entries (window of 64 key bits from L) into registers,
// sorts the first np positions and writes windows and slots in order.
template <int NW, uint32_t CAP, uint32_t E>
__device__ __forceinline__ void psort_leaf_rows(const uint64_t* keys, uint64_t* c1, uint16_t* idx, const uint32_t* rr,
                                                uint32_t np, uint32_t n, uint32_t L, uint32_t w0) {
    const uint32_t lane = threadIdx.x & 31u, wb = (threadIdx.x >> 5) * 32u * E;
    const uint32_t lw = L >> 6, ls = L & 63u;
    PE x[E];
#pragma unroll
    for (uint32_t e = 0; e < E; ++e) {
        const uint32_t g = wb + e * 32u + lane;
        uint64_t c = ~0ull;
        if (g < n) {
            c = keys[(size_t)lw * CAP + g];
            if (ls) {
                const uint64_t nx = lw + 1u < (uint32_t)NW ? keys[(size_t)(lw + 1u) * CAP + g] : 0ull;
                c = (c << ls) | (nx >> (64u - ls));
            }
        }
        x[e] = PE{c, g};
    }
    psort_reg<NW, CAP, E>(x, np, c1, idx, keys, rr, n, w0);
#pragma unroll
    for (uint32_t e = 0; e < E; ++e) {
        const uint32_t g = wb + e * 32u + lane;
        if (g < np) {
            c1[g] = x[e].c;
            idx[g] = (uint16_t)x[e].s;
        }
    }
    __syncthreads();
}

// One leaf: records src[0 .. n) (or base + t when src is null), n at most
// the leaf capacity.
template <int WP, int MODE>
__device__ void pleaf(const PCtx<WP, MODE>& ctx, const uint32_t* src, uint32_t base, uint32_t n, unsigned char* smem,
                      PShared<2 * WP, MODE>& sh, const OutDesc& o) {
    constexpr int NW = 2 * WP;
    using Lay = PLayout<WP, MODE>;
    constexpr uint32_t CAP = Lay::CAP;
    using V = typename ValT<MODE>::T;
    uint64_t* keys = reinterpret_cast<uint64_t*>(smem + Lay::KEYS);
    uint64_t* c1 = reinterpret_cast<uint64_t*>(smem + Lay::C1);
    V* val = reinterpret_cast<V*>(smem + Lay::VAL);
    uint32_t* rr = reinterpret_cast<uint32_t*>(smem + Lay::RR);
    uint16_t* idx = reinterpret_cast<uint16_t*>(smem + Lay::IDX);
    uint16_t* seg = reinterpret_cast<uint16_t*>(smem + Lay::SEG);
    uint8_t* hd = smem + Lay::HD;
    const uint32_t tid = threadIdx.x;

    if (tid < (uint32_t)NW) {
        sh.mask[tid] = 0ull;
        sh.mand[tid] = ~0ull;
    }
    __syncthreads();
    // keys, contributions and records into shared memory, and the positions
    // where keys differ
    {
        uint64_t mo[NW], ma[NW];
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            mo[q] = 0ull;
            ma[q] = ~0ull;
        }
        for (uint32_t t = tid; t < n; t += kPThreads) {
            const uint32_t r = src ? src[t] : base + t;
            uint64_t k[NW];
            val[t] = ctx.value(r, k);
            rr[t] = r;
#pragma unroll
            for (int q = 0; q < NW; ++q) {
                keys[(size_t)q * CAP + t] = k[q];
                mo[q] |= k[q];
                ma[q] &= k[q];
            }
        }
        pmask_reduce<NW>(mo, ma, sh.mask, sh.mand);
    }
    __syncthreads();
    const uint32_t L = pmask_first<NW>(sh.mask, 0u, sh.mand);
    if (L >= 64u * NW) {  // one key: sum every contribution
        Acc<MODE> a;
        for (uint32_t t = tid; t < n; t += kPThreads) a.add(val[t]);
        const Acc<MODE> s = pblock_sum<MODE>(a, sh.acc);
        if (tid == 0) {
            uint64_t k[NW];
#pragma unroll
            for (int q = 0; q < NW; ++q) k[q] = keys[(size_t)q * CAP];
            pemit<WP>(o, sh.out, k, s.result());
            sh.out += 1u;
        }
        __syncthreads();
        return;
    }
    // sort by the window of 64 key bits from L; equal windows fall back to
    // the words from (L + 64) / 64 on (earlier bits are the window's or
    // shared)
    const uint32_t w0 = (L + 64u) >> 6;
    uint32_t npow = 32;
    while (npow < n) npow <<= 1;
    if (npow <= (uint32_t)kPThreads) psort_leaf_rows<NW, CAP, 1>(keys, c1, idx, rr, npow, n, L, w0);
    else if (npow <= 2u * kPThreads || CAP <= 2u * kPThreads)
        psort_leaf_rows<NW, CAP, (CAP > (uint32_t)kPThreads ? 2u : 1u)>(keys, c1, idx, rr, npow, n, L, w0);
    else psort_leaf_rows<NW, CAP, (CAP > 2u * kPThreads ? 4u : 1u)>(keys, c1, idx, rr, npow, n, L, w0);
    for (uint32_t t = tid; t < n; t += kPThreads)
        hd[t] = (t == 0 || pleaf_cmp<NW, CAP>(keys, c1, idx, t - 1u, t, n, w0) != 0) ? 1 : 0;
    __syncthreads();
    const uint32_t U = prank_heads(hd, seg, n, sh.warp);
    // sum each run in record order and write its term
    for (uint32_t t = tid; t < n; t += kPThreads) {
        if (!hd[t]) continue;
        Acc<MODE> a;
        a.add(val[idx[t]]);
        for (uint32_t u = t + 1; u < n && !hd[u]; ++u) a.add(val[idx[u]]);
        uint64_t k[NW];
        const uint32_t s = idx[t];
#pragma unroll
        for (int q = 0; q < NW; ++q) k[q] = keys[(size_t)q * CAP + s];
        pemit<WP>(o, sh.out + seg[t], k, a.result());
    }
    __syncthreads();
    if (tid == 0) sh.out += U;
    __syncthreads();
}

// Splits records src[0 .. n) (or base + t), whose keys agree before position
// D, into key ranges: by splitters taken from a sorted sample of their
// skip-zero codes (PCtx::skip) from D (digits false) or by the kPDigitBits
// key bits at D (digits true).  Each record's child goes to bid[t]; the records, grouped
// by child, to dst[0 .. n); the level is pushed.  A sample split that would
// leave every record in one child returns false with nothing pushed.
template <int WP, int MODE>
__device__ bool psplit(const PCtx<WP, MODE>& ctx, const uint32_t* src, uint32_t base, uint32_t n, uint32_t D,
                       bool digits, uint32_t cap, uint32_t fan, uint8_t* bid, uint32_t* dst, uint32_t lo,
                       uint32_t dbuf, PLevel* levels, unsigned char* smem, PShared<2 * WP, MODE>& sh) {
    constexpr int NW = 2 * WP;
    using Lay = PLayout<WP, MODE>;
    uint64_t* samp = reinterpret_cast<uint64_t*>(smem + Lay::KEYS);
    uint64_t* spl = samp + kPSample;
    const uint32_t tid = threadIdx.x;
    uint32_t nspl = kPFan - 1u;
    if (!digits) {
        // about fan * n / cap children: a fan-th of a leaf each on average
        const uint64_t want = ((uint64_t)fan * n + cap - 1) / cap;
        nspl = (uint32_t)(want < 2 ? 2 : (want > kPFan ? kPFan : want)) - 1u;
        // about 16 sampled codes per child (64 .. kPSample, a power of two)
        uint32_t S = 64;
        while (S < 16u * (nspl + 1u) && S < kPSample) S <<= 1;
        for (uint32_t t0 = tid; t0 < S; t0 += kPU * kPThreads) {
            uint32_t r[kPU];
            uint64_t c[kPU];
#pragma unroll
            for (int u = 0; u < kPU; ++u) {
                const uint32_t t = t0 + (uint32_t)u * kPThreads;
                const uint32_t pos = (uint32_t)(((uint64_t)t * n) / S);
                r[u] = t < S ? (src ? src[pos] : base + pos) : 0u;
            }
#pragma unroll
            for (int u = 0; u < kPU; ++u) c[u] = ctx.skip(r[u], D);
#pragma unroll
            for (int u = 0; u < kPU; ++u) {
                const uint32_t t = t0 + (uint32_t)u * kPThreads;
                if (t < S) samp[t] = c[u];
            }
        }
        __syncthreads();
        psort_codes(samp, S);
        // A code repeated among the splitters is frequent: its last copy
        // becomes its successor, so that the code gets a child of its own.
        uint64_t c = 0ull;
        if (tid < nspl) {
            c = samp[((uint64_t)(tid + 1u) * S) / (nspl + 1u)];
            const bool dup = tid > 0 && samp[((uint64_t)tid * S) / (nspl + 1u)] == c;
            const bool last = tid + 1u == nspl || samp[((uint64_t)(tid + 2u) * S) / (nspl + 1u)] != c;
            if (dup && last && c != ~0ull) c += 1ull;
        }
        __syncthreads();
        if (tid < nspl) spl[tid] = c;
    }
    sh.hist[tid] = 0;
    __syncthreads();
    for (uint32_t t0 = tid; t0 < n; t0 += kPU * kPThreads) {
        uint32_t r[kPU];
        uint64_t c[kPU];
#pragma unroll
        for (int u = 0; u < kPU; ++u) {
            const uint32_t t = t0 + (uint32_t)u * kPThreads;
            r[u] = t < n ? (src ? src[t] : base + t) : 0u;
        }
#pragma unroll
        for (int u = 0; u < kPU; ++u) {
            c[u] = digits ? ctx.window(r[u], D) : ctx.skip(r[u], D);
        }
#pragma unroll
        for (int u = 0; u < kPU; ++u) {
            const uint32_t t = t0 + (uint32_t)u * kPThreads;
            if (t >= n) continue;
            uint32_t b;
            if (digits) {
                b = (uint32_t)(c[u] >> (64u - kPDigitBits));
            } else {  // splitters at or below the code
                uint32_t l = 0, len = nspl;
                while (len > 0) {
                    const uint32_t half = len >> 1;
                    if (c[u] >= spl[l + half]) {
                        l += half + 1u;
                        len -= half + 1u;
                    } else {
                        len = half;
                    }
                }
                b = l;
            }
            bid[t] = (uint8_t)b;
            atomicAdd(&sh.hist[b], 1u);
        }
    }
    __syncthreads();
    if (!digits) {
        if (tid == 0) sh.full = 0;
        __syncthreads();
        if (sh.hist[tid] == n) sh.full = 1;
        __syncthreads();
        if (sh.full) return false;
    }
    uint32_t tot;
    const uint32_t ex = block_excl_scan<kPThreads>(sh.hist[tid], sh.warp, tot);
    sh.curs[tid] = ex;
    PLevel* L = levels + sh.depth;
    L->start[tid] = ex;
    {
        // Child tid's keys agree before D (and on the digit after a digit
        // split).  After a sample split its codes lie in [lo_c, hi_c) and
        // share the leading bits of lo_c and hi_c - 1: when those cover the
        // 6-bit field, every key has the same first nonzero window j1 after
        // D, so the keys agree up to that window's shared leading bits.
        uint32_t Dc = digits ? D + kPDigitBits : D;
        if (!digits && tid <= nspl) {
            const uint64_t lo_c = tid > 0 ? spl[tid - 1] : 0ull;
            if (tid == nspl || spl[tid] > lo_c) {
                const uint64_t hi_m = tid < nspl ? spl[tid] - 1ull : ~0ull;
                const uint32_t plen = (lo_c ^ hi_m) ? (uint32_t)__clzll((long long)(lo_c ^ hi_m)) : 64u;
                const uint32_t F = (uint32_t)(lo_c >> 58);
                const uint32_t K = D < 64u * NW ? (64u * NW - D + 63u) >> 6 : 0u;
                if (plen >= 6u && F == 0u) Dc = 64u * NW;  // every window zero: one key from D on
                else if (plen >= 6u && F <= K) Dc = D + 64u * (K - F) + (plen - 6u);
            }
        }
        L->D[tid] = (uint16_t)(Dc < 64u * NW ? Dc : 64u * NW);
    }
    if (tid == 0) {
        L->start[kPFan] = n;
        L->lo = lo;
        L->buf = dbuf;
        L->next = 0;
    }
    __syncthreads();
    for (uint32_t t0 = tid; t0 < n; t0 += kPU * kPThreads) {
        uint32_t r[kPU], b[kPU];
#pragma unroll
        for (int u = 0; u < kPU; ++u) {
            const uint32_t t = t0 + (uint32_t)u * kPThreads;
            r[u] = t < n ? (src ? src[t] : base + t) : 0u;
            b[u] = t < n ? bid[t] : 0u;
        }
#pragma unroll
        for (int u = 0; u < kPU; ++u) {
            const uint32_t t = t0 + (uint32_t)u * kPThreads;
            if (t < n) dst[atomicAdd(&sh.curs[b[u]], 1u)] = r[u];
        }
    }
    __syncthreads();
    if (tid == 0) sh.depth += 1u;
    __syncthreads();
    return true;
}

// A range larger than a leaf: split by sample while the walk is shallow;
// else (or when the sample separates nothing) find the range's first
// varying position and split by the digit there, or sum the range when all
// its keys are equal.
template <int WP, int MODE>
__device__ void pbig(const PCtx<WP, MODE>& ctx, const uint32_t* src, uint32_t base, uint32_t n, uint32_t Dhint,
                     uint32_t cap, uint32_t fan, uint8_t* bid, uint32_t* dst, uint32_t lo, uint32_t dbuf, PLevel* levels,
                     unsigned char* smem, PShared<2 * WP, MODE>& sh, const OutDesc& o, int32_t* err) {
    constexpr int NW = 2 * WP;
    const uint32_t tid = threadIdx.x;
    if (sh.depth < kPSampleDepth &&
        psplit<WP, MODE>(ctx, src, base, n, Dhint, false, cap, fan, bid, dst, lo, dbuf, levels, smem, sh))
        return;
    if (tid < (uint32_t)NW) {
        sh.mask[tid] = 0ull;
        sh.mand[tid] = ~0ull;
    }
    __syncthreads();
    {
        uint64_t mo[NW], ma[NW];
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            mo[q] = 0ull;
            ma[q] = ~0ull;
        }
        for (uint32_t t = tid; t < n; t += kPThreads) {
            uint64_t k[NW];
            ctx.key(src ? src[t] : base + t, k);
#pragma unroll
            for (int q = 0; q < NW; ++q) {
                mo[q] |= k[q];
                ma[q] &= k[q];
            }
        }
        pmask_reduce<NW>(mo, ma, sh.mask, sh.mand);
    }
    __syncthreads();
    const uint32_t D = pmask_first<NW>(sh.mask, 0u, sh.mand);
    if (D < 64u * NW) {
        if (sh.depth >= persist_depth<NW>()) {  // cannot happen: the depth is bounded
            if (tid == 0) atomicOr(err, ERR_STACK);
            __syncthreads();
            return;
        }
        psplit<WP, MODE>(ctx, src, base, n, D, true, cap, fan, bid, dst, lo, dbuf, levels, smem, sh);
        return;
    }
    Acc<MODE> a;
    for (uint32_t t = tid; t < n; t += kPThreads) {
        uint64_t k[NW];
        a.add(ctx.value(src ? src[t] : base + t, k));
    }
    const Acc<MODE> s = pblock_sum<MODE>(a, sh.acc);
    if (tid == 0) {
        uint64_t k[NW];
        ctx.key(src ? src[0] : base, k);
        pemit<WP>(o, sh.out, k, s.result());
        sh.out += 1u;
    }
    __syncthreads();
}

template <int WP, int MODE>
__global__ void __launch_bounds__(kPThreads, 2)
    k_batch_persist(const ProbDesc* __restrict__ probs, const OutDesc* __restrict__ outs,
                    const uint32_t* __restrict__ order, const uint32_t* __restrict__ r0s, uint32_t nprob,
                    uint32_t* buf0, uint32_t* buf1, uint8_t* bid_all, PLevel* level_store, uint32_t* ticket,
                    unsigned long long* counts, int32_t* err, uint32_t cap, uint32_t fan) {
    constexpr int NW = 2 * WP;
    using Lay = PLayout<WP, MODE>;
    using V = typename ValT<MODE>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ PShared<NW, MODE> sh;
    uint64_t* sbk = reinterpret_cast<uint64_t*>(smem + Lay::BK);
    V* sbc = reinterpret_cast<V*>(smem + Lay::BC);
    uint8_t* sbp = smem + Lay::BP;
    PLevel* levels = level_store + (size_t)blockIdx.x * persist_depth<NW>();
    const uint32_t tid = threadIdx.x;
    cap = (cap == 0 || cap > Lay::CAP) ? Lay::CAP : cap;
    fan = fan == 0 ? 2u : fan;

    for (;;) {
        if (tid == 0) sh.prob = atomicAdd(ticket, 1u);
        __syncthreads();
        const uint32_t tk = sh.prob;
        if (tk >= nprob) break;
        const uint32_t b = order[tk];
        const ProbDesc d = probs[b];
        const OutDesc o = outs[b];
        const uint32_t P = d.na * d.nb;  // below 2^32 (checked on the host)
        for (uint32_t q = tid; q < d.nb * (uint32_t)NW; q += kPThreads) sbk[q] = __ldg(d.bk + q);
        for (uint32_t q = tid; q < d.nb; q += kPThreads) {
            sbp[q] = __ldg(d.bp + q);
            sbc[q] = static_cast<const V*>(d.bc)[q];
        }
        if (tid == 0) {
            sh.out = 0;
            sh.depth = 0;
        }
        __syncthreads();
        const PCtx<WP, MODE> ctx{d.ak, d.ap, static_cast<const V*>(d.ac), sbk, sbp, sbc, d.na, d.na_inv};
        const uint32_t r0 = r0s[b];
        uint32_t* bufs[2] = {buf0 + r0, buf1 + r0};
        uint8_t* bid = bid_all + r0;
        if (P > 0 && P <= cap) {
            pleaf<WP, MODE>(ctx, nullptr, 0u, P, smem, sh, o);
        } else if (P > 0) {
            // The first varying position of all products: the positions where
            // some a_i differs from a_0 or some b_j from b_0, since
            // (a_i ^ b_j) ^ (a_0 ^ b_0) = (a_i ^ a_0) ^ (b_j ^ b_0).
            if (tid < (uint32_t)NW) {
                sh.mask[tid] = 0ull;
                sh.mand[tid] = ~0ull;
            }
            __syncthreads();
            {
                uint64_t mo[NW], ma[NW];
#pragma unroll
                for (int q = 0; q < NW; ++q) {
                    mo[q] = 0ull;
                    ma[q] = ~0ull;
                }
                for (uint32_t t = tid; t < d.na; t += kPThreads) {
                    uint64_t k[NW];
                    key_load_g<NW>(d.ak, t, k);
#pragma unroll
                    for (int q = 0; q < NW; ++q) {
                        mo[q] |= k[q];
                        ma[q] &= k[q];
                    }
                }
                pmask_reduce<NW>(mo, ma, sh.mask, sh.mand);
            }
            __syncthreads();
            pmask_finish<NW>(sh.mask, sh.mand);  // positions where A's terms differ
            {
                uint64_t mo[NW];
#pragma unroll
                for (int q = 0; q < NW; ++q) mo[q] = sh.mask[q];  // kept: OR-ed with B's below
                __syncthreads();
                if (tid < (uint32_t)NW) {
                    sh.mask[tid] = 0ull;
                    sh.mand[tid] = ~0ull;
                }
                __syncthreads();
                uint64_t bo[NW], ba[NW];
#pragma unroll
                for (int q = 0; q < NW; ++q) {
                    bo[q] = 0ull;
                    ba[q] = ~0ull;
                }
                for (uint32_t t = tid; t < d.nb; t += kPThreads) {
                    uint64_t k[NW];
                    key_load_s<NW>(sbk, t, k);
#pragma unroll
                    for (int q = 0; q < NW; ++q) {
                        bo[q] |= k[q];
                        ba[q] &= k[q];
                    }
                }
                pmask_reduce<NW>(bo, ba, sh.mask, sh.mand);
                __syncthreads();
                pmask_finish<NW>(sh.mask, sh.mand);  // positions where B's terms differ
#pragma unroll
                for (int q = 0; q < NW; ++q)
                    if (tid == (uint32_t)q) sh.mask[q] |= mo[q];
            }
            __syncthreads();
            const uint32_t D = pmask_first<NW>(sh.mask);
            pbig<WP, MODE>(ctx, nullptr, 0u, P, D, cap, fan, bid, bufs[0], 0u, 0u, levels, smem, sh, o, err);
            // depth-first walk of the children, in key order
            for (;;) {
                if (sh.depth == 0) break;
                PLevel* L = levels + sh.depth - 1u;
                if (tid == 0) sh.next = kPFan;
                __syncthreads();
                if (tid >= L->next && L->start[tid + 1] > L->start[tid]) atomicMin(&sh.next, tid);
                __syncthreads();
                const uint32_t dg = sh.next;
                if (dg >= kPFan) {
                    __syncthreads();
                    if (tid == 0) sh.depth -= 1u;
                    __syncthreads();
                    continue;
                }
                const uint32_t lo = L->lo + L->start[dg];
                const uint32_t n = L->start[dg + 1] - L->start[dg];
                const uint32_t cb = L->buf;
                const uint32_t Dh = L->D[dg];
                __syncthreads();
                if (tid == 0) L->next = dg + 1u;
                __syncthreads();
                if (n <= cap)
                    pleaf<WP, MODE>(ctx, bufs[cb] + lo, 0u, n, smem, sh, o);
                else
                    pbig<WP, MODE>(ctx, bufs[cb] + lo, 0u, n, Dh, cap, fan, bid + lo, bufs[cb ^ 1u] + lo, lo, cb ^ 1u,
                                   levels, smem, sh, o, err);
            }
        }
        if (tid == 0) counts[b] = sh.out;
        __syncthreads();
    }
}

}  // namespace paulib
