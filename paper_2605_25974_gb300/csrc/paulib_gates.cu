// paulib_gates.cu -- Clifford gate application and the Pauli rotation step
// (PauLIB Sec. III-B: conjugation Q' = U Q U^dagger; gate application of
// Sec. VI), on the library's device sums.
//
// A term is c * i^phase * P(x, z) with P(x, z) = i^{|x&z|} X^x Z^z, a
// Hermitian Pauli string.  Conjugation by a Clifford gate maps P(x, z) to
// +-P(x', z'), so a gate rewrites a few key bits and at most flips the sign of
// the coefficient.  The bit rules follow from the gates' action on X and Z:
//   H:    X <-> Z                          (x, z) -> (z, x)
//   S:    X -> XZ*i (= Y), Z -> Z           z ^= x
//   CNOT: X_c -> X_c X_t, Z_t -> Z_c Z_t    x_t ^= x_c, z_c ^= z_t
//   CZ:   X_c -> X_c Z_t, X_t -> Z_c X_t    z_t ^= x_c, z_c ^= x_t
// Written in the X^x Z^z product form the image carries a factor i^u
// (u = 2xz for H, x for S, 0 for CNOT, 2 x_c x_t for CZ, from reordering the
// factors); renormalising to P(x', z') multiplies it by
// i^{|x&z| - |x'&z'|} over the gate's qubits.  The total exponent is 0 or 2.
#include "paulib_pipeline.cuh"

namespace paulib {

constexpr int kCliffordThreads = 256;

// One gate's action on the bits of its qubits: (xc, zc) of q1 and (xt, zt) of
// q2 (zero for one-qubit gates) become (nxc, nzc, nxt, nzt).  Returns the
// exponent e (mod 4) the image's sign carries in the normal form: the factor
// i^u from reordering X and Z, times i^{|x&z| - |x'&z'|} over the two qubits.
__device__ __forceinline__ uint32_t gate_rule(int32_t gate, uint32_t xc, uint32_t zc, uint32_t xt, uint32_t zt,
                                              uint32_t& nxc, uint32_t& nzc, uint32_t& nxt, uint32_t& nzt) {
    nxc = xc;
    nzc = zc;
    nxt = xt;
    nzt = zt;
    uint32_t u = 0;
    if (gate == PAULIB_GATE_H) {
        nxc = zc;
        nzc = xc;
        u = 2u * (xc & zc);
    } else if (gate == PAULIB_GATE_S) {
        nzc = zc ^ xc;
        u = xc;
    } else if (gate == PAULIB_GATE_CNOT) {
        nxt = xt ^ xc;
        nzc = zc ^ zt;
    } else {  // CZ
        nzc = zc ^ xt;
        nzt = zt ^ xc;
        u = 2u * (xc & xt);
    }
    const uint32_t before = (xc & zc) + (xt & zt);
    const uint32_t after = (nxc & nzc) + (nxt & nzt);
    return (u + before - after) & 3u;
}

// Applies the gate list to one term held in shared memory, word-major (word
// w of this thread's term at sk[w * kCliffordThreads]), so that a gate reads
// and writes just the words it touches without bank conflicts; returns the
// exponent e (mod 4) with U P(x,z) U^dagger = i^e P(x',z').
template <int WP>
__device__ __forceinline__ uint32_t conjugate_term(uint64_t* sk, const int32_t* __restrict__ ops, int32_t nops) {
    uint32_t e = 0;
    for (int32_t g = 0; g < nops; ++g) {
        const int32_t gate = __ldg(ops + 3 * g), q1 = __ldg(ops + 3 * g + 1), q2 = __ldg(ops + 3 * g + 2);
        const uint32_t w1 = (uint32_t)q1 >> 6, b1 = (uint32_t)q1 & 63u;
        const uint32_t w2 = (uint32_t)q2 >> 6, b2 = (uint32_t)q2 & 63u;
        uint64_t* x1 = sk + (size_t)w1 * kCliffordThreads;
        uint64_t* z1 = sk + (size_t)(WP + w1) * kCliffordThreads;
        uint64_t* x2 = sk + (size_t)w2 * kCliffordThreads;
        uint64_t* z2 = sk + (size_t)(WP + w2) * kCliffordThreads;
        const bool two = gate == PAULIB_GATE_CNOT || gate == PAULIB_GATE_CZ;
        const uint32_t xc = (uint32_t)(*x1 >> b1) & 1u, zc = (uint32_t)(*z1 >> b1) & 1u;
        const uint32_t xt = two ? (uint32_t)(*x2 >> b2) & 1u : 0u, zt = two ? (uint32_t)(*z2 >> b2) & 1u : 0u;
        uint32_t nxc, nzc, nxt, nzt;
        e = (e + gate_rule(gate, xc, zc, xt, zt, nxc, nzc, nxt, nzt)) & 3u;
        *x1 ^= (uint64_t)(xc ^ nxc) << b1;
        *z1 ^= (uint64_t)(zc ^ nzc) << b1;
        if (two) {
            *x2 ^= (uint64_t)(xt ^ nxt) << b2;
            *z2 ^= (uint64_t)(zt ^ nzt) << b2;
        }
    }
    return e;
}

// Each term is read once, conjugated by the whole gate list and written
// once: HBM traffic per term is one record read and one written, whatever
// the number of gates.
template <int WP>
__global__ void __launch_bounds__(kCliffordThreads) k_clifford(uint64_t* keys, double2* coef, uint8_t* pbase,
                                                               const uint8_t* __restrict__ phase, int64_t n,
                                                               const int32_t* __restrict__ ops, int32_t nops) {
    constexpr int NW = 2 * WP;
    extern __shared__ uint64_t s_keys[];  // [NW][kCliffordThreads]
    uint64_t* sk = s_keys + threadIdx.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k[NW];
        key_load_g<NW>(keys, (uint64_t)t, k);
#pragma unroll
        for (int w = 0; w < NW; ++w) sk[(size_t)w * kCliffordThreads] = k[w];
        const uint32_t e = conjugate_term<WP>(sk, ops, nops);
#pragma unroll
        for (int w = 0; w < NW; ++w) k[w] = sk[(size_t)w * kCliffordThreads];
        key_store<NW>(keys, (uint64_t)t, k);
        if (e) {
            const double2 c = coef[t];
            coef[t] = make_double2(-c.x, -c.y);  // e is 2: an exact sign flip
        }
        pbase[t] = (uint8_t)normal_phase<WP>(k, phase ? (uint32_t)phase[t] : 0u);
    }
}

// Gate lists whose qubits all lie in one 64-bit word w (any single gate, for
// instance): the term's other words do not change, so each term reads and
// writes only its x and z words w (the struct-of-arrays observation of Sec.
// III-G, on the per-term key layout), its phase byte, which moves by the change
// of |x&z| on word w, and its coefficient where the image is -P; a term the
// gates leave unchanged is only read.
template <int WP>
__global__ void __launch_bounds__(kCliffordThreads) k_clifford_word(uint64_t* keys, double2* coef, uint8_t* pbase,
                                                                    int64_t n, int32_t w,
                                                                    const int32_t* __restrict__ ops, int32_t nops) {
    constexpr int NW = 2 * WP;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        uint64_t* kx = keys + t * NW + w;
        const uint64_t x0 = kx[0], z0 = kx[WP];
        uint64_t x = x0, z = z0;
        const int before = __popcll(x & z);
        uint32_t e = 0;
        for (int32_t g = 0; g < nops; ++g) {
            const int32_t gate = __ldg(ops + 3 * g);
            const uint32_t b1 = (uint32_t)__ldg(ops + 3 * g + 1) & 63u, b2 = (uint32_t)__ldg(ops + 3 * g + 2) & 63u;
            const bool two = gate == PAULIB_GATE_CNOT || gate == PAULIB_GATE_CZ;
            const uint32_t xc = (uint32_t)(x >> b1) & 1u, zc = (uint32_t)(z >> b1) & 1u;
            const uint32_t xt = two ? (uint32_t)(x >> b2) & 1u : 0u, zt = two ? (uint32_t)(z >> b2) & 1u : 0u;
            uint32_t nxc, nzc, nxt, nzt;
            e = (e + gate_rule(gate, xc, zc, xt, zt, nxc, nzc, nxt, nzt)) & 3u;
            x ^= (uint64_t)(xc ^ nxc) << b1;
            z ^= (uint64_t)(zc ^ nzc) << b1;
            if (two) {
                x ^= (uint64_t)(xt ^ nxt) << b2;
                z ^= (uint64_t)(zt ^ nzt) << b2;
            }
        }
        if (x != x0 || z != z0) {  // unchanged terms (identity on the gates' qubits) write nothing
            kx[0] = x;
            kx[WP] = z;
            const int after = __popcll(x & z);
            if (after != before) pbase[t] = (uint8_t)((pbase[t] + after - before) & 3);
        }
        if (e) {
            const double2 c = coef[t];
            coef[t] = make_double2(-c.x, -c.y);  // e is 2: an exact sign flip
        }
    }
}

void apply_clifford(paulib_sum* s, int32_t nops, const int32_t* ops_host, cudaStream_t st) {
    if (nops == 0 || s->n_terms == 0) return;
    Scratch ops((size_t)nops * 3 * sizeof(int32_t), st);
    check_cuda(cudaMemcpyAsync(ops.p, ops_host, (size_t)nops * 3 * sizeof(int32_t), cudaMemcpyHostToDevice, st),
               "gate list copy");
    const int sms = device_sm_count();
    const unsigned grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((s->n_terms + kCliffordThreads - 1) / kCliffordThreads, (int64_t)sms * 8));
    const size_t sm = (size_t)2 * s->WP * kCliffordThreads * 8;
    StageScope ss(ST_CONVERT, st);
    note_launch(ST_CONVERT);
    // one word holding every qubit of the list: touch only that word
    const int32_t w0 = ops_host[1] >> 6;
    bool one_word = true;
    for (int32_t g = 0; g < nops && one_word; ++g) {
        const int32_t gate = ops_host[3 * g];
        const bool two = gate == PAULIB_GATE_CNOT || gate == PAULIB_GATE_CZ;
        one_word = (ops_host[3 * g + 1] >> 6) == w0 && (!two || (ops_host[3 * g + 2] >> 6) == w0);
    }
    if (one_word) {
#define LW(WPv) k_clifford_word<WPv><<<grid, kCliffordThreads, 0, st>>>(s->keys, s->coef, s->pbase, s->n_terms, w0, \
                                                                        ops.as<int32_t>(), nops);
        PAULIB_DISPATCH_WP(s->WP, LW);
#undef LW
        check_cuda(cudaGetLastError(), "k_clifford_word");
        s->is_canonical = 0;
        return;
    }
#define L(WPv)                                                                                               \
    {                                                                                                        \
        auto kern = k_clifford<WPv>;                                                                         \
        smem_attr(kern, sm);                                                                                 \
        kern<<<grid, kCliffordThreads, sm, st>>>(s->keys, s->coef, s->pbase, s->phase, s->n_terms,         \
                                                 ops.as<int32_t>(), nops);                                   \
    }
    PAULIB_DISPATCH_WP(s->WP, L);
#undef L
    check_cuda(cudaGetLastError(), "k_clifford");
    // the keys moved: the sum keeps its terms and their order but is no longer sorted
    s->is_canonical = 0;
}

// ---------------------------------------------------------------- pair products

// Output t = a_t * b_t (the single Pauli multiplication of Sec. III-A/III-E,
// applied pair by pair): product key, phase exponent k (both inputs' phases
// included) and coefficient c_a c_b, in the raw form.
template <int WP>
__global__ void __launch_bounds__(256) k_pairwise(const uint64_t* __restrict__ ak, const double2* __restrict__ ac,
                                                  const uint8_t* __restrict__ ap, const uint64_t* __restrict__ bk,
                                                  const double2* __restrict__ bc, const uint8_t* __restrict__ bp,
                                                  int64_t n, uint64_t* ok, double2* oc, uint8_t* oph, uint8_t* opb) {
    constexpr int NW = 2 * WP;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        uint64_t a[NW], b[NW], o[NW];
        key_load_g<NW>(ak, (uint64_t)t, a);
        key_load_g<NW>(bk, (uint64_t)t, b);
        const uint32_t k = string_product<WP>(a, b, ap[t], bp[t], o);
        key_store<NW>(ok, (uint64_t)t, o);
        oc[t] = cmul(ac[t], bc[t]);
        oph[t] = (uint8_t)k;
        opb[t] = (uint8_t)normal_phase<WP>(o, k);
    }
}

paulib_sum* multiply_pairwise(const paulib_sum* a, const paulib_sum* b, cudaStream_t st) {
    paulib_sum* out = sum_alloc(a->n_qubits, a->n_terms, true, st);
    if (a->n_terms == 0) return out;
    const int sms = device_sm_count();
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((a->n_terms + 255) / 256, (int64_t)sms * 8));
    StageScope ss(ST_RAW, st);
    note_launch(ST_RAW);
#define L(WPv)                                                                                                \
    k_pairwise<WPv><<<grid, 256, 0, st>>>(a->keys, a->coef, a->pbase, b->keys, b->coef, b->pbase, a->n_terms, \
                                          out->keys, out->coef, out->phase, out->pbase)
    PAULIB_DISPATCH_WP(a->WP, L);
#undef L
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        sum_free(out, st);
        check_cuda(e, "k_pairwise");
    }
    return out;
}

// ---------------------------------------------------------------- Pauli rotation

// Flags the terms that anti-commute with P: the symplectic inner product
// <x|z_P> + <z|x_P> (mod 2) is 1 (Sec. III-F).
template <int WP>
__global__ void __launch_bounds__(256) k_rot_flags(const uint64_t* __restrict__ keys, int64_t n,
                                                   const uint64_t* __restrict__ pk, uint8_t* flags) {
    constexpr int NW = 2 * WP;
    uint64_t p[NW];
    key_load_g<NW>(pk, 0, p);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k[NW];
        key_load_g<NW>(keys, (uint64_t)t, k);
        uint64_t s = 0;
#pragma unroll
        for (int q = 0; q < WP; ++q) s ^= (k[q] & p[WP + q]) ^ (k[WP + q] & p[q]);
        flags[t] = (uint8_t)(__popcll(s) & 1);
    }
}

// Term t of the input, scaled by cos(theta) when it anti-commutes, to slot t
// of the raw output.
template <int WP>
__global__ void __launch_bounds__(256) k_rot_copy(const uint64_t* __restrict__ keys, const double2* __restrict__ coef,
                                                  const uint8_t* __restrict__ phase, const uint8_t* __restrict__ flags,
                                                  int64_t n, double cth, uint64_t* okeys, double2* ocoef,
                                                  uint8_t* ophase, uint8_t* opb) {
    constexpr int NW = 2 * WP;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k[NW];
        key_load_g<NW>(keys, (uint64_t)t, k);
        key_store<NW>(okeys, (uint64_t)t, k);
        double2 c = coef[t];
        if (flags[t]) c = make_double2(c.x * cth, c.y * cth);
        ocoef[t] = c;
        const uint32_t ph = phase ? phase[t] : 0u;
        ophase[t] = (uint8_t)ph;
        opb[t] = (uint8_t)normal_phase<WP>(k, ph);
    }
}

// The partner -i sin(theta) P Q of each anti-commuting term, at slot
// n + (its rank among them).  P Q = i^k P(x_P ^ x, z_P ^ z), k from the
// string product (Sec. III-E) with Q's own phase folded into its exponent.
template <int WP>
__global__ void __launch_bounds__(kChunkThreads) k_rot_partner(uint32_t nch, const uint8_t* __restrict__ flags,
                                                             const uint64_t* __restrict__ coff,
                                                             const uint64_t* __restrict__ keys,
                                                             const double2* __restrict__ coef,
                                                             const uint8_t* __restrict__ pbase,
                                                             const uint64_t* __restrict__ pk, uint32_t p_pb,
                                                             int64_t n, double sth, uint64_t* okeys, double2* ocoef,
                                                             uint8_t* ophase, uint8_t* opb) {
    constexpr int NW = 2 * WP;
    __shared__ uint32_t s_warp[32];
    uint64_t p[NW];
    key_load_g<NW>(pk, 0, p);
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
        for_each_flagged(c, flags, coff, s_warp, [&](uint64_t t, uint64_t d) {
            uint64_t q[NW], o[NW];
            key_load_g<NW>(keys, t, q);
            const uint32_t k = string_product<WP>(p, q, p_pb, pbase[t], o);
            const uint64_t slot = (uint64_t)n + d;
            key_store<NW>(okeys, slot, o);
            const double2 cq = coef[t];
            ocoef[slot] = make_double2(cq.y * sth, -cq.x * sth);  // c * (-i sin theta)
            ophase[slot] = (uint8_t)k;
            opb[slot] = (uint8_t)normal_phase<WP>(o, k);
        });
    }
}

template <int WP>
__global__ void __launch_bounds__(256) k_trunc_flags(const double2* __restrict__ coef, int64_t n, double thr2,
                                                     uint8_t* flags) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const double2 c = coef[t];
        flags[t] = (uint8_t)(c.x * c.x + c.y * c.y >= thr2);
    }
}

// Flag scan over n slots: flags (nch * kChunk bytes, zeroed) -> coff; returns
// the number of flagged slots (one host synchronisation).
static uint64_t flag_offsets(const uint8_t* flags, uint32_t nch, Scratch& coff, cudaStream_t st) {
    Scratch cnt((size_t)nch * 4, st);
    coff = Scratch((size_t)(nch + 1) * 8, st);
    const int sms = device_sm_count();
    k_flag_count<<<std::max<uint32_t>(1, std::min<uint32_t>(nch, (uint32_t)sms * 8)), kChunkThreads, 0, st>>>(
        flags, nch, cnt.as<uint32_t>());
    k_scan_counts<<<1, 1024, 0, st>>>(cnt.as<uint32_t>(), nch, coff.as<uint64_t>());
    note_launch(ST_COMPACT);
    note_launch(ST_COMPACT);
    check_cuda(cudaGetLastError(), "flag scan");
    uint64_t total = 0;
    check_cuda(cudaMemcpyAsync(&total, coff.as<uint64_t>() + nch, 8, cudaMemcpyDeviceToHost, st), "count copy");
    check_cuda(cudaStreamSynchronize(st), "count sync");
    return total;
}

// ---------------------------------------------------------------- canonical merge
//
// A rotation of a canonical sum keeps its terms Q in key order (scaled by
// cos(theta) where they anti-commute with P); only the partners P Q need
// sorting.  The partners are canonicalised on their own and the two sorted,
// duplicate-free lists are merged, a partner equal to some Q adding its
// coefficient to that Q's: merge-path tiles of kMergeTile outputs.

constexpr int kMergeThreads = 128;
constexpr int kMergeItems = 4;
constexpr int kMergeTile = kMergeThreads * kMergeItems;
constexpr int kMergeCols = kMergeTile + 2;  // the tile's keys plus A[a0-1] and B[b1]

// Keys compared word by word, word 0 most significant: -1, 0 or 1.
template <int NW>
__device__ __forceinline__ int key_cmp3(const uint64_t* a, int sa, const uint64_t* b, int sb) {
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        const uint64_t x = a[q * sa], y = b[q * sb];
        if (x != y) return x < y ? -1 : 1;
    }
    return 0;
}

// split[c] = number of A terms among the first min(L, c * kMergeTile) outputs
// of the merge (A before B on equal keys).
template <int WP>
__global__ void __launch_bounds__(256) k_merge_split(const uint64_t* __restrict__ ak, int64_t na,
                                                     const uint64_t* __restrict__ bk, int64_t nb, int64_t ntiles,
                                                     int64_t* split) {
    constexpr int NW = 2 * WP;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c > ntiles) return;
    const int64_t d = min(na + nb, c * (int64_t)kMergeTile);
    int64_t lo = max((int64_t)0, d - nb), hi = min(d, na);
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (key_cmp3<NW>(ak + mid * NW, 1, bk + (d - 1 - mid) * NW, 1) <= 0) lo = mid + 1;
        else hi = mid;
    }
    split[c] = lo;
}

// One tile: stage its keys word-major in shared memory (A[a0-1], A[a0..a1),
// B[b0..b1), B[b1]), split it again per thread, merge kMergeItems outputs per
// thread into slot order.  An A term equal to the B term that follows it
// takes that term's coefficient; the B slot is then left unflagged.  With
// thr2 > 0, slots whose |c|^2 < thr2 are left unflagged too (truncation).
template <int WP>
__global__ void __launch_bounds__(kMergeThreads) k_merge_tile(const uint64_t* __restrict__ ak,
                                                              const double2* __restrict__ ac, int64_t na,
                                                              const uint64_t* __restrict__ bk,
                                                              const double2* __restrict__ bc, int64_t nb,
                                                              const int64_t* __restrict__ split, double thr2,
                                                              uint64_t* tk, double2* tc, uint8_t* tflag) {
    constexpr int NW = 2 * WP;
    constexpr int S = kMergeCols;
    extern __shared__ uint64_t s_key[];  // [NW][S]
    const int64_t L = na + nb;
    const int64_t d0 = (int64_t)blockIdx.x * kMergeTile, d1 = min(L, d0 + kMergeTile);
    const int64_t a0 = split[blockIdx.x], a1 = split[blockIdx.x + 1];
    const int64_t b0 = d0 - a0, b1 = d1 - a1;
    const int ta = (int)(a1 - a0), tb = (int)(b1 - b0);
    // staged column j: 0 = A[a0-1], 1..ta = A[a0..a1), ta+1..ta+tb = B[b0..b1), ta+tb+1 = B[b1]
    for (int e = threadIdx.x; e < (ta + 1) * NW; e += kMergeThreads) {
        const int j = e / NW, q = e - j * NW;
        const int64_t ga = a0 - 1 + j;
        if (ga >= 0 && ga < na) s_key[q * S + j] = __ldg(ak + ga * NW + q);
    }
    for (int e = threadIdx.x; e < (tb + 1) * NW; e += kMergeThreads) {
        const int j = e / NW, q = e - j * NW;
        const int64_t gb = b0 + j;
        if (gb < nb) s_key[q * S + ta + 1 + j] = __ldg(bk + gb * NW + q);
    }
    __syncthreads();
    const uint64_t* sA = s_key + 1;       // sA[i], i in [-1, ta)
    const uint64_t* sB = s_key + ta + 1;  // sB[j], j in [0, tb]
    const int k = threadIdx.x * kMergeItems;
    if (d0 + k >= d1) return;
    int lo = max(0, k - tb), hi = min(k, ta);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (key_cmp3<NW>(sA + mid, S, sB + (k - 1 - mid), S) <= 0) lo = mid + 1;
        else hi = mid;
    }
    int a = lo, b = k - lo;
    for (int it = 0; it < kMergeItems; ++it) {
        const int64_t p = d0 + k + it;
        if (p >= d1) break;
        const bool takeA = b >= tb || (a < ta && key_cmp3<NW>(sA + a, S, sB + b, S) <= 0);
        const uint64_t* src;
        double2 c;
        bool keep;
        if (takeA) {
            src = sA + a;
            c = ac[a0 + a];
            // the B term right after it in key order: in the tile, or B[b1]
            if (b0 + b < nb && key_cmp3<NW>(sA + a, S, sB + b, S) == 0) {
                const double2 cb = bc[b0 + b];
                c = make_double2(c.x + cb.x, c.y + cb.y);
            }
            keep = true;
            ++a;
        } else {
            src = sB + b;
            c = bc[b0 + b];
            // equal to the A term before it: already added there
            keep = !(a0 + a > 0 && key_cmp3<NW>(sA + a - 1, S, sB + b, S) == 0);
            ++b;
        }
        if (thr2 > 0 && c.x * c.x + c.y * c.y < thr2) keep = false;
        tflag[p] = keep ? 1 : 0;
        if (keep) {
#pragma unroll
            for (int q = 0; q < NW; ++q) tk[p * NW + q] = src[q * S];
            tc[p] = c;
        }
    }
}

// Merges the canonical Q part (the first n terms of raw) with the separately
// canonicalised partners pc into a new canonical sum, truncating at threshold.
template <int WP>
static paulib_sum* merge_rotated(const paulib_sum* raw, int64_t n, const paulib_sum* pc, double threshold,
                                 cudaStream_t st) {
    constexpr int NW = 2 * WP;
    const int64_t nb = pc->n_terms, L = n + nb;
    const int64_t ntiles = (L + kMergeTile - 1) / kMergeTile;
    Scratch split((size_t)(ntiles + 1) * 8, st);
    const uint32_t nch = (uint32_t)((L + kChunk - 1) / kChunk);
    Scratch tkeys((size_t)L * NW * 8, st), tcoef((size_t)L * 16, st), tflag((size_t)nch * kChunk, st), coff;
    check_cuda(cudaMemsetAsync(tflag.p, 0, (size_t)nch * kChunk, st), "memset flags");
    {
        StageScope ss(ST_COMPACT, st);
        note_launch(ST_COMPACT);
        k_merge_split<WP><<<(unsigned)((ntiles + 1 + 255) / 256), 256, 0, st>>>(raw->keys, n, pc->keys, nb, ntiles,
                                                                                split.as<int64_t>());
        const size_t sm = (size_t)NW * kMergeCols * 8;
        smem_attr(k_merge_tile<WP>, sm);
        note_launch(ST_COMPACT);
        k_merge_tile<WP><<<(unsigned)ntiles, kMergeThreads, sm, st>>>(
            raw->keys, raw->coef, n, pc->keys, pc->coef, nb, split.as<int64_t>(),
            threshold > 0 ? threshold * threshold : 0.0, tkeys.as<uint64_t>(), tcoef.as<double2>(),
            tflag.as<uint8_t>());
        check_cuda(cudaGetLastError(), "merge kernels");
    }
    const uint64_t keep = flag_offsets(tflag.as<uint8_t>(), nch, coff, st);
    paulib_sum* out = sum_alloc(raw->n_qubits, (int64_t)keep, false, st);
    out->is_canonical = 1;
    if (keep > 0) {
        StageScope ss(ST_COMPACT, st);
        note_launch(ST_COMPACT);
        const int sms = device_sm_count();
        k_compact<WP><<<std::max<uint32_t>(1, std::min<uint32_t>(nch, (uint32_t)sms * 8)), kChunkThreads, 0, st>>>(
            nch, tflag.as<uint8_t>(), coff.as<uint64_t>(), tkeys.as<uint64_t>(), tcoef.as<double2>(), out->keys,
            out->coef, out->pbase);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            sum_free(out, st);
            check_cuda(e, "k_compact");
        }
    }
    return out;
}

template <int WP>
static paulib_sum* rotate_wp(const paulib_sum* s, const uint64_t* pk_host, double theta, double threshold, int mode,
                             cudaStream_t st) {
    constexpr int NW = 2 * WP;
    const int64_t n = s->n_terms;
    const int sms = device_sm_count();
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8));
    Scratch pk((size_t)NW * 8, st);
    check_cuda(cudaMemcpyAsync(pk.p, pk_host, (size_t)NW * 8, cudaMemcpyHostToDevice, st), "generator copy");
    uint32_t p_pb = 0;
    for (int q = 0; q < WP; ++q) p_pb += (uint32_t)__builtin_popcountll(pk_host[q] & pk_host[WP + q]);
    p_pb &= 3u;
    const uint32_t nch = (uint32_t)((n + kChunk - 1) / kChunk);
    Scratch flags((size_t)nch * kChunk, st), coff;
    check_cuda(cudaMemsetAsync(flags.p, 0, (size_t)nch * kChunk, st), "memset flags");
    {
        StageScope ss(ST_CONVERT, st);
        note_launch(ST_CONVERT);
        k_rot_flags<WP><<<grid, 256, 0, st>>>(s->keys, n, pk.as<uint64_t>(), flags.as<uint8_t>());
        check_cuda(cudaGetLastError(), "k_rot_flags");
    }
    const uint64_t anti = flag_offsets(flags.as<uint8_t>(), nch, coff, st);
    if ((uint64_t)n + anti >= ((uint64_t)1 << 32) - 1) fail(PAULIB_ERR_UNSUPPORTED, "rotation result needs < 2^32 terms");
    paulib_sum* raw = sum_alloc(s->n_qubits, n + (int64_t)anti, true, st);
    {
        StageScope ss(ST_RAW, st);
        note_launch(ST_RAW);
        k_rot_copy<WP><<<grid, 256, 0, st>>>(s->keys, s->coef, s->phase, flags.as<uint8_t>(), n, std::cos(theta),
                                             raw->keys, raw->coef, raw->phase, raw->pbase);
        if (anti) {
            note_launch(ST_RAW);
            k_rot_partner<WP><<<std::max<uint32_t>(1, std::min<uint32_t>(nch, (uint32_t)sms * 8)), kChunkThreads, 0,
                                st>>>(nch, flags.as<uint8_t>(), coff.as<uint64_t>(), s->keys, s->coef, s->pbase,
                                      pk.as<uint64_t>(), p_pb, n, std::sin(theta), raw->keys, raw->coef, raw->phase,
                                      raw->pbase);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            sum_free(raw, st);
            check_cuda(e, "rotation kernels");
        }
    }
    if (s->is_canonical && anti > 0) {
        // canonical input: the Q part is sorted and duplicate-free already;
        // canonicalise only the partners (a view of raw's tail), then merge
        paulib_sum pv = *raw;
        pv.n_terms = (int64_t)anti;
        pv.keys = raw->keys + (size_t)n * NW;
        pv.coef = raw->coef + n;
        pv.pbase = raw->pbase + n;
        pv.phase = raw->phase + n;
        pv.is_canonical = 0;
        pv.block = nullptr;
        pv.plan_owned = true;
        paulib_sum* pc = nullptr;
        paulib_sum* out = nullptr;
        try {
            pc = canon_terms(&pv, mode, st);
            out = merge_rotated<WP>(raw, n, pc, threshold, st);
        } catch (...) {
            if (pc) sum_free(pc, st);
            sum_free(raw, st);
            throw;
        }
        sum_free(pc, st);
        sum_free(raw, st);
        return out;
    }
    paulib_sum* canon = nullptr;
    try {
        canon = canon_terms(raw, mode, st);
    } catch (...) {
        sum_free(raw, st);
        throw;
    }
    sum_free(raw, st);
    if (!(threshold > 0) || canon->n_terms == 0) return canon;
    // truncation: drop merged terms with |c| < threshold
    const int64_t u = canon->n_terms;
    const uint32_t nch2 = (uint32_t)((u + kChunk - 1) / kChunk);
    Scratch tflags((size_t)nch2 * kChunk, st), tcoff;
    check_cuda(cudaMemsetAsync(tflags.p, 0, (size_t)nch2 * kChunk, st), "memset flags");
    k_trunc_flags<WP><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((u + 255) / 256, (int64_t)sms * 8)), 256, 0,
                        st>>>(canon->coef, u, threshold * threshold, tflags.as<uint8_t>());
    note_launch(ST_COMPACT);
    const uint64_t keep = flag_offsets(tflags.as<uint8_t>(), nch2, tcoff, st);
    if (keep == (uint64_t)u) return canon;
    paulib_sum* out = sum_alloc(s->n_qubits, (int64_t)keep, false, st);
    out->is_canonical = 1;
    if (keep > 0) {
        StageScope ss(ST_COMPACT, st);
        note_launch(ST_COMPACT);
        k_compact<WP><<<std::max<uint32_t>(1, std::min<uint32_t>(nch2, (uint32_t)sms * 8)), kChunkThreads, 0, st>>>(
            nch2, tflags.as<uint8_t>(), tcoff.as<uint64_t>(), canon->keys, canon->coef, out->keys, out->coef,
            out->pbase);
    }
    cudaError_t e = cudaGetLastError();
    sum_free(canon, st);
    if (e != cudaSuccess) {
        sum_free(out, st);
        check_cuda(e, "truncation");
    }
    return out;
}

paulib_sum* rotate(const paulib_sum* s, const uint64_t* pk_host, double theta, double threshold, int mode,
                   cudaStream_t st) {
    if (s->n_terms == 0) return empty_canonical(s->n_qubits, st);
#define L(WPv) return rotate_wp<WPv>(s, pk_host, theta, threshold, mode, st)
    PAULIB_DISPATCH_WP(s->WP, L);
#undef L
    return nullptr;
}

}  // namespace paulib
