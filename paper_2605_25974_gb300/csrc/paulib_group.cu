// paulib_group.cu -- greedy commutation grouping (PauLIB Sec. V-D; the
// sequential variant of Sec. IV-C) of a device sum.
//
// The result is the first-fit partition: the terms are visited in their order
// and each joins the first group (in the order groups were opened) all of whose
// members commute with it, or opens a new group.  Two strings commute when
// their symplectic inner product <x1,z2> + <z1,x2> is even (Sec. III-F).
// Equivalently, a term's group is the smallest index not taken by an earlier
// term that anti-commutes with it: first-fit colouring of the
// anti-commutation graph in term order.  The kernels compute exactly that:
//
//   k_anticomm  the strict upper triangle of the anti-commutation matrix as
//               bits.  Column word w covers the terms u = 64w .. 64w+63; its
//               rows s < 64w+64 are stored contiguously from word 32w(w+1)
//               (column-word-major, packed), one thread per (s, w).  A pair
//               costs 2*WP ANDs, 2*WP XORs and one popcount: the GF(2) inner
//               product of 64-bit words, with no tensor-core form worth having
//               (there is no 1-bit tcgen05 kind, and a 0/1 bf16 expansion
//               would spend 2n flops on what 2n/64 word operations do).
//   k_greedy    one CTA walks the terms in blocks of 64.  For block b it holds,
//               per group g, the mask N[g] of the block's terms that
//               anti-commute with some member of g (the OR of the column-b
//               words of g's members), transposes the masks into per-term
//               availability rows over groups with warp ballots, and keeps each
//               term's first few available groups.  One warp then decides the
//               64 terms in order, a lane per term: a term takes its first
//               candidate (or new group) not taken by an earlier anti-commuting
//               term of the block (the diagonal matrix words); its choice is
//               broadcast with a shuffle and the later terms mark it taken.
//               Meanwhile the other warps OR the column-(b+1) words of every
//               earlier term into the masks of block b+1.  At most 64 groups
//               open per block, so the masks need room for the G groups so far
//               plus 64.
//   k_group_csr the members of each group in term order (optional).
#include <atomic>
#include <climits>
#include <type_traits>

#include "paulib_pipeline.cuh"

namespace paulib {

constexpr int kAntiThreads = 256;
constexpr int kGreedyThreads = 1024;
constexpr int kGroupCands = 4;  // most available groups a term keeps at its block's start
constexpr int kCsrThreads = 1024;
constexpr int kMaxRowWordsPerLane = 16;  // availability row of 32*16 words: 32,768 groups

__host__ __device__ __forceinline__ int64_t anti_col_offset(int64_t w) { return 32 * w * (w + 1); }

template <int WP>
__global__ void __launch_bounds__(kAntiThreads) k_anticomm(const uint64_t* __restrict__ keys, int64_t m,
                                                           uint64_t* __restrict__ at) {
    constexpr int NW = 2 * WP;
    __shared__ uint64_t su[64 * NW];  // the 64 terms of this column word, as stored (x words, then z)
    const int64_t w = blockIdx.y;
    const int64_t u0 = w * 64;
    const int64_t s0 = (int64_t)blockIdx.x * kAntiThreads;
    if (s0 >= u0 + 64 || s0 >= m) return;  // whole CTA at or below the diagonal block: nothing stored
    const int nu = (int)(m - u0 < 64 ? m - u0 : 64);
    for (int i = threadIdx.x; i < nu * NW; i += kAntiThreads) su[i] = __ldg(keys + u0 * NW + i);
    __syncthreads();
    const int64_t s = s0 + threadIdx.x;
    if (s >= m || s >= u0 + 64) return;
    uint64_t k[NW];
    key_load_g<NW>(keys, (uint64_t)s, k);
    uint64_t word = 0;
    for (int j = s >= u0 ? (int)(s - u0) + 1 : 0; j < nu; ++j) {
        const uint64_t* ku = su + j * NW;
        uint64_t acc = 0;
#pragma unroll
        for (int q = 0; q < WP; ++q) acc ^= (k[q] & ku[WP + q]) ^ (k[WP + q] & ku[q]);
        word |= (uint64_t)(__popcll(acc) & 1) << j;
    }
    at[anti_col_offset(w) + s] = word;
}

// meta[0] receives the number of groups, meta[1] is set when a block would
// need more than 64 * 32 * RMAX groups.  kc (1..kGroupCands): candidates a
// term keeps; any value gives the same partition.  MASKS_SMEM / AVAIL_SMEM:
// the group masks (2 x GC words) and the availability rows (64 x AVS words)
// live in shared memory, else in the global buffers g_masks / g_avail.
//
// Per block: (A1) the masks of the groups opened so far are transposed into
// one availability row per term; (A2) each row yields the term's first
// kGroupCands available groups (and whether there are more); (B) one warp
// decides the terms in order, lane l holding terms l and l+32: a term's
// choice is its first candidate not taken by an earlier anti-commuting term
// of the block, else the first new group not taken by one; the owner's
// choice is broadcast with one shuffle and every later term that
// anti-commutes with it marks that group blocked.  A term whose candidates
// are all blocked while it has more scans its whole row (rare).
template <int RMAX, bool MASKS_SMEM, bool AVAIL_SMEM>
__global__ void __launch_bounds__(kGreedyThreads, 1)
    k_greedy(const uint64_t* __restrict__ at, int32_t m, int32_t* group, int32_t* meta, uint64_t* g_masks,
             uint64_t* g_avail, int kc) {
    constexpr int GW = 32 * RMAX;  // words per availability row
    constexpr int AVS = GW + 1;    // row stride (odd: rows fall in different banks)
    constexpr int GC = 64 * GW;    // group capacity
    constexpr int K = kGroupCands;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ uint64_t g_smem[];
    __shared__ uint64_t s_diag[64];  // row words (bits j > i) of the block's own terms in column b
    __shared__ int32_t s_cand[64][K];
    __shared__ int32_t s_ncand[64];  // existing candidates found, kc + 1 meaning more than kc
    __shared__ int s_groups;
    uint64_t* masks;
    uint64_t* avail;
    if constexpr (MASKS_SMEM) masks = g_smem;
    else masks = g_masks;
    if constexpr (AVAIL_SMEM) avail = g_smem + (MASKS_SMEM ? 2 * GC : 0);
    else avail = g_avail;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nwarps = kGreedyThreads / 32;
    const int nblocks = (m + 63) >> 6;
    for (int i = tid; i < 2 * GC; i += kGreedyThreads) masks[i] = 0ull;
    if (tid == 0) {
        s_groups = 0;
        meta[0] = 0;
        meta[1] = 0;
    }
    __syncthreads();
    uint64_t* ncur = masks;       // masks of block b (complete)
    uint64_t* nnxt = masks + GC;  // masks of block b+1 (being accumulated)
    for (int b = 0; b < nblocks; ++b) {
        const int t0 = b << 6;
        const int nb = min(64, m - t0);
        const int g0 = s_groups;  // groups opened before this block
        if (g0 + 64 > GC) {       // uniform: every thread read the same count
            if (tid == 0) meta[1] = 1;
            return;
        }
        const int wx = (g0 + 63) >> 6;  // row words holding the existing groups
        // (A1) bit g of row i: group g (< g0) has no member that anti-commutes
        // with term t0+i
        uint32_t* av32 = reinterpret_cast<uint32_t*>(avail);
        for (int task = warp; task < 2 * wx; task += nwarps) {
            const int w = task >> 1, h = task & 1;
            const int g = 64 * w + 32 * h + lane;
            const uint64_t nm = g < g0 ? ncur[g] : ~0ull;
            uint32_t lo = 0, hi = 0;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const uint32_t b0 = __ballot_sync(FULL, !((nm >> i) & 1ull));
                const uint32_t b1 = __ballot_sync(FULL, !((nm >> (i + 32)) & 1ull));
                if (lane == i) { lo = b0; hi = b1; }
            }
            av32[2 * (lane * AVS + w) + h] = lo;
            av32[2 * ((lane + 32) * AVS + w) + h] = hi;
        }
        const uint64_t* col = at + anti_col_offset(b);
        if (tid < nb) s_diag[tid] = col[t0 + tid];
        __syncthreads();
        // (A2) each term's first kc available groups (and whether it has more):
        // word popcounts, a warp scan of them, and the lanes whose words hold
        // candidates 0..kc-1 extract those bits
        for (int i = warp; i < nb; i += nwarps) {
            int found = 0;
            for (int w0 = 0; w0 < wx && found <= kc; w0 += 32) {
                const int w = w0 + lane;
                uint64_t word = w < wx ? avail[i * AVS + w] : 0ull;
                const int cnt = __popcll(word);
                int inc = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(FULL, inc, o);
                    if (lane >= o) inc += v;
                }
                int slot = found + inc - cnt;
                while (word && slot < kc) {
                    s_cand[i][slot++] = w * 64 + __ffsll((long long)word) - 1;
                    word &= word - 1ull;
                }
                found += __shfl_sync(FULL, inc, 31);
            }
            if (lane == 0) s_ncand[i] = min(found, kc + 1);
        }
        const bool has_next = b + 1 < nblocks;
        const uint64_t* ncol = at + anti_col_offset(b + 1);
        __syncthreads();
        if (warp == 0) {
            // lane state for its terms t = lane (slot 0) and lane + 32 (slot 1):
            // candidates c0..c3 (INT_MAX: none) with the untaken ones as bits of
            // fr, taken new groups nblk (bit k: group g0 + k), and the current
            // choice cur: a group id, -1 for the lowest untaken new group (one-hot
            // in noh), -2 when the row must be scanned.  The per-term chain uses
            // only shuffles, compares, selects and adds: find-first-set and
            // popcount cost tens of cycles each and stay off it.
            int c0[2], c1[2], c2[2], c3[2], cur[2], fin[2];
            uint32_t fr[2];
            bool more[2];
            uint64_t nblk[2], noh[2], foh[2], drow[2], a[2];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int t = lane + 32 * s;
                const bool on = t < nb;
                const int nc = on ? s_ncand[t] : 0;
                const int kk = min(nc, kc);
                c0[s] = kk > 0 ? s_cand[t][0] : INT_MAX;
                c1[s] = kk > 1 ? s_cand[t][1] : INT_MAX;
                c2[s] = kk > 2 ? s_cand[t][2] : INT_MAX;
                c3[s] = kk > 3 ? s_cand[t][3] : INT_MAX;
                fr[s] = (1u << kk) - 1u;
                more[s] = nc > kc;
                nblk[s] = 0ull;
                noh[s] = 1ull;
                cur[s] = kk > 0 ? c0[s] : (more[s] ? -2 : -1);
                fin[s] = 0;
                foh[s] = 0ull;
                drow[s] = on ? s_diag[t] : 0ull;
                a[s] = on && has_next ? ncol[t0 + t] : 0ull;
            }
            // term i chose (g, oh): g a group id, or -1 with oh the new group's bit.
            // Record it; the later terms that anti-commute with term i (an*) lose
            // it and recompute their choice.  Selects only, no branches.
            auto apply = [&](auto both, int i, int g, uint64_t oh, bool an0, bool an1) {
                const bool mine = lane == (i & 31);
                fin[0] = mine && i < 32 ? g : fin[0];
                foh[0] = mine && i < 32 ? oh : foh[0];
                fin[1] = mine && i >= 32 ? g : fin[1];
                foh[1] = mine && i >= 32 ? oh : foh[1];
#pragma unroll
                for (int s = decltype(both)::value ? 0 : 1; s < 2; ++s) {
                    const bool an = s ? an1 : an0;
                    const uint32_t hit = (uint32_t)(c0[s] == g) | ((uint32_t)(c1[s] == g) << 1) |
                                         ((uint32_t)(c2[s] == g) << 2) | ((uint32_t)(c3[s] == g) << 3);
                    fr[s] &= an ? ~hit : ~0u;
                    nblk[s] |= an ? oh : 0ull;
                    noh[s] = ~nblk[s] & (nblk[s] + 1ull);
                    const uint32_t f = fr[s];
                    const int c = (f & 1u) ? c0[s] : (f & 2u) ? c1[s] : (f & 4u) ? c2[s] : c3[s];
                    cur[s] = f ? c : (more[s] ? -2 : -1);
                }
            };
            auto anti = [&](int i, bool& an0, bool& an1) {
                const uint64_t d = s_diag[i];
                an0 = (uint32_t)(d >> lane) & 1u;
                an1 = (uint32_t)(d >> 32 >> lane) & 1u;
            };
            int i = 0;
            while (i < nb) {
                // the hot loops: the owner's choice by shuffle, then the update
                bool an0, an1;
                anti(i, an0, an1);
                for (; i < min(nb, 32); ++i) {
                    const int g = __shfl_sync(FULL, cur[0], i);
                    const uint32_t ohl = __shfl_sync(FULL, (uint32_t)noh[0], i);
                    const uint32_t ohh = __shfl_sync(FULL, (uint32_t)(noh[0] >> 32), i);
                    if (g == -2) break;
                    bool n0, n1;
                    anti(i + 1 < nb ? i + 1 : i, n0, n1);
                    apply(std::true_type(), i, g, g < 0 ? ((uint64_t)ohh << 32 | ohl) : 0ull, an0, an1);
                    an0 = n0;
                    an1 = n1;
                }
                if (i >= 32 || i == nb) {
                    for (; i < nb; ++i) {
                        const int g = __shfl_sync(FULL, cur[1], i & 31);
                        const uint32_t ohl = __shfl_sync(FULL, (uint32_t)noh[1], i & 31);
                        const uint32_t ohh = __shfl_sync(FULL, (uint32_t)(noh[1] >> 32), i & 31);
                        if (g == -2) break;
                        bool n0, n1;
                        anti(i + 1 < nb ? i + 1 : i, n0, n1);
                        apply(std::false_type(), i, g, g < 0 ? ((uint64_t)ohh << 32 | ohl) : 0ull, an0, an1);
                        an0 = n0;
                        an1 = n1;
                    }
                }
                if (i < nb) {
                    // every kept candidate of term i is taken: clear from its row the
                    // groups chosen by earlier anti-commuting terms, take the first left
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        const int j = lane + 32 * s;
                        if (j < i && ((drow[s] >> i) & 1ull) && fin[s] >= 0)
                            atomicAnd(reinterpret_cast<unsigned long long*>(avail + i * AVS + (fin[s] >> 6)),
                                      ~(1ull << (fin[s] & 63)));
                    }
                    __syncwarp();
                    int g = -1;
                    for (int w0 = 0; w0 < wx && g < 0; w0 += 32) {
                        const uint64_t word = w0 + lane < wx ? avail[i * AVS + w0 + lane] : 0ull;
                        const uint32_t bal = __ballot_sync(FULL, word != 0ull);
                        if (bal) {
                            const int fl = __ffs(bal) - 1;
                            const uint64_t v = __shfl_sync(FULL, word, fl);
                            g = (w0 + fl) * 64 + __ffsll((long long)v) - 1;
                        }
                    }
                    const uint64_t oh = __shfl_sync(FULL, i >= 32 ? noh[1] : noh[0], i & 31);
                    anti(i, an0, an1);
                    if (i < 32) apply(std::true_type(), i, g, g < 0 ? oh : 0ull, an0, an1);
                    else apply(std::false_type(), i, g, g < 0 ? oh : 0ull, an0, an1);
                    ++i;
                }
            }
            // the block's results (new groups numbered from their bits), and their
            // words of column b+1 into the next masks
            int top = g0 - 1;
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int t = lane + 32 * s;
                if (t < nb) {
                    const int gf = fin[s] >= 0 ? fin[s] : g0 + __ffsll((long long)foh[s]) - 1;
                    top = max(top, gf);
                    group[t0 + t] = gf;
                    if (a[s]) atomicOr(reinterpret_cast<unsigned long long*>(nnxt + gf), (unsigned long long)a[s]);
                }
            }
            top = __reduce_max_sync(FULL, top);
            if (lane == 0) s_groups = top + 1;
        } else {
            // meanwhile: the masks just transposed become block b+2's accumulator
            // (cleared), and every earlier term's column-(b+1) word goes into its
            // group's mask for block b+1
            const int ht = tid - 32, hn = kGreedyThreads - 32;
            for (int g = ht; g < g0; g += hn) ncur[g] = 0ull;
            if (has_next) {  // four independent loads in flight per thread
                int s = ht;
                for (; s + 3 * hn < t0; s += 4 * hn) {
                    uint64_t av[4];
                    int32_t gs[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        av[u] = ncol[s + u * hn];
                        gs[u] = __ldcg(group + s + u * hn);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (av[u]) atomicOr(reinterpret_cast<unsigned long long*>(nnxt + gs[u]), (unsigned long long)av[u]);
                }
                for (; s < t0; s += hn) {
                    const uint64_t v = ncol[s];
                    if (v) atomicOr(reinterpret_cast<unsigned long long*>(nnxt + __ldcg(group + s)), (unsigned long long)v);
                }
            }
        }
        __syncthreads();
        uint64_t* tmp = ncur;
        ncur = nnxt;
        nnxt = tmp;
    }
    if (tid == 0) meta[0] = s_groups;
}

// offsets[g] = first member slot of group g (offsets[G] = m, G = meta[0]);
// members lists each group's terms in increasing order.  Nothing is written
// when meta[1] reports an overflow.
__global__ void __launch_bounds__(kCsrThreads, 1)
    k_group_csr(const int32_t* __restrict__ group, int32_t m, const int32_t* __restrict__ meta, int32_t* offsets,
                int32_t* members) {
    extern __shared__ int32_t cursor[];  // [ngroups]
    if (meta[1]) return;
    const int32_t ngroups = meta[0];
    __shared__ int32_t s_warp[kCsrThreads / 32];
    constexpr unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int g = tid; g < ngroups; g += kCsrThreads) cursor[g] = 0;
    __syncthreads();
    for (int t = tid; t < m; t += kCsrThreads) atomicAdd(cursor + __ldg(group + t), 1);
    __syncthreads();
    // exclusive scan: thread tid owns groups [tid*per, (tid+1)*per)
    const int per = (ngroups + kCsrThreads - 1) / kCsrThreads;
    const int lo = min(ngroups, tid * per), hi = min(ngroups, lo + per);
    int32_t own = 0;
    for (int g = lo; g < hi; ++g) own += cursor[g];
    int32_t inc = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t v = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int32_t v = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t u = __shfl_up_sync(FULL, v, o);
            if (lane >= o) v += u;
        }
        s_warp[lane] = v;  // inclusive over warps
    }
    __syncthreads();
    int32_t run = inc - own + (warp ? s_warp[warp - 1] : 0);
    for (int g = lo; g < hi; ++g) {
        const int32_t c = cursor[g];
        if (offsets) offsets[g] = run;
        cursor[g] = run;
        run += c;
    }
    if (tid == 0 && offsets) offsets[ngroups] = m;
    __syncthreads();
    if (!members || warp != 0) return;
    for (int c = 0; c < m; c += 32) {
        const int t = c + lane;
        const int g = t < m ? __ldg(group + t) : -1;
        const unsigned peers = __match_any_sync(FULL, g);
        const int leader = __ffs(peers) - 1;
        const int rank = __popc(peers & ((1u << lane) - 1u));
        int base = (lane == leader && g >= 0) ? cursor[g] : 0;
        base = __shfl_sync(FULL, base, leader);
        if (g >= 0) members[base + rank] = t;
        __syncwarp();
        if (lane == leader && g >= 0) cursor[g] = base + __popc(peers);
        __syncwarp();
    }
}

static std::atomic<int> g_group_cands{kGroupCands};

// Raises a kernel's dynamic shared-memory limit once per device.
template <class F>
static void set_smem_once(F* kern, size_t bytes, std::atomic<uint64_t>& done) {
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "device");
    const uint64_t bit = 1ull << (dev & 63);
    if (done.load() & bit) return;
    check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes), "attr");
    done.fetch_or(bit);
}

void set_group_cands(int k) { g_group_cands.store(k); }
static int group_cands() { return g_group_cands.load(); }

template <int RMAX>
static void launch_greedy(const uint64_t* at, int32_t m, int32_t* group, int32_t* meta, cudaStream_t st,
                          std::vector<Scratch>& keep) {
    constexpr int GW = 32 * RMAX, AVS = GW + 1, GC = 64 * GW;
    constexpr bool masks_in_smem = RMAX <= 4, avail_in_smem = RMAX <= 8;
    const size_t smem = (masks_in_smem ? (size_t)2 * GC * 8 : 0) + (avail_in_smem ? (size_t)64 * AVS * 8 : 0);
    keep.emplace_back(masks_in_smem ? 0 : (size_t)2 * GC * 8, st);
    uint64_t* gm = keep.back().as<uint64_t>();
    keep.emplace_back(avail_in_smem ? 0 : (size_t)64 * AVS * 8, st);
    uint64_t* ga = keep.back().as<uint64_t>();
    auto kern = k_greedy<RMAX, masks_in_smem, avail_in_smem>;
    static std::atomic<uint64_t> attr_set{0};  // devices whose attribute is set
    set_smem_once(kern, smem, attr_set);
    note_launch(ST_GROUP);
    kern<<<1, kGreedyThreads, smem, st>>>(at, m, group, meta, gm, ga, group_cands());
    check_cuda(cudaGetLastError(), "k_greedy");
}

int64_t group_commuting(const paulib_sum* s, int32_t* group, int32_t* offsets, int32_t* members, cudaStream_t st) {
    const int64_t m = s->n_terms;
    if (m == 0) {
        if (offsets) check_cuda(cudaMemsetAsync(offsets, 0, sizeof(int32_t), st), "offsets");
        check_cuda(cudaStreamSynchronize(st), "group sync");
        return 0;
    }
    const int64_t nblocks = (m + 63) / 64;
    if (m > INT32_MAX || nblocks > 65535) fail(PAULIB_ERR_UNSUPPORTED, "grouping supports at most 4,194,240 terms");
    StageScope ss(ST_GROUP, st);
    // one allocation: the greedy kernel's two result words, then the bit matrix
    Scratch blockmem(256 + (size_t)anti_col_offset(nblocks) * sizeof(uint64_t), st);
    int32_t* meta = blockmem.as<int32_t>();
    uint64_t* atm = reinterpret_cast<uint64_t*>(blockmem.as<char>() + 256);
    {
        const dim3 grid((unsigned)((m + kAntiThreads - 1) / kAntiThreads), (unsigned)nblocks);
        note_launch(ST_GROUP);
#define L(WPv) k_anticomm<WPv><<<grid, kAntiThreads, 0, st>>>(s->keys, m, atm);
        PAULIB_DISPATCH_WP(s->WP, L);
#undef L
        check_cuda(cudaGetLastError(), "k_anticomm");
    }
    int rmax = 1;  // smallest row that holds every group m terms can open, plus 64
    while (rmax < kMaxRowWordsPerLane && m + 64 > (int64_t)2048 * rmax) rmax *= 2;
    std::vector<Scratch> keep;
    keep.reserve(2);
    const int32_t mi = (int32_t)m;
    switch (rmax) {
        case 1: launch_greedy<1>(atm, mi, group, meta, st, keep); break;
        case 2: launch_greedy<2>(atm, mi, group, meta, st, keep); break;
        case 4: launch_greedy<4>(atm, mi, group, meta, st, keep); break;
        case 8: launch_greedy<8>(atm, mi, group, meta, st, keep); break;
        default: launch_greedy<16>(atm, mi, group, meta, st, keep); break;
    }
    if (offsets || members) {
        // sized for every partition the greedy kernel can return: G <= min(m, 32,704)
        const size_t smem = (size_t)std::min<int64_t>(m, 64 * 32 * kMaxRowWordsPerLane - 64) * sizeof(int32_t);
        static std::atomic<uint64_t> attr_set{0};
        set_smem_once(k_group_csr, (size_t)(64 * 32 * kMaxRowWordsPerLane - 64) * sizeof(int32_t), attr_set);
        note_launch(ST_GROUP);
        k_group_csr<<<1, kCsrThreads, smem, st>>>(group, mi, meta, offsets, members);
        check_cuda(cudaGetLastError(), "k_group_csr");
    }
    int32_t h[2] = {0, 0};
    check_cuda(cudaMemcpyAsync(h, meta, sizeof(h), cudaMemcpyDeviceToHost, st), "group count");
    check_cuda(cudaStreamSynchronize(st), "group sync");
    if (h[1]) fail(PAULIB_ERR_UNSUPPORTED, "the partition needs more than 32,704 groups");
    return h[0];
}

}  // namespace paulib
