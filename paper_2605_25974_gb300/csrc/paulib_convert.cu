// paulib_convert.cu -- layout conversion between the paper's struct-of-arrays
// form (Sec. IV-A, the ABI format) and the library's per-term packed keys,
// plus the raw outer product (Sec. IV-C: every left term times every right
// term, product (i, j) at index j*|A| + i).
#include "paulib_device.cuh"
#include "paulib_internal.h"

namespace paulib {

// ---------------------------------------------------------------- create

template <int WP>
__global__ void __launch_bounds__(256) k_create(int64_t n, int W, int nq, const uint64_t* __restrict__ xs,
                                                const uint64_t* __restrict__ zs,
                                                const double2* __restrict__ cs,
                                                const uint8_t* __restrict__ ph, uint64_t* keys,
                                                double2* coef, uint8_t* pbase, uint8_t* phase,
                                                int32_t* err) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    uint64_t k[2 * WP];
    const int tail = nq & 63;
    const uint64_t tail_mask = tail ? ~((1ull << tail) - 1ull) : 0ull;
#pragma unroll
    for (int w = 0; w < WP; ++w) {
        uint64_t x = 0, z = 0;
        if (w < W) {
            x = xs[(int64_t)w * n + t];
            z = zs[(int64_t)w * n + t];
            if (w == W - 1 && ((x | z) & tail_mask)) atomicOr(err, 1);
        }
        k[w] = x;
        k[WP + w] = z;
    }
    key_store<2 * WP>(keys, (uint64_t)t, k);
    coef[t] = cs[t];
    const uint32_t own = ph ? (ph[t] & 3u) : 0u;
    if (phase) phase[t] = (uint8_t)own;
    pbase[t] = (uint8_t)normal_phase<WP>(k, own);
}

void launch_create(paulib_sum* s, const uint64_t* x_soa, const uint64_t* z_soa, const double* coef,
                   const uint8_t* phase, int32_t* err_flag, cudaStream_t st) {
    const int64_t n = s->n_terms;
    const unsigned grid = (unsigned)((n + 255) / 256);
#define L(WP)                                                                                  \
    k_create<WP><<<grid, 256, 0, st>>>(n, s->W, s->n_qubits, x_soa, z_soa,                     \
                                       reinterpret_cast<const double2*>(coef), phase, s->keys, \
                                       s->coef, s->pbase, s->phase, err_flag)
    StageScope ss(ST_CONVERT, st);
    note_launch(ST_CONVERT);
    PAULIB_DISPATCH_WP(s->WP, L);
#undef L
    check_cuda(cudaGetLastError(), "k_create launch");
}

// ---------------------------------------------------------------- export

template <int WP>
__global__ void __launch_bounds__(256) k_export(int64_t n, int W, const uint64_t* __restrict__ keys,
                                                const double2* __restrict__ coef,
                                                const uint8_t* __restrict__ phase, uint64_t* xs,
                                                uint64_t* zs, double2* cs, uint8_t* ph) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    uint64_t k[2 * WP];
    key_load_g<2 * WP>(keys, (uint64_t)t, k);
#pragma unroll
    for (int w = 0; w < WP; ++w) {
        if (w < W) {
            xs[(int64_t)w * n + t] = k[w];
            zs[(int64_t)w * n + t] = k[WP + w];
        }
    }
    cs[t] = coef[t];
    if (ph) ph[t] = phase ? phase[t] : (uint8_t)0;
}

void launch_export(const paulib_sum* s, uint64_t* x_soa, uint64_t* z_soa, double* coef,
                   uint8_t* phase, cudaStream_t st) {
    const int64_t n = s->n_terms;
    const unsigned grid = (unsigned)((n + 255) / 256);
#define L(WP)                                                                                   \
    k_export<WP><<<grid, 256, 0, st>>>(n, s->W, s->keys, s->coef, s->phase, x_soa, z_soa,       \
                                       reinterpret_cast<double2*>(coef), phase)
    StageScope ss(ST_EXPORT, st);
    note_launch(ST_EXPORT);
    PAULIB_DISPATCH_WP(s->WP, L);
#undef L
    check_cuda(cudaGetLastError(), "k_export launch");
}

// ---------------------------------------------------------------- raw outer product
//
// CTA tile: RA = blockDim.x left terms (one per thread, held in registers)
// times CB right terms staged in shared memory and read as warp broadcasts.
// Consecutive threads own consecutive output indices j*|A| + i.  A warp's 32
// product keys pass through a padded shared buffer and are written as
// contiguous 16-byte pieces (one 512-byte segment per store instruction);
// coefficients and phase bytes are contiguous per warp as they are.
constexpr int kRawThreads = 128;
constexpr int kRawCols = 32;

template <int WP>
__global__ void __launch_bounds__(kRawThreads) k_outer_raw(
    int64_t na, int64_t nb, const uint64_t* __restrict__ ak, const double2* __restrict__ ac,
    const uint8_t* __restrict__ ap, const uint64_t* __restrict__ bk,
    const double2* __restrict__ bc, const uint8_t* __restrict__ bp, uint64_t* ok, double2* oc,
    uint8_t* oph, uint8_t* opb) {
    constexpr int NW = 2 * WP;
    constexpr int KS = NW + 1;  // padded key stride in the staging buffer (words)
    __shared__ __align__(16) uint64_t sk[kRawCols * NW];
    __shared__ double2 sc[kRawCols];
    __shared__ uint32_t sp[kRawCols];
    __shared__ uint64_t stage[kRawThreads / 32][32 * KS];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint64_t* ws = stage[warp];
    const int64_t tiles_i = (na + kRawThreads - 1) / kRawThreads;
    const int64_t tiles_j = (nb + kRawCols - 1) / kRawCols;
    for (int64_t tile = blockIdx.x; tile < tiles_i * tiles_j; tile += gridDim.x) {
        const int64_t ti = tile % tiles_i, tj = tile / tiles_i;
        const int64_t i = ti * kRawThreads + threadIdx.x;
        const int64_t i0 = ti * kRawThreads + warp * 32;  // first row of this warp
        const int64_t j0 = tj * kRawCols;
        const int ncols = (int)mn<int64_t>(kRawCols, nb - j0);
        __syncthreads();
        for (int q = threadIdx.x; q < ncols * NW; q += blockDim.x) sk[q] = bk[j0 * NW + q];
        for (int q = threadIdx.x; q < ncols; q += blockDim.x) {
            sc[q] = bc[j0 + q];
            sp[q] = bp[j0 + q];
        }
        __syncthreads();
        if (i0 >= na) continue;  // the whole warp is past the last row
        const bool live = i < na;
        const uint32_t nrow = (uint32_t)mn<int64_t>(32, na - i0);  // rows of this warp
        uint64_t a[NW];
        double2 ca = make_double2(0.0, 0.0);
        uint32_t pa = 0;
        if (live) {
            key_load_g<NW>(ak, (uint64_t)i, a);
            ca = ac[i];
            pa = ap[i];
        } else {
#pragma unroll
            for (int w = 0; w < NW; ++w) a[w] = 0;
        }
        for (int c = 0; c < ncols; ++c) {
            uint64_t b[NW], o[NW];
            key_load_s<NW>(sk, (uint32_t)c, b);
            const uint32_t k = string_product<WP>(a, b, pa, sp[c], o);
            const int64_t r0 = (j0 + c) * na + i0;  // record of this warp's first row
            // keys: staged per warp, then written as contiguous 16-byte pieces
#pragma unroll
            for (int w = 0; w < NW; ++w) ws[lane * KS + w] = o[w];
            __syncwarp();
            uint64_t* dst = ok + (uint64_t)r0 * NW;
            for (uint32_t q = lane; q < nrow * (NW / 2); q += 32u) {
                const uint32_t row = (2u * q) / NW, wd = (2u * q) % NW;
                reinterpret_cast<ulonglong2*>(dst)[q] = make_ulonglong2(ws[row * KS + wd], ws[row * KS + wd + 1]);
            }
            __syncwarp();
            if (live) {
                const int64_t r = r0 + lane;
                oc[r] = cmul(ca, sc[c]);
                oph[r] = (uint8_t)k;
                opb[r] = (uint8_t)normal_phase<WP>(o, k);
            }
        }
    }
}

void launch_outer_raw(const paulib_sum* a, const paulib_sum* b, paulib_sum* out, cudaStream_t st) {
    const int64_t tiles = ((a->n_terms + kRawThreads - 1) / kRawThreads) *
                          ((b->n_terms + kRawCols - 1) / kRawCols);
    const int64_t maxgrid = (int64_t)device_sm_count() * 16;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, maxgrid));
#define L(WP)                                                                                    \
    k_outer_raw<WP><<<grid, kRawThreads, 0, st>>>(a->n_terms, b->n_terms, a->keys, a->coef,      \
                                                  a->pbase, b->keys, b->coef, b->pbase, out->keys, \
                                                  out->coef, out->phase, out->pbase)
    StageScope ss(ST_RAW, st);
    note_launch(ST_RAW);
    PAULIB_DISPATCH_WP(a->WP, L);
#undef L
    check_cuda(cudaGetLastError(), "k_outer_raw launch");
}

}  // namespace paulib
