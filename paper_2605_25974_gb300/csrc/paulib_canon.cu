// paulib_canon.cu -- canonical product of two sums (paulib_multiply with
// PAULIB_OUT_CANONICAL) and the allocation-free variant; the pipeline itself
// is in paulib_pipeline.cuh.
#include "paulib_slots.cuh"

namespace paulib {

paulib_sum* canon_product(const paulib_sum* a, const paulib_sum* b, int mode, cudaStream_t st) {
    const int64_t R = a->n_terms * b->n_terms;
    if (R == 0) return empty_canonical(a->n_qubits, st);
    if (R >= ((int64_t)1 << 32) - 1)
        fail(PAULIB_ERR_UNSUPPORTED, "canonical product needs |A|*|B| < 2^32, got " + std::to_string(R));
#define L(WP)                                                          \
    {                                                                  \
        if (mode == M_FP64) return product_mode<WP, M_FP64>(a, b, st); \
        if (mode == M_F32_D64) return product_mode<WP, M_F32_D64>(a, b, st); \
        return product_mode<WP, M_F32_TWOSUM>(a, b, st);               \
    }
    PAULIB_DISPATCH_WP(a->WP, L);
#undef L
    return nullptr;
}

// ---------------------------------------------------------------- allocation-free product
//
// For callers that cannot let the library allocate device memory (their
// memory belongs to their own pool or fixed budget), paulib_multiply_noalloc
// runs the canonical product on a fixed scratch area compiled into this
// file.  Layout (bytes, each part a multiple of 256): both operands in the
// packed key form for up to 16384 terms of up to 256 qubits, the record and
// staging arrays for up to 65536 products, one worklist stack and the
// splitter scratch of one range CTA, the output flags and leaf lists, and a
// few counters.

namespace na {
constexpr size_t kTerms = PAULIB_NOALLOC_MAX_TERMS;
constexpr size_t kProducts = PAULIB_NOALLOC_MAX_PRODUCTS;
constexpr size_t kKeyBytes = 2 * 4 * 8;  // up to 4 words per half (256 qubits)
constexpr size_t kOffAK = 0;
constexpr size_t kOffAC = kOffAK + kTerms * kKeyBytes;
constexpr size_t kOffAP = kOffAC + kTerms * 16;
constexpr size_t kOffBK = kOffAP + kTerms;
constexpr size_t kOffBC = kOffBK + kTerms * kKeyBytes;
constexpr size_t kOffBP = kOffBC + kTerms * 16;
constexpr size_t kOffRecA = kOffBP + kTerms;
constexpr size_t kOffRecB = kOffRecA + kProducts * 4;
constexpr size_t kOffSub = kOffRecB + kProducts * 4;
constexpr size_t kOffTK = kOffSub + kProducts * 2;
constexpr size_t kOffTC = kOffTK + kProducts * kKeyBytes;
constexpr size_t kOffStack = kOffTC + kProducts * 16;
constexpr size_t kOffSpl = kOffStack + (size_t)kStackCap * sizeof(StackEnt);
constexpr size_t kSplBytes = 32768;  // (leaf capacity / 2) splitters of one CTA, largest case
constexpr size_t kOffFlag = kOffSpl + kSplBytes;
constexpr size_t kSmallCap = kProducts / 2 + 1;  // warp leaves hold >= 2 records
constexpr size_t kMedCap = kProducts / 33 + 1;   // block leaves hold more than a warp leaf (>= 32)
constexpr size_t kOffList = kOffFlag + kProducts;
constexpr size_t kOffMisc = kOffList + (((kSmallCap + kMedCap) * 8 + 255) & ~(size_t)255);
constexpr size_t kBytes = kOffMisc + 512;
static_assert(kBytes == PAULIB_NOALLOC_SCRATCH_BYTES, "scratch size must match the header");
static_assert(kOffAC % 256 == 0 && kOffAP % 256 == 0 && kOffBK % 256 == 0 && kOffRecA % 256 == 0 &&
                  kOffSub % 256 == 0 && kOffTK % 256 == 0 && kOffStack % 256 == 0 && kOffFlag % 256 == 0 &&
                  kOffList % 256 == 0 && kOffMisc % 256 == 0,
              "scratch parts stay 256-byte aligned");
}  // namespace na

static __device__ __align__(256) unsigned char g_noalloc_scratch[na::kBytes];

template <int WP>
__global__ void k_na_convert(int64_t n, int W, int nq, const uint64_t* __restrict__ xs,
                             const uint64_t* __restrict__ zs, const double2* __restrict__ cs, uint64_t* keys,
                             double2* coef, uint8_t* pbase, int32_t* err) {
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
            if (w == W - 1 && ((x | z) & tail_mask)) atomicOr(err, 8);
        }
        k[w] = x;
        k[WP + w] = z;
    }
    key_store<2 * WP>(keys, (uint64_t)t, k);
    coef[t] = cs[t];
    pbase[t] = (uint8_t)normal_phase<WP>(k, 0u);
}

template <int WP>
__global__ void __launch_bounds__(kChunkThreads) k_na_output(int W, uint32_t nch, const uint8_t* __restrict__ oflag,
                                                           const uint64_t* __restrict__ coff,
                                                           const uint64_t* __restrict__ Tkeys,
                                                           const double2* __restrict__ Tcoef, uint64_t* ox,
                                                           uint64_t* oz, double2* oc, int64_t cap, int64_t* out_n) {
    __shared__ uint32_t s_warp[32];
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
        for_each_flagged(c, oflag, coff, s_warp, [&](uint64_t p, uint64_t d) {
            uint64_t k[2 * WP];
            key_load_g<2 * WP>(Tkeys, p, k);
            for (int w = 0; w < W; ++w) {
                ox[(uint64_t)w * cap + d] = k[w];
                oz[(uint64_t)w * cap + d] = k[WP + w];
            }
            oc[d] = Tcoef[p];
        });
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *out_n = (int64_t)coff[nch];
}

static std::mutex g_na_mu;
static unsigned char* g_na_base[64] = {};

// Device address of the scratch array on the current device, looked up once
// per device with that device current.
static unsigned char* noalloc_base() {
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= 64) fail(PAULIB_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_base[dev]) {
        void* p = nullptr;
        check_cuda(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(scratch)");
        g_na_base[dev] = static_cast<unsigned char*>(p);
    }
    return g_na_base[dev];
}

template <int WP>
static void noalloc_run(int32_t n_qubits, int64_t na_, const uint64_t* a_x, const uint64_t* a_z, const double* a_c,
                        int64_t nb_, const uint64_t* b_x, const uint64_t* b_z, const double* b_c, uint64_t* out_x,
                        uint64_t* out_z, double* out_c, int64_t cap, int64_t* out_n, cudaStream_t st) {
    using Src = ProdSrc<WP, M_FP64>;
    using Cfg = L2Cfg<Src, M_FP64>;
    constexpr int NW = 2 * WP;
    static_assert((size_t)(Cfg::CAP / 2) * NW * 8 <= na::kSplBytes, "splitter scratch too small");
    unsigned char* base = noalloc_base();
    uint64_t* ak = reinterpret_cast<uint64_t*>(base + na::kOffAK);
    double2* ac = reinterpret_cast<double2*>(base + na::kOffAC);
    uint8_t* ap = base + na::kOffAP;
    uint64_t* bk = reinterpret_cast<uint64_t*>(base + na::kOffBK);
    double2* bc = reinterpret_cast<double2*>(base + na::kOffBC);
    uint8_t* bp = base + na::kOffBP;
    uint32_t* recA = reinterpret_cast<uint32_t*>(base + na::kOffRecA);
    uint32_t* recB = reinterpret_cast<uint32_t*>(base + na::kOffRecB);
    uint16_t* sub = reinterpret_cast<uint16_t*>(base + na::kOffSub);
    uint64_t* tk = reinterpret_cast<uint64_t*>(base + na::kOffTK);
    double2* tc = reinterpret_cast<double2*>(base + na::kOffTC);
    StackEnt* stack = reinterpret_cast<StackEnt*>(base + na::kOffStack);
    uint64_t* spl = reinterpret_cast<uint64_t*>(base + na::kOffSpl);
    uint8_t* oflag = base + na::kOffFlag;
    uint2* lists = reinterpret_cast<uint2*>(base + na::kOffList);
    unsigned char* misc = base + na::kOffMisc;
    uint64_t* boff = reinterpret_cast<uint64_t*>(misc);         // [2]
    uint32_t* ctr = reinterpret_cast<uint32_t*>(misc + 16);     // [4]
    int32_t* err = reinterpret_cast<int32_t*>(misc + 32);
    uint8_t* bflags = misc + 36;                                 // [1]
    uint32_t* ccount = reinterpret_cast<uint32_t*>(misc + 64);  // [8]
    uint64_t* coff = reinterpret_cast<uint64_t*>(misc + 128);   // [9]
    static_assert(na::kProducts / kChunk <= 8, "chunk counters fit the counter block");
    const int W = (n_qubits + 63) / 64;
    const uint32_t R = (uint32_t)(na_ * nb_);
    const uint32_t nch = (R + kChunk - 1) / kChunk;
    // counters and offsets that must start at zero
    check_cuda(cudaMemsetAsync(misc, 0, 512, st), "memset scratch counters");
    if (R > 0) {
        check_cuda(cudaMemsetAsync(oflag, 0, (size_t)nch * kChunk, st), "memset flags");
        k_na_convert<WP><<<(unsigned)((na_ + 255) / 256), 256, 0, st>>>(
            na_, W, n_qubits, a_x, a_z, reinterpret_cast<const double2*>(a_c), ak, ac, ap, err);
        k_na_convert<WP><<<(unsigned)((nb_ + 255) / 256), 256, 0, st>>>(
            nb_, W, n_qubits, b_x, b_z, reinterpret_cast<const double2*>(b_c), bk, bc, bp, err);
        k_iota<<<(R + 255) / 256, 256, 0, st>>>(recA, R, boff, bflags);
        Src src{ak, bk, ap, bp, ac, bc, (uint32_t)na_, 0u, recip64((uint32_t)na_)};
        L2Bufs lb{recA, recB, sub, ctr, stack, spl, tk, tc, oflag, lists, lists + na::kSmallCap,
                  (uint32_t)na::kSmallCap, (uint32_t)na::kMedCap, err};
        launch_level2<Src, M_FP64>(src, 1u, boff, bflags, lb, 1u, nch, ccount, coff, st);
    }
    k_na_output<WP><<<std::max<unsigned>(1, nch), kChunkThreads, 0, st>>>(
        W, nch, oflag, coff, tk, tc, out_x, out_z, reinterpret_cast<double2*>(out_c), cap, out_n);
    check_cuda(cudaGetLastError(), "noalloc launch");
    int32_t h = 0;
    check_cuda(cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, st), "error word copy");
    check_cuda(cudaStreamSynchronize(st), "noalloc sync");
    if (h & 8) fail(PAULIB_ERR_TAIL_BITS, "a bit at qubit >= n_qubits is set in the last word");
    if (h) fail(PAULIB_ERR_INTERNAL, "canonicalisation failed on device (error word " + std::to_string(h) + ")");
}

void multiply_noalloc(int32_t n_qubits, int64_t na_, const uint64_t* a_x, const uint64_t* a_z, const double* a_c,
                      int64_t nb_, const uint64_t* b_x, const uint64_t* b_z, const double* b_c, uint64_t* out_x,
                      uint64_t* out_z, double* out_c, int64_t cap, int64_t* out_n, cudaStream_t st) {
    if (n_qubits < 1) fail(PAULIB_ERR_INVALID_ARG, "n_qubits must be >= 1");
    if (n_qubits > PAULIB_NOALLOC_MAX_QUBITS)
        fail(PAULIB_ERR_UNSUPPORTED, "paulib_multiply_noalloc supports at most 256 qubits, got " +
                                         std::to_string(n_qubits));
    if (na_ < 0 || nb_ < 0) fail(PAULIB_ERR_INVALID_ARG, "negative term count");
    if (na_ > PAULIB_NOALLOC_MAX_TERMS || nb_ > PAULIB_NOALLOC_MAX_TERMS)
        fail(PAULIB_ERR_UNSUPPORTED, "paulib_multiply_noalloc supports at most 16384 terms per operand");
    if (na_ * nb_ > PAULIB_NOALLOC_MAX_PRODUCTS)
        fail(PAULIB_ERR_UNSUPPORTED, "paulib_multiply_noalloc supports at most 65536 products, got " +
                                         std::to_string(na_ * nb_));
    if (cap < na_ * nb_) fail(PAULIB_ERR_INVALID_ARG, "out_capacity must be >= na*nb");
    if (!out_n || (na_ * nb_ > 0 && (!out_x || !out_z || !out_c)))
        fail(PAULIB_ERR_INVALID_ARG, "output pointers must be non-NULL");
    if ((na_ > 0 && (!a_x || !a_z || !a_c)) || (nb_ > 0 && (!b_x || !b_z || !b_c)))
        fail(PAULIB_ERR_INVALID_ARG, "input pointers must be non-NULL");
    const int WP = padded_words((n_qubits + 63) / 64);
#define L(WPv) noalloc_run<WPv>(n_qubits, na_, a_x, a_z, a_c, nb_, b_x, b_z, b_c, out_x, out_z, out_c, cap, out_n, st)
    switch (WP) {
        case 1: L(1); break;
        case 2: L(2); break;
        case 4: L(4); break;
        default: fail(PAULIB_ERR_INTERNAL, "unexpected word count");
    }
#undef L
}

}  // namespace paulib
