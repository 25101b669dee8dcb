// paulib_batch.cu -- batched canonical products and the prepared, graph-
// capturable batch plan; the pipeline is in paulib_pipeline.cuh.
#include "paulib_persist.cuh"

namespace paulib {

// ---------------------------------------------------------------- batched products
//
// Many independent products canonicalised together.  Two methods give the
// same sums:
//   * the persistent kernel (paulib_persist.cuh), when every right operand
//     has at most kPNB terms: one launch, one CTA per problem at a time;
//   * the general pipeline otherwise: problem b's records are the global
//     record range [r0s[b], r0s[b+1]); its products' keys are prefixed by two
//     words (b, 0), so one sort keeps problems apart and emits them in order,
//     and the output of problem b is then copied into its own sum.
// Either way problem b's output sum has capacity |A_b||B_b|.

template <int WP_, int MODE>
struct BatchSrc {
    static constexpr int WP = WP_;
    static constexpr int NW = 2 * WP + 2;
    using V = typename ValT<MODE>::T;
    const ProbDesc* probs;
    const uint32_t* r0s;
    uint32_t nprob;
    // problem of record r: the largest b with r0s[b] <= r (empty problems are skipped)
    __device__ __forceinline__ uint32_t find(uint32_t r) const {
        uint32_t lo = 0, hi = nprob;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(r0s + mid) <= r) lo = mid; else hi = mid;
        }
        return lo;
    }
    __device__ __forceinline__ uint32_t kp(uint32_t r, uint64_t (&k)[NW], bool want_phase) const {
        const uint32_t b = find(r);
        const ProbDesc d = probs[b];
        const uint32_t q = r - __ldg(r0s + b);
        const uint32_t j = q / d.na, i = q - j * d.na;
        uint64_t a[2 * WP], bb[2 * WP], o[2 * WP];
        key_load_g<2 * WP>(d.ak, i, a);
        key_load_g<2 * WP>(d.bk, j, bb);
        uint32_t ph = 0;
        if (want_phase) {
            ph = string_product<WP>(a, bb, __ldg(d.ap + i), __ldg(d.bp + j), o);
        } else {
#pragma unroll
            for (int w = 0; w < 2 * WP; ++w) o[w] = a[w] ^ bb[w];
        }
        k[0] = b;
        k[1] = 0;
#pragma unroll
        for (int w = 0; w < 2 * WP; ++w) k[2 + w] = o[w];
        return ph;
    }
    __device__ __forceinline__ void key(uint32_t r, uint64_t (&k)[NW]) const { kp(r, k, false); }
    __device__ __forceinline__ uint32_t keyphase(uint32_t r, uint64_t (&k)[NW]) const { return kp(r, k, true); }
    __device__ __forceinline__ V coefv(uint32_t r, uint32_t ph) const {
        const uint32_t b = find(r);
        const ProbDesc d = probs[b];
        const uint32_t q = r - __ldg(r0s + b);
        const uint32_t j = q / d.na, i = q - j * d.na;
        return rot_v(mul_v(static_cast<const V*>(d.ac)[i], static_cast<const V*>(d.bc)[j]), ph);
    }
    __device__ __forceinline__ V value(uint32_t r, uint64_t (&k)[NW]) const { return coefv(r, keyphase(r, k)); }
};

// Distinct output strings per problem.  The merged terms are in key order,
// so problems form runs; each thread adds up the runs among its slots.
template <int NW>
__global__ void __launch_bounds__(kChunkThreads) k_batch_counts(uint32_t nch, const uint8_t* __restrict__ oflag,
                                                              const uint64_t* __restrict__ coff,
                                                              const uint64_t* __restrict__ Tkeys,
                                                              unsigned long long* counts) {
    __shared__ uint32_t s_warp[32];
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
        uint64_t run = 0, cur = ~0ull;
        for_each_flagged(c, oflag, coff, s_warp, [&](uint64_t p, uint64_t) {
            const uint64_t b = Tkeys[p * NW];
            if (b != cur) {
                if (run) atomicAdd(&counts[cur], (unsigned long long)run);
                cur = b;
                run = 0;
            }
            ++run;
        });
        if (run) atomicAdd(&counts[cur], (unsigned long long)run);
    }
}

template <int WP>
__global__ void __launch_bounds__(kChunkThreads) k_batch_scatter(uint32_t nch, const uint8_t* __restrict__ oflag,
                                                               const uint64_t* __restrict__ coff,
                                                               const uint64_t* __restrict__ Tkeys,
                                                               const double2* __restrict__ Tcoef,
                                                               const uint64_t* __restrict__ pstart,
                                                               const OutDesc* __restrict__ outs) {
    constexpr int NW = 2 * WP + 2;
    __shared__ uint32_t s_warp[32];
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
        for_each_flagged(c, oflag, coff, s_warp, [&](uint64_t p, uint64_t d) {
            uint64_t k[NW];
            key_load_g<NW>(Tkeys, p, k);
            const uint32_t b = (uint32_t)k[0];
            const uint64_t pos = d - pstart[b];
            const OutDesc o = outs[b];
            uint64_t kk[2 * WP];
#pragma unroll
            for (int w = 0; w < 2 * WP; ++w) kk[w] = k[2 + w];
            key_store<2 * WP>(o.keys, pos, kk);
            o.coef[pos] = Tcoef[p];
            o.pbase[pos] = (uint8_t)normal_phase<WP>(kk, 0u);
        });
    }
}

// FP32 copies of operand coefficients: job j converts n[j] values.
struct F32Job {
    const double2* src;
    float2* dst;
    uint64_t n;
    uint64_t pad;
};
__global__ void k_batch_to_f32(const F32Job* jobs, uint32_t njobs) {
    for (uint32_t j = blockIdx.x; j < njobs; j += gridDim.x) {
        const F32Job jb = jobs[j];
        for (uint64_t t = threadIdx.x; t < jb.n; t += blockDim.x)
            jb.dst[t] = make_float2(__double2float_rn(jb.src[t].x), __double2float_rn(jb.src[t].y));
    }
}

}  // namespace paulib

struct paulib_batch_plan {
    int32_t batch = 0, n_qubits = 0, WP = 0, mode = 0;
    uint64_t R = 0;
    std::vector<paulib_sum*> outs;
    void* desc = nullptr;  // descriptors, offsets, counters (one allocation)
    void* f32 = nullptr;   // FP32 coefficient copies (mixed-precision modes)
    void* arena = nullptr;
    size_t arena_bytes = 0;
    bool released = false;
    paulib::ProbDesc* d_probs = nullptr;
    uint32_t* d_r0s = nullptr;
    paulib::OutDesc* d_outs = nullptr;
    unsigned long long* d_counts = nullptr;
    uint64_t* d_pstart = nullptr;
    int32_t* d_err = nullptr;
    uint32_t* d_order = nullptr;  // problems by decreasing |A_b||B_b| (persistent kernel)
    uint32_t* d_ticket = nullptr;
    bool persist = false;
    uint32_t leaf_cap = 0;   // 0: the compiled capacity
    uint32_t split_fan = 0;  // 0: the kernel's default
    int ctas_per_sm = 2;
};

namespace paulib {

template <int WP, int MODE>
static void persist_launch(paulib_batch_plan* p, cudaStream_t st) {
    constexpr int NW = 2 * WP;
    using Lay = PLayout<WP, MODE>;
    auto kern = k_batch_persist<WP, MODE>;
    smem_attr(kern, Lay::BYTES);
    int per_sm = 0;
    if (!capture_safe())
        check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPThreads, Lay::BYTES), "occupancy");
    if (per_sm > 0) p->ctas_per_sm = per_sm;
    const uint32_t grid = (uint32_t)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)p->batch, (int64_t)device_sm_count() * std::max(1, p->ctas_per_sm)));
    Scratch bufs((size_t)p->R * 9, st);  // two record buffers and a child byte per record
    Scratch levels((size_t)grid * persist_depth<NW>() * sizeof(PLevel), st);
    StageScope ss(ST_LEAF, st);
    check_cuda(cudaMemsetAsync(p->d_ticket, 0, 4, st), "memset ticket");
    kern<<<grid, kPThreads, Lay::BYTES, st>>>(p->d_probs, p->d_outs, p->d_order, p->d_r0s, (uint32_t)p->batch,
                                              bufs.as<uint32_t>(), bufs.as<uint32_t>() + p->R,
                                              reinterpret_cast<uint8_t*>(bufs.as<uint32_t>() + 2 * p->R),
                                              levels.as<PLevel>(), p->d_ticket, p->d_counts, p->d_err,
                                              p->leaf_cap, p->split_fan);
    note_launch(ST_LEAF);
    check_cuda(cudaGetLastError(), "k_batch_persist");
}

template <int WP, int MODE>
static void batch_launch_impl(paulib_batch_plan* p, cudaStream_t st) {
    using Src = BatchSrc<WP, MODE>;
    constexpr int NW = Src::NW;
    check_cuda(cudaMemsetAsync(p->d_counts, 0, (size_t)p->batch * 8, st), "memset counts");
    check_cuda(cudaMemsetAsync(p->d_err, 0, 4, st), "memset err");
    if (p->R == 0) return;
    if (p->persist) {
        persist_launch<WP, MODE>(p, st);
        return;
    }
    Src src{p->d_probs, p->d_r0s, (uint32_t)p->batch};
    Staged sg;
    run_pipeline<Src, MODE>(src, (uint32_t)p->R, 0, st, sg);
    StageScope ss(ST_COMPACT, st);
    const unsigned grid = std::max<uint32_t>(1, std::min<uint32_t>(sg.nch, (uint32_t)device_sm_count() * 8));
    k_or_err<<<1, 32, 0, st>>>(sg.err.as<int32_t>(), p->d_err);
    k_batch_counts<NW><<<grid, kChunkThreads, 0, st>>>(sg.nch, sg.oflag.as<uint8_t>(), sg.coff.as<uint64_t>(),
                                                       sg.Tkeys.as<uint64_t>(), p->d_counts);
    k_scan_u64<<<1, 1024, 0, st>>>(reinterpret_cast<const uint64_t*>(p->d_counts), (uint32_t)p->batch, p->d_pstart);
    k_batch_scatter<WP><<<grid, kChunkThreads, 0, st>>>(sg.nch, sg.oflag.as<uint8_t>(), sg.coff.as<uint64_t>(),
                                                        sg.Tkeys.as<uint64_t>(), sg.Tcoef.as<double2>(), p->d_pstart,
                                                        p->d_outs);
    for (int q = 0; q < 4; ++q) note_launch(ST_COMPACT);
    check_cuda(cudaGetLastError(), "batched output");
}

static void batch_launch(paulib_batch_plan* p, cudaStream_t st) {
#define L(WPv)                                                                                  \
    {                                                                                           \
        if (p->mode == M_FP64) batch_launch_impl<WPv, M_FP64>(p, st);                           \
        else if (p->mode == M_F32_D64) batch_launch_impl<WPv, M_F32_D64>(p, st);                \
        else batch_launch_impl<WPv, M_F32_TWOSUM>(p, st);                                       \
    }
    PAULIB_DISPATCH_WP(p->WP, L);
#undef L
}

struct ArenaRecordGuard {
    bool on = true;
    ArenaRecordGuard() { arena_record_begin(); }
    size_t end() { on = false; return arena_record_end(); }
    ~ArenaRecordGuard() { if (on) arena_record_end(); }
};
struct ArenaReplayGuard {
    ArenaReplayGuard(void* b, size_t n) { arena_replay_begin(b, n); }
    ~ArenaReplayGuard() { arena_replay_end(); }
};

static void plan_free(paulib_batch_plan* p, cudaStream_t st) {
    if (!p) return;
    if (!p->released)
        for (paulib_sum* s : p->outs) sum_free(s, st);
    dev_free(p->desc, st);
    dev_free(p->f32, st);
    dev_free(p->arena, st);
    delete p;
}

paulib_batch_plan* batch_plan_create(int32_t batch, const paulib_sum* const* a, const paulib_sum* const* b,
                                     int mode, cudaStream_t st) {
    paulib_batch_plan* p = new paulib_batch_plan;
    try {
        p->batch = batch;
        p->n_qubits = a[0]->n_qubits;
        p->WP = a[0]->WP;
        p->mode = mode;
        std::vector<uint32_t> r0s(batch + 1, 0);
        uint64_t R = 0;
        for (int32_t q = 0; q < batch; ++q) {
            r0s[q] = (uint32_t)R;
            R += (uint64_t)a[q]->n_terms * (uint64_t)b[q]->n_terms;
            if (R >= ((uint64_t)1 << 32) - 1) fail(PAULIB_ERR_UNSUPPORTED, "batched products need sum |A_b||B_b| < 2^32");
        }
        r0s[batch] = (uint32_t)R;
        p->R = R;
        p->outs.assign(batch, nullptr);
        for (int32_t q = 0; q < batch; ++q) {
            p->outs[q] = sum_alloc(p->n_qubits, a[q]->n_terms * b[q]->n_terms, false, st);
            p->outs[q]->is_canonical = 1;
            p->outs[q]->plan_owned = true;
            p->outs[q]->n_terms = 0;
        }
        // descriptor block
        const size_t szP = (size_t)batch * sizeof(ProbDesc);
        const size_t szR = ((size_t)(batch + 1) * 4 + 255) / 256 * 256;
        const size_t szO = (size_t)batch * sizeof(OutDesc);
        const size_t szC = ((size_t)batch * 8 + 255) / 256 * 256;
        const size_t szS = ((size_t)(batch + 1) * 8 + 255) / 256 * 256;
        const size_t szQ = ((size_t)batch * 4 + 255) / 256 * 256;
        const size_t total = szP + szR + szO + szC + szS + 256 + szQ + 256;
        p->desc = dev_alloc(total, st);
        char* base = static_cast<char*>(p->desc);
        p->d_probs = reinterpret_cast<ProbDesc*>(base);
        p->d_r0s = reinterpret_cast<uint32_t*>(base + szP);
        p->d_outs = reinterpret_cast<OutDesc*>(base + szP + szR);
        p->d_counts = reinterpret_cast<unsigned long long*>(base + szP + szR + szO);
        p->d_pstart = reinterpret_cast<uint64_t*>(base + szP + szR + szO + szC);
        p->d_err = reinterpret_cast<int32_t*>(base + szP + szR + szO + szC + szS);
        p->d_order = reinterpret_cast<uint32_t*>(base + szP + szR + szO + szC + szS + 256);
        p->d_ticket = reinterpret_cast<uint32_t*>(base + szP + szR + szO + szC + szS + 256 + szQ);
        // the persistent kernel takes the batch when every right operand fits
        // its shared memory; problems go largest first
        const DebugSettings dbg = debug_settings();
        p->persist = dbg.batch_general == 0;
        for (int32_t q = 0; q < batch && p->persist; ++q)
            if ((uint64_t)b[q]->n_terms > kPNB) p->persist = false;
        const BatchTuning bt = batch_tuning();
        p->leaf_cap = dbg.persist_leaf > 0 ? (uint32_t)dbg.persist_leaf : (uint32_t)bt.leaf_cap;
        p->split_fan = (uint32_t)bt.split_fan;
        std::vector<uint32_t> order(batch);
        for (int32_t q = 0; q < batch; ++q) order[q] = (uint32_t)q;
        std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
            return (uint64_t)(r0s[x + 1] - r0s[x]) > (uint64_t)(r0s[y + 1] - r0s[y]);
        });
        std::vector<ProbDesc> hp(batch);
        std::vector<OutDesc> ho(batch);
        std::vector<F32Job> jobs;
        size_t f32_total = 0;
        if (mode != M_FP64)
            for (int32_t q = 0; q < batch; ++q) f32_total += (size_t)(a[q]->n_terms + b[q]->n_terms);
        if (f32_total) p->f32 = dev_alloc(f32_total * sizeof(float2), st);
        float2* f = static_cast<float2*>(p->f32);
        for (int32_t q = 0; q < batch; ++q) {
            ProbDesc& d = hp[q];
            d.ak = a[q]->keys;
            d.bk = b[q]->keys;
            d.ap = a[q]->pbase;
            d.bp = b[q]->pbase;
            d.na = (uint32_t)a[q]->n_terms;
            d.nb = (uint32_t)b[q]->n_terms;
            d.na_inv = recip64(d.na);
            if (mode == M_FP64) {
                d.ac = a[q]->coef;
                d.bc = b[q]->coef;
            } else {
                d.ac = f;
                if (a[q]->n_terms) jobs.push_back(F32Job{a[q]->coef, f, (uint64_t)a[q]->n_terms, 0});
                f += a[q]->n_terms;
                d.bc = f;
                if (b[q]->n_terms) jobs.push_back(F32Job{b[q]->coef, f, (uint64_t)b[q]->n_terms, 0});
                f += b[q]->n_terms;
            }
            ho[q] = OutDesc{p->outs[q]->keys, p->outs[q]->coef, p->outs[q]->pbase, 0};
        }
        check_cuda(cudaMemcpyAsync(p->d_probs, hp.data(), szP, cudaMemcpyHostToDevice, st), "desc copy");
        check_cuda(cudaMemcpyAsync(p->d_r0s, r0s.data(), (size_t)(batch + 1) * 4, cudaMemcpyHostToDevice, st), "r0 copy");
        check_cuda(cudaMemcpyAsync(p->d_outs, ho.data(), szO, cudaMemcpyHostToDevice, st), "out copy");
        check_cuda(cudaMemcpyAsync(p->d_order, order.data(), (size_t)batch * 4, cudaMemcpyHostToDevice, st),
                   "order copy");
        Scratch jobs_d;
        if (!jobs.empty()) {
            jobs_d = Scratch(jobs.size() * sizeof(F32Job), st);
            check_cuda(cudaMemcpyAsync(jobs_d.p, jobs.data(), jobs.size() * sizeof(F32Job), cudaMemcpyHostToDevice, st),
                       "job copy");
            k_batch_to_f32<<<std::min<size_t>(jobs.size(), 4096), 256, 0, st>>>(jobs_d.as<F32Job>(), (uint32_t)jobs.size());
            note_launch(ST_CONVERT);
            check_cuda(cudaGetLastError(), "k_batch_to_f32");
        }
        // one full run that records the workspace it asks for
        {
            ArenaRecordGuard rec;
            batch_launch(p, st);
            p->arena_bytes = rec.end();
        }
        if (p->arena_bytes) p->arena = dev_alloc(p->arena_bytes, st);
        check_cuda(cudaStreamSynchronize(st), "plan sync");  // host vectors above must outlive their copies
    } catch (...) {
        plan_free(p, st);
        throw;
    }
    return p;
}

void batch_plan_launch(paulib_batch_plan* p, cudaStream_t st) {
    ArenaReplayGuard g(p->arena, p->arena_bytes);
    batch_launch(p, st);
}

void batch_plan_outputs(paulib_batch_plan* p, cudaStream_t st, paulib_sum** out) {
    std::vector<unsigned long long> cnt(p->batch);
    int32_t e = 0;
    check_cuda(cudaMemcpyAsync(cnt.data(), p->d_counts, (size_t)p->batch * 8, cudaMemcpyDeviceToHost, st), "count copy");
    check_cuda(cudaMemcpyAsync(&e, p->d_err, 4, cudaMemcpyDeviceToHost, st), "err copy");
    check_cuda(cudaStreamSynchronize(st), "outputs sync");
    if (e) fail(PAULIB_ERR_INTERNAL, "batched canonicalisation failed on device (error word " + std::to_string(e) + ")");
    for (int32_t q = 0; q < p->batch; ++q) {
        p->outs[q]->n_terms = (int64_t)cnt[q];
        out[q] = p->outs[q];
    }
}

void batch_plan_destroy(paulib_batch_plan* p) { plan_free(p, nullptr); }

void canon_batched(int32_t batch, const paulib_sum* const* a, const paulib_sum* const* b, int mode,
                   cudaStream_t st, paulib_sum** out) {
    paulib_batch_plan* p = batch_plan_create(batch, a, b, mode, st);
    try {
        batch_plan_outputs(p, st, out);
    } catch (...) {
        plan_free(p, st);
        throw;
    }
    for (paulib_sum* s : p->outs) s->plan_owned = false;  // ownership passes to the caller
    p->released = true;
    plan_free(p, st);
}

}  // namespace paulib
