// paulib_api.cu -- the C ABI (include/paulib.h): argument checks, memory
// management, host<->device staging, and dispatch to the kernels.
#include <cstdio>
#include <cstring>
#include <limits>
#include <mutex>
#include <new>
#include <vector>
#include "paulib_internal.h"

namespace paulib {

namespace {
thread_local std::string g_last_error;
paulib_alloc_fn g_alloc = nullptr;
paulib_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;
std::mutex g_pool_mu;
bool g_pool_configured[64] = {};
}  // namespace

void fail(paulib_status st, const std::string& msg) { throw Error{st, msg}; }

void check_cuda(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (e == cudaErrorMemoryAllocation) fail(PAULIB_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
        fail(PAULIB_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
}

static void configure_pool_once() {
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev < 0 || dev >= 64 || g_pool_configured[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        // Keep freed blocks cached in the pool instead of returning them to
        // the driver at every synchronisation.
        uint64_t thr = std::numeric_limits<uint64_t>::max();
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    g_pool_configured[dev] = true;
}

namespace {
struct ArenaState {
    int mode = 0;  // 0 off, 1 recording, 2 replaying
    char* base = nullptr;
    size_t cap = 0, off = 0, total = 0;
};
thread_local ArenaState g_arena;
constexpr size_t kArenaAlign = 256;
}  // namespace

void arena_record_begin() {
    g_arena = ArenaState{};
    g_arena.mode = 1;
}
size_t arena_record_end() {
    const size_t t = g_arena.total;
    g_arena = ArenaState{};
    return t;
}
void arena_replay_begin(void* base, size_t bytes) {
    g_arena = ArenaState{};
    g_arena.mode = 2;
    g_arena.base = static_cast<char*>(base);
    g_arena.cap = bytes;
}
void arena_replay_end() { g_arena = ArenaState{}; }
bool capture_safe() { return g_arena.mode == 2; }

void* dev_alloc(size_t bytes, cudaStream_t s) {
    if (bytes == 0) return nullptr;
    const size_t rounded = (bytes + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
    if (g_arena.mode == 2) {
        if (g_arena.off + rounded > g_arena.cap)
            fail(PAULIB_ERR_INTERNAL, "plan workspace exhausted (launch does not match its recording)");
        void* p = g_arena.base + g_arena.off;
        g_arena.off += rounded;
        return p;
    }
    if (g_arena.mode == 1) g_arena.total += rounded;
    if (g_alloc) {
        void* p = g_alloc(bytes, (void*)s, g_alloc_ctx);
        if (!p) fail(PAULIB_ERR_OOM, "allocator callback returned NULL for " + std::to_string(bytes) + " bytes");
        return p;
    }
    configure_pool_once();
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, s);
    if (e == cudaErrorMemoryAllocation) {
        // give back the cached scratch blocks and the pool's unused memory, then try once more
        cudaGetLastError();
        scratch_cache_flush();
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess)
            cudaMemPoolTrimTo(pool, 0);
        cudaGetLastError();
        p = nullptr;
        e = cudaMallocAsync(&p, bytes, s);
    }
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        fail(PAULIB_ERR_OOM, "cudaMallocAsync(" + std::to_string(bytes) + ") failed: " + cudaGetErrorString(e));
    }
    return p;
}

void dev_free(void* p, cudaStream_t s) {
    if (!p || g_arena.mode == 2) return;
    if (g_free) { g_free(p, (void*)s, g_alloc_ctx); return; }
    cudaFreeAsync(p, s);
}

// ---- scratch cache (see paulib_internal.h)
namespace {
struct CachedBlock {
    void* p;
    size_t bytes;
    int dev;
    cudaStream_t s;
};
std::mutex g_cache_mu;
std::vector<CachedBlock> g_cache;
constexpr size_t kCacheMin = (size_t)1 << 20;
constexpr size_t kCacheMaxBlocks = 64;
}  // namespace

void* scratch_alloc(size_t bytes, cudaStream_t s) {
    if (bytes < kCacheMin || g_arena.mode != 0 || g_alloc) return dev_alloc(bytes, s);
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        size_t best = g_cache.size();
        for (size_t i = 0; i < g_cache.size(); ++i) {
            const CachedBlock& b = g_cache[i];
            if (b.dev != dev || b.s != s || b.bytes < bytes || b.bytes > bytes + bytes / 4) continue;
            if (best == g_cache.size() || b.bytes < g_cache[best].bytes) best = i;
        }
        if (best != g_cache.size()) {
            void* p = g_cache[best].p;
            g_cache[best] = g_cache.back();
            g_cache.pop_back();
            return p;
        }
    }
    return dev_alloc(bytes, s);  // on running out of memory it flushes this cache and retries
}

void scratch_free(void* p, size_t bytes, cudaStream_t s) {
    if (!p) return;
    if (bytes < kCacheMin || g_arena.mode != 0 || g_free) {
        dev_free(p, s);
        return;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev_free(p, s);
        return;
    }
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_cache.push_back(CachedBlock{p, bytes, dev, s});
    if (g_cache.size() > kCacheMaxBlocks) {  // bounded: the oldest block goes back to the pool
        const CachedBlock old = g_cache.front();
        g_cache.erase(g_cache.begin());
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(old.dev);
        cudaFreeAsync(old.p, old.s);
        cudaSetDevice(cur);
        cudaGetLastError();
    }
}

void scratch_cache_flush() {
    std::vector<CachedBlock> blocks;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        blocks.swap(g_cache);
    }
    int cur = 0;
    cudaGetDevice(&cur);
    for (const CachedBlock& b : blocks) {
        cudaSetDevice(b.dev);
        cudaFreeAsync(b.p, b.s);
    }
    cudaSetDevice(cur);
    cudaDeviceSynchronize();  // the frees must complete before the pool can reuse the memory
    cudaGetLastError();
}

int padded_words(int W) {
    int wp = 1;
    while (wp < W) wp *= 2;
    return wp;
}

int device_sm_count() {
    static int cached[64] = {};
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev >= 0 && dev < 64 && cached[dev]) return cached[dev];
    int n = 0;
    check_cuda(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev), "sm count");
    if (dev >= 0 && dev < 64) cached[dev] = n;
    return n;
}

// ---------------------------------------------------------------- stage timing

namespace {
struct TimedSpan {
    int stage;
    cudaEvent_t a, b;
};
std::mutex g_t_mu;
bool g_timing = false;
int g_depth = 0;
int g_outer_stage = -1;
std::vector<TimedSpan> g_spans;
std::vector<cudaEvent_t> g_event_pool;
double g_ms[PAULIB_STAGES] = {};
int64_t g_launches[PAULIB_STAGES] = {};

cudaEvent_t take_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}
}  // namespace

StageScope::StageScope(int st, cudaStream_t str) : stage(st), s(str), outer(false) {
    std::lock_guard<std::mutex> lk(g_t_mu);
    if (g_depth++ == 0) {
        outer = true;
        g_outer_stage = st;
        if (g_timing && !capture_safe()) {
            a = take_event();
            if (a && cudaEventRecord(a, s) != cudaSuccess) {
                cudaGetLastError();
                g_event_pool.push_back(a);
                a = nullptr;
            }
        }
    }
}

StageScope::~StageScope() {
    std::lock_guard<std::mutex> lk(g_t_mu);
    --g_depth;
    if (outer) {
        g_outer_stage = -1;
        if (a) {
            cudaEvent_t b = take_event();
            if (b && cudaEventRecord(b, s) == cudaSuccess) g_spans.push_back(TimedSpan{stage, a, b});
            else g_event_pool.push_back(a);
        }
    }
}

void note_launch(int stage) {
    std::lock_guard<std::mutex> lk(g_t_mu);
    const int st = g_outer_stage >= 0 ? g_outer_stage : stage;
    if (st >= 0 && st < PAULIB_STAGES) g_launches[st] += 1;
}

// ---------------------------------------------------------------- tuning

namespace {
std::mutex g_tune_mu;
bool g_tune_loaded = false;
Tuning g_tune_all;
std::vector<std::pair<int, Tuning>> g_tune_by_words;

void merge_tuning(Tuning& dst, const Tuning& src) {
    if (src.coarse_factor > 0) dst.coarse_factor = std::min(256, std::max(2, src.coarse_factor));
    if (src.oversample > 0) dst.oversample = std::min(128, std::max(4, src.oversample));
    if (src.count_ctas_per_sm > 0) dst.count_ctas_per_sm = std::min(16, src.count_ctas_per_sm);
    if (src.range_ctas_per_sm > 0) dst.range_ctas_per_sm = std::min(2, src.range_ctas_per_sm);
}

void set_tuning_locked(int key_words, const Tuning& t) {
    if (key_words <= 0) {
        merge_tuning(g_tune_all, t);
        for (auto& kv : g_tune_by_words) merge_tuning(kv.second, t);
        return;
    }
    for (auto& kv : g_tune_by_words)
        if (kv.first == key_words) {
            merge_tuning(kv.second, t);
            return;
        }
    Tuning base = g_tune_all;
    merge_tuning(base, t);
    g_tune_by_words.push_back({key_words, base});
}

void load_tune_file_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = std::getenv("PAULIB_TUNE_FILE");
    if (!path || !*path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    char line[256];
    while (std::fgets(line, sizeof line, f)) {
        int kw = 0;
        Tuning t{0, 0, 0, 0};
        SlotTuning st;
        if (line[0] == '#') continue;
        BatchTuning bt;
        if (std::sscanf(line, "batch %d %d", &bt.leaf_cap, &bt.split_fan) == 2) {
            set_batch_tuning(bt);
            continue;
        }
        const int got = std::sscanf(line, "%d %d %d %d %d %d %d %d %d", &kw, &t.coarse_factor, &t.oversample,
                                    &t.count_ctas_per_sm, &t.range_ctas_per_sm, &st.method, &st.leaf_cap,
                                    &st.target, &st.oversample);
        if (got >= 5) set_tuning_locked(kw, t);
        if (got == 9 && (st.method == 0 || st.method == 1)) set_slot_tuning(kw, st, false);
    }
    std::fclose(f);
}
}  // namespace

Tuning tuning_for(int key_words) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_tune_file_locked();
    for (const auto& kv : g_tune_by_words)
        if (kv.first == key_words) return kv.second;
    return g_tune_all;
}

void set_tuning(int key_words, const Tuning& t) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_tune_file_locked();
    set_tuning_locked(key_words, t);
}

namespace {
std::mutex g_slot_mu;
SlotTuning g_slot_all;
std::vector<std::pair<int, SlotTuning>> g_slot_by_words;
thread_local int g_canon_method = -1;
thread_local int g_canon_bits = 0;
}  // namespace

namespace {
std::mutex g_batch_mu;
BatchTuning g_batch;
}  // namespace

BatchTuning batch_tuning() {
    {
        std::lock_guard<std::mutex> lt(g_tune_mu);  // the tune file may set it
        load_tune_file_locked();
    }
    std::lock_guard<std::mutex> lk(g_batch_mu);
    return g_batch;
}

void set_batch_tuning(const BatchTuning& t) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    g_batch = t;
}

SlotTuning slot_tuning_for(int key_words) {
    {
        std::lock_guard<std::mutex> lt(g_tune_mu);  // the tune file may set it
        load_tune_file_locked();
    }
    std::lock_guard<std::mutex> lk(g_slot_mu);
    for (const auto& kv : g_slot_by_words)
        if (kv.first == key_words) return kv.second;
    return g_slot_all;
}

void set_slot_tuning(int key_words, const SlotTuning& t, bool) {
    std::lock_guard<std::mutex> lk(g_slot_mu);
    if (key_words <= 0) {
        g_slot_all = t;
        g_slot_by_words.clear();
        return;
    }
    for (auto& kv : g_slot_by_words)
        if (kv.first == key_words) {
            kv.second = t;
            return;
        }
    g_slot_by_words.push_back({key_words, t});
}

namespace {
std::mutex g_debug_mu;
DebugSettings g_debug;
}  // namespace

DebugSettings debug_settings() {
    std::lock_guard<std::mutex> lk(g_debug_mu);
    return g_debug;
}

void set_debug(int knob, int64_t value) {
    std::lock_guard<std::mutex> lk(g_debug_mu);
    if (knob == 1) g_debug.hash_bits = (int)value;
    else if (knob == 2) g_debug.stack_cap = (int)value;
    else if (knob == 3) g_debug.batch_general = (int)value;
    else if (knob == 4) g_debug.persist_leaf = (int)value;
}

void note_canon_method(int method, int bits) {
    g_canon_method = method;
    g_canon_bits = bits;
}

int last_canon_method(int* bits) {
    *bits = g_canon_bits;
    return g_canon_method;
}

namespace {
thread_local int64_t g_canon_stats[5] = {0, 0, 0, 0, 0};
}

void note_canon_stats(int64_t ranges, int64_t slots_per_range, int64_t leaves, int64_t leaf_cap, int64_t target) {
    g_canon_stats[0] = ranges;
    g_canon_stats[1] = slots_per_range;
    g_canon_stats[2] = leaves;
    g_canon_stats[3] = leaf_cap;
    g_canon_stats[4] = target;
}

void last_canon_stats(int64_t* out5) {
    for (int q = 0; q < 5; ++q) out5[q] = g_canon_stats[q];
}

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

paulib_sum* sum_alloc(int32_t n_qubits, int64_t n_terms, bool with_phase, cudaStream_t s) {
    paulib_sum* r = new (std::nothrow) paulib_sum;
    if (!r) fail(PAULIB_ERR_OOM, "host allocation failed");
    r->n_qubits = n_qubits;
    r->W = (n_qubits + 63) / 64;
    r->WP = padded_words(r->W);
    r->n_terms = n_terms;
    check_cuda(cudaGetDevice(&r->device), "cudaGetDevice");
    r->stream = s;
    const size_t nt = (size_t)n_terms;
    const size_t kb = align_up(nt * 2 * r->WP * sizeof(uint64_t), 256);
    const size_t cb = align_up(nt * sizeof(double2), 256);
    const size_t pb = align_up(nt, 256);
    const size_t hb = with_phase ? align_up(nt, 256) : 0;
    r->block_bytes = kb + cb + pb + hb;
    if (n_terms > 0) {
        try {
            r->block = dev_alloc(r->block_bytes, s);
        } catch (...) {
            delete r;
            throw;
        }
        char* base = static_cast<char*>(r->block);
        r->keys = reinterpret_cast<uint64_t*>(base);
        r->coef = reinterpret_cast<double2*>(base + kb);
        r->pbase = reinterpret_cast<uint8_t*>(base + kb + cb);
        r->phase = with_phase ? reinterpret_cast<uint8_t*>(base + kb + cb + pb) : nullptr;
    }
    return r;
}

void sum_free(paulib_sum* s, cudaStream_t st) {
    if (!s) return;
    if (s->block) dev_free(s->block, st);
    delete s;
}

static bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Page-locked host memory is mapped into the device's address space: returns
// the device-side address of such a pointer, or NULL for device or pageable
// memory.  A kernel can then write there directly over the host link.
static void* mapped_host_ptr(void* p) {
    if (!p) return nullptr;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Returns a device pointer holding `bytes` of `src` (staging host data).
static const void* to_device(const void* src, size_t bytes, cudaStream_t s, Scratch& keep) {
    if (!src || bytes == 0) return src;
    if (is_device_ptr(src)) return src;
    keep = Scratch(bytes, s);
    check_cuda(cudaMemcpyAsync(keep.p, src, bytes, cudaMemcpyHostToDevice, s), "host-to-device copy");
    return keep.p;
}

}  // namespace paulib

using namespace paulib;

#define PAULIB_API_BEGIN try {
#define PAULIB_API_END                                             \
    }                                                              \
    catch (const Error& e) {                                       \
        g_last_error = e.msg;                                      \
        return e.status;                                           \
    }                                                              \
    catch (const std::bad_alloc&) {                                \
        g_last_error = "host allocation failed";                   \
        return PAULIB_ERR_OOM;                                     \
    }                                                              \
    catch (...) {                                                  \
        g_last_error = "unexpected internal exception";            \
        return PAULIB_ERR_INTERNAL;                                \
    }

extern "C" {

int32_t paulib_abi_version(void) { return PAULIB_ABI_VERSION; }

const char* paulib_last_error(void) { return g_last_error.c_str(); }

paulib_status paulib_set_allocator(paulib_alloc_fn alloc, paulib_free_fn free_, void* ctx) {
    if ((alloc == nullptr) != (free_ == nullptr)) {
        g_last_error = "allocator and free callbacks must both be set or both be NULL";
        return PAULIB_ERR_INVALID_ARG;
    }
    g_alloc = alloc;
    g_free = free_;
    g_alloc_ctx = ctx;
    return PAULIB_OK;
}

paulib_status paulib_sum_create(int32_t n_qubits, int64_t n_terms, const uint64_t* x_words,
                                const uint64_t* z_words, const double* coeffs, const uint8_t* phase,
                                void* stream, paulib_sum** out) {
    if (out) *out = nullptr;
    PAULIB_API_BEGIN
    if (!out) fail(PAULIB_ERR_INVALID_ARG, "out is NULL");
    if (n_qubits < 1 || n_qubits > PAULIB_MAX_QUBITS)
        fail(PAULIB_ERR_INVALID_ARG, "n_qubits must be in 1..1024, got " + std::to_string(n_qubits));
    if (n_terms < 0) fail(PAULIB_ERR_INVALID_ARG, "n_terms must be >= 0");
    if (n_terms > 0 && (!x_words || !z_words || !coeffs))
        fail(PAULIB_ERR_INVALID_ARG, "x_words, z_words and coeffs must be non-NULL when n_terms > 0");
    if (n_terms > ((int64_t)1 << 40)) fail(PAULIB_ERR_UNSUPPORTED, "n_terms too large");
    cudaStream_t s = (cudaStream_t)stream;
    paulib_sum* r = sum_alloc(n_qubits, n_terms, phase != nullptr, s);
    try {
        if (n_terms > 0) {
            const size_t wbytes = (size_t)r->W * (size_t)n_terms * sizeof(uint64_t);
            Scratch kx, kz, kc, kp;
            const uint64_t* dx = (const uint64_t*)to_device(x_words, wbytes, s, kx);
            const uint64_t* dz = (const uint64_t*)to_device(z_words, wbytes, s, kz);
            const double* dc = (const double*)to_device(coeffs, (size_t)n_terms * 16, s, kc);
            const uint8_t* dp = (const uint8_t*)to_device(phase, (size_t)n_terms, s, kp);
            Scratch flag(sizeof(int32_t), s);
            check_cuda(cudaMemsetAsync(flag.p, 0, sizeof(int32_t), s), "memset");
            launch_create(r, dx, dz, dc, dp, flag.as<int32_t>(), s);
            int32_t h = 0;
            check_cuda(cudaMemcpyAsync(&h, flag.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "flag copy");
            check_cuda(cudaStreamSynchronize(s), "create sync");
            if (h) fail(PAULIB_ERR_TAIL_BITS, "a bit at qubit >= n_qubits is set in the last word");
        }
    } catch (...) {
        sum_free(r, s);
        throw;
    }
    *out = r;
    return PAULIB_OK;
    PAULIB_API_END
}

paulib_status paulib_sum_info(const paulib_sum* s, int32_t* n_qubits, int64_t* n_terms,
                              int32_t* is_canonical) {
    PAULIB_API_BEGIN
    if (!s) fail(PAULIB_ERR_INVALID_ARG, "sum is NULL");
    if (n_qubits) *n_qubits = s->n_qubits;
    if (n_terms) *n_terms = s->n_terms;
    if (is_canonical) *is_canonical = s->is_canonical;
    return PAULIB_OK;
    PAULIB_API_END
}

static void export_impl(const paulib_sum* s, uint64_t* x_words, uint64_t* z_words, double* coeffs,
                        uint8_t* phase, void* stream);

paulib_status paulib_sum_export(const paulib_sum* s, uint64_t* x_words, uint64_t* z_words,
                                double* coeffs, uint8_t* phase, void* stream) {
    PAULIB_API_BEGIN
    if (!s) fail(PAULIB_ERR_INVALID_ARG, "sum is NULL");
    export_impl(s, x_words, z_words, coeffs, phase, stream);
    return PAULIB_OK;
    PAULIB_API_END
}

paulib_status paulib_sum_export_range(const paulib_sum* s, int64_t first, int64_t count, uint64_t* x_words,
                                      uint64_t* z_words, double* coeffs, uint8_t* phase, void* stream) {
    PAULIB_API_BEGIN
    if (!s) fail(PAULIB_ERR_INVALID_ARG, "sum is NULL");
    if (first < 0 || count < 0 || first > s->n_terms || count > s->n_terms - first)
        fail(PAULIB_ERR_INVALID_ARG, "terms [" + std::to_string(first) + ", " + std::to_string(first + count) +
                                         ") are outside the sum's " + std::to_string(s->n_terms) + " terms");
    paulib_sum v = *s;  // a view of terms [first, first + count): no ownership
    v.n_terms = count;
    if (count > 0) {
        v.keys = s->keys + (size_t)first * 2 * s->WP;
        v.coef = s->coef + first;
        v.pbase = s->pbase + first;
        v.phase = s->phase ? s->phase + first : nullptr;
    }
    export_impl(&v, x_words, z_words, coeffs, phase, stream);
    return PAULIB_OK;
    PAULIB_API_END
}

static void export_impl(const paulib_sum* s, uint64_t* x_words, uint64_t* z_words, double* coeffs,
                        uint8_t* phase, void* stream) {
    if (s->n_terms == 0) return;
    if (!x_words || !z_words || !coeffs) fail(PAULIB_ERR_INVALID_ARG, "output arrays must be non-NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nt = (size_t)s->n_terms;
    const size_t wbytes = (size_t)s->W * nt * sizeof(uint64_t);
    const bool dx = is_device_ptr(x_words), dz = is_device_ptr(z_words), dc = is_device_ptr(coeffs);
    const bool dp = phase ? is_device_ptr(phase) : true;
    // page-locked host outputs are written by the export kernel itself (no
    // staging copy); pageable ones are staged in device memory and copied
    void* const mx = dx ? nullptr : mapped_host_ptr(x_words);
    void* const mz = dz ? nullptr : mapped_host_ptr(z_words);
    void* const mc = dc ? nullptr : mapped_host_ptr(coeffs);
    void* const mp = (phase && !dp) ? mapped_host_ptr(phase) : nullptr;
    Scratch sx, sz, sc, sp;
    uint64_t* tx = dx ? x_words : static_cast<uint64_t*>(mx);
    uint64_t* tz = dz ? z_words : static_cast<uint64_t*>(mz);
    double* tc = dc ? coeffs : static_cast<double*>(mc);
    uint8_t* tp = dp ? phase : static_cast<uint8_t*>(mp);
    const bool cx = !tx, cz = !tz, cc = !tc, cp = phase && !tp;
    if (cx) { sx = Scratch(wbytes, st); tx = sx.as<uint64_t>(); }
    if (cz) { sz = Scratch(wbytes, st); tz = sz.as<uint64_t>(); }
    if (cc) { sc = Scratch(nt * 16, st); tc = sc.as<double>(); }
    if (cp) { sp = Scratch(nt, st); tp = sp.as<uint8_t>(); }
    launch_export(s, tx, tz, tc, tp, st);
    if (cx) check_cuda(cudaMemcpyAsync(x_words, tx, wbytes, cudaMemcpyDeviceToHost, st), "export copy");
    if (cz) check_cuda(cudaMemcpyAsync(z_words, tz, wbytes, cudaMemcpyDeviceToHost, st), "export copy");
    if (cc) check_cuda(cudaMemcpyAsync(coeffs, tc, nt * 16, cudaMemcpyDeviceToHost, st), "export copy");
    if (cp) check_cuda(cudaMemcpyAsync(phase, tp, nt, cudaMemcpyDeviceToHost, st), "export copy");
}

void paulib_sum_destroy(paulib_sum* s) {
    if (!s || s->plan_owned) return;
    try {
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != s->device) cudaSetDevice(s->device);
        sum_free(s, s->stream);
        if (cur != s->device) cudaSetDevice(cur);
    } catch (...) {
    }
}

static void check_pair(const paulib_sum* a, const paulib_sum* b) {
    if (!a || !b) fail(PAULIB_ERR_INVALID_ARG, "operand is NULL");
    if (a->n_qubits != b->n_qubits)
        fail(PAULIB_ERR_QUBIT_MISMATCH, "operands have " + std::to_string(a->n_qubits) + " and " +
                                            std::to_string(b->n_qubits) + " qubits");
}

static void check_mode(int32_t precision) {
    if (precision < PAULIB_FP64 || precision > PAULIB_FP32_MUL_TWOSUM_MERGE)
        fail(PAULIB_ERR_INVALID_ARG, "unknown precision mode " + std::to_string(precision));
}

paulib_status paulib_multiply(const paulib_sum* a, const paulib_sum* b, int32_t precision,
                              int32_t out_kind, void* stream, paulib_sum** out) {
    if (out) *out = nullptr;
    PAULIB_API_BEGIN
    if (!out) fail(PAULIB_ERR_INVALID_ARG, "out is NULL");
    check_pair(a, b);
    check_mode(precision);
    cudaStream_t s = (cudaStream_t)stream;
    if (out_kind == PAULIB_OUT_RAW) {
        if (precision != PAULIB_FP64) fail(PAULIB_ERR_INVALID_ARG, "raw products are FP64 only");
        const int64_t n = a->n_terms * b->n_terms;
        if (a->n_terms > 0 && n / a->n_terms != b->n_terms) fail(PAULIB_ERR_UNSUPPORTED, "size overflow");
        paulib_sum* r = sum_alloc(a->n_qubits, n, true, s);
        try {
            if (n > 0) launch_outer_raw(a, b, r, s);
        } catch (...) {
            sum_free(r, s);
            throw;
        }
        *out = r;
        return PAULIB_OK;
    }
    if (out_kind != PAULIB_OUT_CANONICAL) fail(PAULIB_ERR_INVALID_ARG, "unknown out_kind");
    *out = canon_product(a, b, precision, s);
    return PAULIB_OK;
    PAULIB_API_END
}

paulib_status paulib_compress(const paulib_sum* in, int32_t precision, void* stream,
                              paulib_sum** out) {
    if (out) *out = nullptr;
    PAULIB_API_BEGIN
    if (!out || !in) fail(PAULIB_ERR_INVALID_ARG, "NULL argument");
    check_mode(precision);
    *out = canon_terms(in, precision, (cudaStream_t)stream);
    return PAULIB_OK;
    PAULIB_API_END
}

paulib_status paulib_multiply_pairwise(const paulib_sum* a, const paulib_sum* b, void* stream, paulib_sum** out) {
    if (out) *out = nullptr;
    PAULIB_API_BEGIN
    if (!a || !b || !out) fail(PAULIB_ERR_INVALID_ARG, "NULL argument");
    if (a->n_qubits != b->n_qubits) fail(PAULIB_ERR_QUBIT_MISMATCH, "operands have different qubit counts");
    if (a->n_terms != b->n_terms) fail(PAULIB_ERR_INVALID_ARG, "pairwise product needs |a| == |b|");
    *out = multiply_pairwise(a, b, (cudaStream_t)stream);
    return PAULIB_OK;
    PAULIB_API_END
}

paulib_status paulib_group_commuting(const paulib_sum* s, int32_t* group_of_term, int32_t* group_offsets,
                                     int32_t* members, int64_t* n_groups, void* stream) {
    PAULIB_API_BEGIN
    if (!s || !n_groups || (!group_of_term && s->n_terms > 0)) fail(PAULIB_ERR_INVALID_ARG, "NULL argument");
    *n_groups = group_commuting(s, group_of_term, group_offsets, members, (cudaStream_t)stream);
    return PAULIB_OK;
    PAULIB_API_END
}

paulib_status paulib_set_group_candidates(int32_t k) {
    PAULIB_API_BEGIN
    if (k < 1 || k > 4) fail(PAULIB_ERR_INVALID_ARG, "candidates per term must be in 1..4");
    set_group_cands(k);
    return PAULIB_OK;
    PAULIB_API_END
}

paulib_status paulib_apply_clifford(paulib_sum* s, int32_t n_gates, const int32_t* gates, void* stream) {
    PAULIB_API_BEGIN
    if (!s) fail(PAULIB_ERR_INVALID_ARG, "NULL sum");
    if (n_gates < 0) fail(PAULIB_ERR_INVALID_ARG, "n_gates < 0");
    if (n_gates > 0 && !gates) fail(PAULIB_ERR_INVALID_ARG, "NULL gate list");
    for (int32_t g = 0; g < n_gates; ++g) {
        const int32_t gate = gates[3 * g], q1 = gates[3 * g + 1], q2 = gates[3 * g + 2];
        if (gate < PAULIB_GATE_H || gate > PAULIB_GATE_CZ)
            fail(PAULIB_ERR_INVALID_ARG, "unknown gate " + std::to_string(gate) + " at position " + std::to_string(g));
        const bool two = gate == PAULIB_GATE_CNOT || gate == PAULIB_GATE_CZ;
        if (q1 < 0 || q1 >= s->n_qubits || (two && (q2 < 0 || q2 >= s->n_qubits)))
            fail(PAULIB_ERR_INVALID_ARG, "gate " + std::to_string(g) + " acts outside the sum's qubits");
        if (two && q1 == q2) fail(PAULIB_ERR_INVALID_ARG, "two-qubit gate " + std::to_string(g) + " with q1 == q2");
    }
    apply_clifford(s, n_gates, gates, (cudaStream_t)stream);
    return PAULIB_OK;
    PAULIB_API_END
}

paulib_status paulib_rotate(const paulib_sum* s, const uint64_t* p_x, const uint64_t* p_z, double theta,
                            double threshold, int32_t precision, void* stream, paulib_sum** out) {
    if (out) *out = nullptr;
    PAULIB_API_BEGIN
    if (!s || !p_x || !p_z || !out) fail(PAULIB_ERR_INVALID_ARG, "NULL argument");
    check_mode(precision);
    const cudaStream_t st = (cudaStream_t)stream;
    const int W = s->W, WP = s->WP;
    std::vector<uint64_t> px(W), pz(W);
    if (is_device_ptr(p_x) || is_device_ptr(p_z)) {
        check_cuda(cudaMemcpyAsync(px.data(), p_x, (size_t)W * 8, cudaMemcpyDefault, st), "generator copy");
        check_cuda(cudaMemcpyAsync(pz.data(), p_z, (size_t)W * 8, cudaMemcpyDefault, st), "generator copy");
        check_cuda(cudaStreamSynchronize(st), "generator sync");
    } else {
        std::memcpy(px.data(), p_x, (size_t)W * 8);
        std::memcpy(pz.data(), p_z, (size_t)W * 8);
    }
    const int tail = s->n_qubits & 63;
    const uint64_t tail_mask = tail ? ~((1ull << tail) - 1ull) : 0ull;
    if ((px[W - 1] | pz[W - 1]) & tail_mask) fail(PAULIB_ERR_TAIL_BITS, "a generator bit at qubit >= n_qubits is set");
    std::vector<uint64_t> pk(2 * (size_t)WP, 0ull);  // the device key layout: x words, then z words, zero padded
    for (int w = 0; w < W; ++w) {
        pk[w] = px[w];
        pk[WP + w] = pz[w];
    }
    *out = rotate(s, pk.data(), theta, threshold, precision, st);
    return PAULIB_OK;
    PAULIB_API_END
}

paulib_status paulib_multiply_batched(int32_t batch, const paulib_sum* const* a,
                                      const paulib_sum* const* b, int32_t precision, void* stream,
                                      paulib_sum** out) {
    PAULIB_API_BEGIN
    if (batch < 0) fail(PAULIB_ERR_INVALID_ARG, "batch < 0");
    if (batch == 0) return PAULIB_OK;
    if (!a || !b || !out) fail(PAULIB_ERR_INVALID_ARG, "NULL array argument");
    for (int32_t i = 0; i < batch; ++i) out[i] = nullptr;
    check_mode(precision);
    for (int32_t i = 0; i < batch; ++i) {
        check_pair(a[i], b[i]);
        if (a[i]->n_qubits != a[0]->n_qubits)
            fail(PAULIB_ERR_QUBIT_MISMATCH, "batched operands must share one qubit count");
    }
    canon_batched(batch, a, b, precision, (cudaStream_t)stream, out);
    return PAULIB_OK;
    PAULIB_API_END
}

static void check_batch(int32_t batch, const paulib_sum* const* a, const paulib_sum* const* b) {
    if (batch <= 0) fail(PAULIB_ERR_INVALID_ARG, "batch must be >= 1");
    if (!a || !b) fail(PAULIB_ERR_INVALID_ARG, "NULL array argument");
    for (int32_t i = 0; i < batch; ++i) {
        check_pair(a[i], b[i]);
        if (a[i]->n_qubits != a[0]->n_qubits)
            fail(PAULIB_ERR_QUBIT_MISMATCH, "batched operands must share one qubit count");
    }
}

paulib_status paulib_batch_plan_create(int32_t batch, const paulib_sum* const* a,
                                       const paulib_sum* const* b, int32_t precision, void* stream,
                                       paulib_batch_plan** out) {
    if (out) *out = nullptr;
    PAULIB_API_BEGIN
    if (!out) fail(PAULIB_ERR_INVALID_ARG, "out is NULL");
    check_mode(precision);
    check_batch(batch, a, b);
    *out = batch_plan_create(batch, a, b, precision, (cudaStream_t)stream);
    return PAULIB_OK;
    PAULIB_API_END
}

paulib_status paulib_batch_plan_launch(paulib_batch_plan* plan, void* stream) {
    PAULIB_API_BEGIN
    if (!plan) fail(PAULIB_ERR_INVALID_ARG, "plan is NULL");
    batch_plan_launch(plan, (cudaStream_t)stream);
    return PAULIB_OK;
    PAULIB_API_END
}

paulib_status paulib_batch_plan_outputs(paulib_batch_plan* plan, void* stream, paulib_sum** out) {
    PAULIB_API_BEGIN
    if (!plan || !out) fail(PAULIB_ERR_INVALID_ARG, "NULL argument");
    batch_plan_outputs(plan, (cudaStream_t)stream, out);
    return PAULIB_OK;
    PAULIB_API_END
}

void paulib_batch_plan_destroy(paulib_batch_plan* plan) {
    try {
        batch_plan_destroy(plan);
    } catch (...) {
    }
}

paulib_status paulib_multiply_noalloc(int32_t n_qubits, int64_t na, const uint64_t* a_x,
                                      const uint64_t* a_z, const double* a_c, int64_t nb,
                                      const uint64_t* b_x, const uint64_t* b_z, const double* b_c,
                                      uint64_t* out_x, uint64_t* out_z, double* out_c,
                                      int64_t out_capacity, int64_t* out_n, void* stream) {
    PAULIB_API_BEGIN
    multiply_noalloc(n_qubits, na, a_x, a_z, a_c, nb, b_x, b_z, b_c, out_x, out_z, out_c, out_capacity, out_n,
                     (cudaStream_t)stream);
    return PAULIB_OK;
    PAULIB_API_END
}

paulib_status paulib_set_tuning(int32_t key_words, int32_t coarse_factor, int32_t oversample,
                                int32_t count_ctas_per_sm, int32_t range_ctas_per_sm) {
    PAULIB_API_BEGIN
    set_tuning(key_words, Tuning{coarse_factor, oversample, count_ctas_per_sm, range_ctas_per_sm});
    return PAULIB_OK;
    PAULIB_API_END
}

paulib_status paulib_set_batch_tuning(int32_t leaf_cap, int32_t split_fan) {
    PAULIB_API_BEGIN
    if (leaf_cap < -1 || (leaf_cap > 0 && (leaf_cap < 32 || leaf_cap > 2048)))
        fail(PAULIB_ERR_INVALID_ARG, "leaf_cap must be -1, 0 or 32..2048");
    if (split_fan < -1 || split_fan > 8) fail(PAULIB_ERR_INVALID_ARG, "split_fan must be -1..8");
    BatchTuning t = batch_tuning();
    if (leaf_cap >= 0) t.leaf_cap = leaf_cap;
    if (split_fan >= 0) t.split_fan = split_fan;
    set_batch_tuning(t);
    return PAULIB_OK;
    PAULIB_API_END
}

paulib_status paulib_set_slot_tuning(int32_t key_words, int32_t method, int32_t leaf_cap, int32_t slot_target,
                                     int32_t slot_oversample) {
    PAULIB_API_BEGIN
    if (method < -1 || method > 1) fail(PAULIB_ERR_INVALID_ARG, "method must be -1, 0 or 1");
    if (leaf_cap < -1 || (leaf_cap > 0 && (leaf_cap < 16 || leaf_cap > 4096)))
        fail(PAULIB_ERR_INVALID_ARG, "leaf_cap must be -1, 0 or 16..4096");
    if (slot_target < -1 || slot_target > (1 << 20)) fail(PAULIB_ERR_INVALID_ARG, "slot_target must be -1..2^20");
    if (slot_oversample < -1 || slot_oversample > 64) fail(PAULIB_ERR_INVALID_ARG, "slot_oversample must be -1..64");
    SlotTuning t = slot_tuning_for(key_words > 0 ? key_words : -1);
    if (method >= 0) t.method = method;
    if (leaf_cap >= 0) t.leaf_cap = leaf_cap;
    if (slot_target >= 0) t.target = slot_target;
    if (slot_oversample >= 0) t.oversample = slot_oversample;
    set_slot_tuning(key_words, t, true);
    return PAULIB_OK;
    PAULIB_API_END
}

paulib_status paulib_measure_peaks(double* out, int32_t n, void* stream) {
    PAULIB_API_BEGIN
    if (!out || n < 1) fail(PAULIB_ERR_INVALID_ARG, "out must hold at least one value");
    measure_peaks(out, n, (cudaStream_t)stream);
    return PAULIB_OK;
    PAULIB_API_END
}

paulib_status paulib_set_debug(int32_t knob, int64_t value) {
    PAULIB_API_BEGIN
    if (knob == 1) {
        if (value < 0 || value > 64) fail(PAULIB_ERR_INVALID_ARG, "hash bits must be 0..64");
    } else if (knob == 2) {
        if (value < 0 || value > 4096) fail(PAULIB_ERR_INVALID_ARG, "stack capacity must be 0..4096");
    } else if (knob == 3) {
        if (value < 0 || value > 1) fail(PAULIB_ERR_INVALID_ARG, "batched method setting must be 0 or 1");
    } else if (knob == 4) {
        if (value != 0 && (value < 32 || value > 2048))
            fail(PAULIB_ERR_INVALID_ARG, "persistent leaf capacity must be 0 or 32..2048");
    } else {
        fail(PAULIB_ERR_INVALID_ARG, "unknown debug setting " + std::to_string(knob));
    }
    set_debug(knob, value);
    return PAULIB_OK;
    PAULIB_API_END
}

paulib_status paulib_last_canon_stats(int64_t* stats) {
    PAULIB_API_BEGIN
    if (!stats) fail(PAULIB_ERR_INVALID_ARG, "NULL argument");
    last_canon_stats(stats);
    return PAULIB_OK;
    PAULIB_API_END
}

paulib_status paulib_last_canon_method(int32_t* method, int32_t* fallback_bits) {
    PAULIB_API_BEGIN
    if (!method || !fallback_bits) fail(PAULIB_ERR_INVALID_ARG, "NULL argument");
    int bits = 0;
    *method = last_canon_method(&bits);
    *fallback_bits = bits;
    return PAULIB_OK;
    PAULIB_API_END
}

paulib_status paulib_timing_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_t_mu);
    g_timing = on != 0;
    return PAULIB_OK;
}

paulib_status paulib_timing_read(double* ms, int64_t* launches, int32_t reset) {
    PAULIB_API_BEGIN
    std::lock_guard<std::mutex> lk(g_t_mu);
    for (const TimedSpan& sp : g_spans) {
        float t = 0.f;
        check_cuda(cudaEventSynchronize(sp.b), "cudaEventSynchronize");
        check_cuda(cudaEventElapsedTime(&t, sp.a, sp.b), "cudaEventElapsedTime");
        if (sp.stage >= 0 && sp.stage < PAULIB_STAGES) g_ms[sp.stage] += t;
        g_event_pool.push_back(sp.a);
        g_event_pool.push_back(sp.b);
    }
    g_spans.clear();
    for (int i = 0; i < PAULIB_STAGES; ++i) {
        if (ms) ms[i] = g_ms[i];
        if (launches) launches[i] = g_launches[i];
        if (reset) {
            g_ms[i] = 0.0;
            g_launches[i] = 0;
        }
    }
    return PAULIB_OK;
    PAULIB_API_END
}

}  // extern "C"
