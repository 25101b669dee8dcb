// paulib_internal.h -- host-side internals shared by the library's .cu files.
#pragma once
#include <cstdint>
#include <string>
#include <cuda_runtime.h>
#include "../../include/paulib.h"

// A device-resident Pauli sum.  One allocation holds every array.
struct paulib_sum {
    int32_t n_qubits = 0;
    int32_t W = 0;        // ceil(n/64): words per half at the API boundary
    int32_t WP = 0;       // padded words per half in device memory (1,2,4,8,16)
    int64_t n_terms = 0;
    int32_t is_canonical = 0;
    int32_t device = 0;
    cudaStream_t stream = nullptr;  // stream of the call that produced it; destroy frees on it
    uint64_t* keys = nullptr;   // [n_terms][2*WP] : x words then z words, zero padded
    double2* coef = nullptr;    // [n_terms] complex128
    uint8_t* pbase = nullptr;   // [n_terms] (|x&z| + phase) mod 4: exponent in the X^x Z^z form
    uint8_t* phase = nullptr;   // [n_terms] own phase exponent, or null when all zero
    void* block = nullptr;      // the single allocation
    size_t block_bytes = 0;
    bool plan_owned = false;    // storage of a batched plan's output: destroy is a no-op
};

namespace paulib {

struct Error {
    paulib_status status;
    std::string msg;
};

[[noreturn]] void fail(paulib_status st, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);

void* dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

// Workspace arena for prepared (plan) launches.  While recording, every
// dev_alloc is served normally and its size is added up; while replaying,
// dev_alloc hands out consecutive pieces of one pre-allocated block and
// dev_free does nothing, so a launch neither allocates nor frees.  The
// pipeline's allocation sequence depends only on operand sizes, so a replay
// asks for exactly the recorded pieces.  Replay also marks the thread
// capture-safe: no host synchronisation, no event timing, no attribute calls.
void arena_record_begin();
size_t arena_record_end();
void arena_replay_begin(void* base, size_t bytes);
void arena_replay_end();
bool capture_safe();

// Pipeline scratch.  Blocks of 1 MiB or more are kept by the library after
// use and handed to later requests of (about) the same size on the same
// stream and device; the stream order makes the reuse safe without events.
// This keeps the device pool's cached memory for the outputs, whose sizes
// repeat from call to call, instead of letting the large scratch requests
// carve it up (which made every large output map fresh memory).  Other
// blocks, arena replays and user allocators go straight to dev_alloc.
void* scratch_alloc(size_t bytes, cudaStream_t s);
void scratch_free(void* p, size_t bytes, cudaStream_t s);
void scratch_cache_flush();

// A scratch buffer freed (stream ordered) when it goes out of scope.
struct Scratch {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    size_t bytes = 0;
    Scratch() = default;
    Scratch(size_t n, cudaStream_t st) : p(n ? scratch_alloc(n, st) : nullptr), s(st), bytes(n) {}
    Scratch(const Scratch&) = delete;
    Scratch& operator=(const Scratch&) = delete;
    Scratch(Scratch&& o) noexcept : p(o.p), s(o.s), bytes(o.bytes) { o.p = nullptr; }
    Scratch& operator=(Scratch&& o) noexcept {
        if (this != &o) { release(); p = o.p; s = o.s; bytes = o.bytes; o.p = nullptr; }
        return *this;
    }
    ~Scratch() { release(); }
    void release() { if (p) scratch_free(p, bytes, s); p = nullptr; }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

int padded_words(int W);

// Pipeline tuning (paulib_set_tuning); never changes results.
struct Tuning {
    int coarse_factor = 32;
    int oversample = 64;
    int count_ctas_per_sm = 8;
    int range_ctas_per_sm = 2;
};
Tuning tuning_for(int key_words);
void set_tuning(int key_words, const Tuning& t);

// Sizes of the persistent batched kernel (paulib_set_batch_tuning); never
// change results.  leaf_cap: records of a shared-memory leaf (0: the
// compiled capacity); split_fan: children per leaf's worth of records in a
// sample split (0: 2).
struct BatchTuning {
    int leaf_cap = 0;
    int split_fan = 0;
};
BatchTuning batch_tuning();
void set_batch_tuning(const BatchTuning& t);

// Test settings (paulib_set_debug); 0 = off.  hash_bits: keep only the low
// hash_bits bits of the range sort's warp-leaf key hashes (forces the
// hash-clash path); stack_cap: entries of a range CTA's worklist (a small cap
// makes the split raise its stack error and return); batch_general: batch
// plans made afterwards use the general pipeline; persist_leaf: a smaller
// leaf for the persistent batched kernel (more splits on small inputs).
struct DebugSettings {
    int hash_bits = 0;
    int stack_cap = 0;
    int batch_general = 0;  // batch plans take the general pipeline
    int persist_leaf = 0;   // leaf capacity of the persistent batched kernel
};
DebugSettings debug_settings();
void set_debug(int knob, int64_t value);

// Canonicalisation method and slot-sort tuning (paulib_set_slot_tuning);
// never changes results.  0 fields mean the built-in default.
struct SlotTuning {
    int method = 1;      // 0 slot sort, 1 range sort (the default: faster on every workload measured)
    int leaf_cap = 0;    // terms per leaf (at most the compiled capacity)
    int target = 0;      // mean terms per fine slot
    int oversample = 0;  // sample keys per fine slot
};
SlotTuning slot_tuning_for(int key_words);
void set_slot_tuning(int key_words, const SlotTuning& t, bool keep_method);
// Records which method produced the last canonical result on this thread
// (0 slot sort, 1 range sort) and the device bits that made the slot sort
// hand the case over (0 when it did not).
void note_canon_method(int method, int bits);
int last_canon_method(int* bits);
// Shape of the last slot sort on this thread: coarse ranges, slot capacity
// per range, leaves, leaf capacity, slot target.
void note_canon_stats(int64_t ranges, int64_t slots_per_range, int64_t leaves, int64_t leaf_cap, int64_t target);
void last_canon_stats(int64_t* out5);

#define PAULIB_DISPATCH_WP(wp, F)                                                   \
    switch (wp) {                                                                   \
        case 1: F(1); break;                                                        \
        case 2: F(2); break;                                                        \
        case 4: F(4); break;                                                        \
        case 8: F(8); break;                                                        \
        case 16: F(16); break;                                                      \
        default: ::paulib::fail(PAULIB_ERR_INTERNAL, "unsupported padded word count"); \
    }
int device_sm_count();

// ---- stage timing (paulib_timing_*): events are recorded only by the
// outermost active scope, so nested pipelines count toward the outer stage.
enum Stage : int {
    ST_CONVERT = 0, ST_SAMPLE = 1, ST_COUNT = 2, ST_SCATTER = 3, ST_LEVEL2 = 4, ST_COMPACT = 5,
    ST_RAW = 6, ST_EXPORT = 7, ST_LEAF = 8, ST_GROUP = 9, ST_SPLIT = 10, ST_PLACE = 11
};
struct StageScope {
    StageScope(int stage, cudaStream_t s);
    ~StageScope();
    StageScope(const StageScope&) = delete;
    StageScope& operator=(const StageScope&) = delete;
    int stage;
    cudaStream_t s;
    bool outer;
    cudaEvent_t a = nullptr;
};
// Counts one kernel launch toward the outermost active stage (or `stage`
// when none is active).
void note_launch(int stage);

// Allocates an empty sum shell with storage for n terms.
paulib_sum* sum_alloc(int32_t n_qubits, int64_t n_terms, bool with_phase, cudaStream_t s);
void sum_free(paulib_sum* s, cudaStream_t st);

// ---- conversion kernels (paulib_convert.cu)
// SoA device arrays -> sum storage; sets *err_flag (device) nonzero when a
// tail bit is set.
void launch_create(paulib_sum* s, const uint64_t* x_soa, const uint64_t* z_soa, const double* coef,
                   const uint8_t* phase, int32_t* err_flag, cudaStream_t st);
void launch_export(const paulib_sum* s, uint64_t* x_soa, uint64_t* z_soa, double* coef,
                   uint8_t* phase, cudaStream_t st);
void launch_outer_raw(const paulib_sum* a, const paulib_sum* b, paulib_sum* out, cudaStream_t st);

// ---- canonicalisation (paulib_canon.cu)
paulib_sum* canon_product(const paulib_sum* a, const paulib_sum* b, int mode, cudaStream_t st);
paulib_sum* canon_terms(const paulib_sum* in, int mode, cudaStream_t st);
void canon_batched(int32_t batch, const paulib_sum* const* a, const paulib_sum* const* b, int mode,
                   cudaStream_t st, paulib_sum** out);

paulib_batch_plan* batch_plan_create(int32_t batch, const paulib_sum* const* a, const paulib_sum* const* b,
                                     int mode, cudaStream_t st);
void batch_plan_launch(paulib_batch_plan* p, cudaStream_t st);
void batch_plan_outputs(paulib_batch_plan* p, cudaStream_t st, paulib_sum** out);
void batch_plan_destroy(paulib_batch_plan* p);

// ---- gates and rotations (paulib_gates.cu)
paulib_sum* multiply_pairwise(const paulib_sum* a, const paulib_sum* b, cudaStream_t st);
// Greedy commutation grouping (paulib_group.cu); returns the number of groups.
int64_t group_commuting(const paulib_sum* s, int32_t* group, int32_t* offsets, int32_t* members, cudaStream_t st);
void set_group_cands(int k);
void apply_clifford(paulib_sum* s, int32_t nops, const int32_t* ops_host, cudaStream_t st);
paulib_sum* rotate(const paulib_sum* s, const uint64_t* pk_host, double theta, double threshold, int mode,
                   cudaStream_t st);

// Pipe microbenchmarks (paulib_measure_peaks).
void measure_peaks(double* out, int n, cudaStream_t st);

// Allocation-free canonical product using the library's static scratch
// array (see paulib_multiply_noalloc in include/paulib.h).
void multiply_noalloc(int32_t n_qubits, int64_t na, const uint64_t* a_x, const uint64_t* a_z,
                      const double* a_c, int64_t nb, const uint64_t* b_x, const uint64_t* b_z,
                      const double* b_c, uint64_t* out_x, uint64_t* out_z, double* out_c,
                      int64_t out_capacity, int64_t* out_n, cudaStream_t st);

}  // namespace paulib
