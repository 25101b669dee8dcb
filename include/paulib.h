/*
 * paulib.h -- C ABI of the GB300 (sm_103a) Pauli-sum library.
 *
 * The library computes the Pauli-sum outer product and its canonical form as
 * defined in PauLIB (arXiv 2605.25974):
 *
 *   - A Pauli sum is H = sum_j c_j P_j with complex c_j and n-qubit Pauli
 *     strings P_j (Sec. III-A, Eq. 2).
 *   - A string is stored in the binary symplectic form (x|z) (Sec. III-C,
 *     Table I: I=(0,0), Z=(0,1), X=(1,0), Y=(1,1)), packed into W = ceil(n/64)
 *     64-bit X-words and W Z-words.  Qubit q is bit q%64 of word q/64 (the
 *     paper fixes the word index, Sec. III-G; the bit order is this library's).
 *     Bits at qubit >= n of the last word must be zero.
 *   - The product of two strings XORs their words; its phase i^k follows from
 *     popcounts of the words (Sec. III-E).  Concretely, with
 *     P(x,z) = i^{|x&z|} X^x Z^z, the product P_a P_b equals i^k P(x_a^x_b,
 *     z_a^z_b) with k = |x_a&z_a| + |x_b&z_b| + 2|z_a&x_b| - |x&z| (mod 4).
 *   - The product of two sums is the outer product: every left term times
 *     every right term, |A|*|B| products (Sec. IV-B, IV-C, V-C).
 *   - The canonical form sorts terms by a lexicographic key of the packed
 *     words and merges equal strings by adding their coefficients
 *     (Sec. III-H).  Key = (x_0..x_{W-1}, z_0..z_{W-1}) compared as unsigned
 *     64-bit words, word 0 most significant.  Strings whose merged coefficient
 *     is exactly zero are kept.
 *
 * Conventions for every call:
 *   - Sums are opaque, device resident and owned by the library.  A sum is
 *     immutable after creation; destroy it with paulib_sum_destroy.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     stream ordered; a call returns once its work is enqueued, except where
 *     noted (calls that must learn an output size synchronise `stream` once).
 *   - Array arguments may be host or device pointers (CUDA unified addressing
 *     decides); host arrays are copied through the stream.
 *   - No call aborts or throws.  A non-OK status leaves outputs untouched
 *     (output handles are set to NULL) and records a message readable with
 *     paulib_last_error() on the calling thread.
 *   - Only one GPU is used: the device current on the calling thread.
 */
#ifndef PAULIB_H
#define PAULIB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PAULIB_ABI_VERSION 3
#define PAULIB_MAX_QUBITS 1024

typedef struct paulib_sum paulib_sum;

typedef enum paulib_status {
    PAULIB_OK = 0,
    PAULIB_ERR_INVALID_ARG = 1,     /* bad pointer, size or enum value            */
    PAULIB_ERR_QUBIT_MISMATCH = 2,  /* operands have different qubit counts       */
    PAULIB_ERR_TAIL_BITS = 3,       /* a bit at qubit >= n is set                  */
    PAULIB_ERR_OOM = 4,             /* device allocation failed                    */
    PAULIB_ERR_CUDA = 5,            /* a CUDA runtime call failed                  */
    PAULIB_ERR_TIMEOUT = 6,         /* a bounded device wait expired               */
    PAULIB_ERR_UNSUPPORTED = 7,     /* size beyond this build's limits             */
    PAULIB_ERR_INTERNAL = 8         /* an internal consistency check failed        */
} paulib_status;

/* Arithmetic of the coefficient products and of the duplicate merge.  The
 * phase exponent and the key set are exact integers in every mode; outputs
 * are always complex128.  (The paper keeps a real double plus 2 phase bits,
 * Sec. III-C; this library keeps complex coefficients as in Eq. 2.)         */
typedef enum paulib_precision {
    PAULIB_FP64 = 0,                    /* FP64 products, FP64 merge             */
    PAULIB_FP32_MUL_FP64_MERGE = 1,     /* FP32 products widened to FP64 sums    */
    PAULIB_FP32_MUL_TWOSUM_MERGE = 2    /* FP32 products, FP32 TwoSum-compensated merge */
} paulib_precision;

enum { PAULIB_OUT_RAW = 0, PAULIB_OUT_CANONICAL = 1 };

int32_t paulib_abi_version(void);

/* Creates a sum of n_terms n-qubit terms (1 <= n_qubits <= 1024, n_terms >= 0).
 *   x_words, z_words: struct-of-arrays as in the paper's PauliSumSoA
 *       (Sec. IV-A): word w of term t at [w * n_terms + t], W = ceil(n/64)
 *       words per term.  NULL allowed only when n_terms == 0.
 *   coeffs: complex128 interleaved (re, im), n_terms entries.
 *   phase:  optional (NULL = all zero) exponents k in 0..3; term t is then
 *       i^k[t] * c[t] * P[t].  Higher bits are ignored.
 * Any order and repeated strings are accepted.  The library copies the data;
 * the caller keeps ownership of its arrays.  Synchronises `stream` once to
 * validate the tail bits (PAULIB_ERR_TAIL_BITS).                            */
paulib_status paulib_sum_create(int32_t n_qubits, int64_t n_terms, const uint64_t* x_words,
                                const uint64_t* z_words, const double* coeffs, const uint8_t* phase,
                                void* stream, paulib_sum** out);

/* Size and shape of a sum.  Any output pointer may be NULL. */
paulib_status paulib_sum_info(const paulib_sum* s, int32_t* n_qubits, int64_t* n_terms,
                              int32_t* is_canonical);

/* Export of terms [first, first + count) of a sum, with the layout and
 * rules of paulib_sum_export for a sum of `count` terms (arrays hold W*count
 * words, count coefficients, count phase bytes).  Lets a caller stream a
 * large sum out in slices.  No counterpart in the paper.
 * Errors: INVALID_ARG (NULL sum or outputs, a range outside the sum), CUDA. */
paulib_status paulib_sum_export_range(const paulib_sum* s, int64_t first, int64_t count, uint64_t* x_words,
                                      uint64_t* z_words, double* coeffs, uint8_t* phase, void* stream);

/* Copies a sum out in the paulib_sum_create layout (host or device arrays of
 * at least W*n_terms words / n_terms coefficients).  `phase` may be NULL; a
 * canonical sum has all phases zero.  Stream ordered: host arrays are valid
 * after `stream` is synchronised.  Page-locked host arrays (cudaHostAlloc,
 * torch pin_memory) are written by the export kernel directly over the host
 * link; pageable ones go through a device staging buffer and a copy.        */
paulib_status paulib_sum_export(const paulib_sum* s, uint64_t* x_words, uint64_t* z_words,
                                double* coeffs, uint8_t* phase, void* stream);

void paulib_sum_destroy(paulib_sum* s);

/* Outer product A*B (Sec. IV-C, V-C): every pair a_i * b_j, A on the left.
 *   out_kind PAULIB_OUT_RAW: |A|*|B| terms, product (i, j) at index
 *       j*|A| + i (one block of |A| per right term, Sec. IV-C); term phase =
 *       k_a + k_b + k_pair (mod 4); coefficient c_a*c_b (not rotated).
 *       `precision` must be PAULIB_FP64.
 *   out_kind PAULIB_OUT_CANONICAL: the canonical form (Sec. III-H) of the
 *       product: distinct strings in ascending key order, coefficient =
 *       sum over contributing pairs of i^k c_a c_b.  Synchronises `stream`
 *       once to learn the number of distinct strings.
 * Requires |A|*|B| < 2^32 for the canonical form (PAULIB_ERR_UNSUPPORTED
 * otherwise).  An empty operand gives an empty result.                      */
paulib_status paulib_multiply(const paulib_sum* a, const paulib_sum* b, int32_t precision,
                              int32_t out_kind, void* stream, paulib_sum** out);

/* Canonical form of one sum (Sec. III-H, sort_and_combine): a term with
 * phase k contributes i^k * c.  Synchronises `stream` once.                 */
paulib_status paulib_compress(const paulib_sum* in, int32_t precision, void* stream,
                              paulib_sum** out);

/* `batch` independent canonical products out[b] = canonical(a[b] * b[b]).
 * All operands must share one qubit count.  When every right operand has at
 * most 64 terms, one persistent kernel computes every product: its CTAs take
 * problems largest first and write each canonical sum directly.  Otherwise
 * all products go through one canonicalisation of keys prefixed by the
 * problem index.  Both give the same sums.                                  */
paulib_status paulib_multiply_batched(int32_t batch, const paulib_sum* const* a,
                                      const paulib_sum* const* b, int32_t precision, void* stream,
                                      paulib_sum** out);

/* Batched plan: the same batched canonical product, prepared once and then
 * launched any number of times without allocating or synchronising, so a
 * launch can be captured in a CUDA graph and replayed (e.g. one graph per
 * Pauli-propagation step shape).  The method is chosen at creation as for
 * paulib_multiply_batched: the persistent kernel (one launch after three
 * memsets) when every right operand has at most 64 terms, else the general
 * pipeline.
 *   create: validates the operands, sizes every buffer from |A_b|, |B_b| (each
 *     output's capacity is |A_b|*|B_b|) and runs the product once to lay out
 *     its workspace.  The operands must stay alive and unchanged while the
 *     plan exists (a launch reads them again).
 *   launch: enqueues the whole product on `stream` (kernels, device memsets
 *     and device-to-device copies only).
 *   outputs: synchronises `stream`, then fills out[batch] with handles to the
 *     plan's output sums (canonical, owned by the plan, valid until the next
 *     launch or destroy; do not destroy them).  Device errors of the last
 *     launch are reported here.                                              */
typedef struct paulib_batch_plan paulib_batch_plan;
paulib_status paulib_batch_plan_create(int32_t batch, const paulib_sum* const* a,
                                       const paulib_sum* const* b, int32_t precision, void* stream,
                                       paulib_batch_plan** out);
paulib_status paulib_batch_plan_launch(paulib_batch_plan* plan, void* stream);
paulib_status paulib_batch_plan_outputs(paulib_batch_plan* plan, void* stream, paulib_sum** out);
void paulib_batch_plan_destroy(paulib_batch_plan* plan);

/* Message for the last non-OK status returned on this thread ("" if none). */
const char* paulib_last_error(void);

/* Replaces the device allocator (NULL, NULL restores the default stream-
 * ordered cudaMallocAsync/cudaFreeAsync).  alloc returns NULL on failure
 * (reported as PAULIB_ERR_OOM).  Memory is freed through free_ on the stream
 * that last used it.  Not thread safe against concurrent calls.            */
typedef void* (*paulib_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*paulib_free_fn)(void* ptr, void* stream, void* ctx);
paulib_status paulib_set_allocator(paulib_alloc_fn alloc, paulib_free_fn free_, void* ctx);

/* Canonical product of two small sums that allocates no memory (the paper
 * has no counterpart; this is a service for callers that cannot allocate).
 * Some callers cannot let a library call cudaMalloc: a process whose device
 * memory is handed out by its own pool or fixed budget (an inference server
 * that reserves all HBM at start-up, a control loop that must never enter
 * the driver's allocator) would see a library allocation fail or break its
 * budget.  This call computes exactly what paulib_multiply(...,
 * PAULIB_FP64, PAULIB_OUT_CANONICAL, ...) computes, using only a fixed
 * scratch area compiled into the library as a static device array of
 * PAULIB_NOALLOC_SCRATCH_BYTES bytes that every GPU which loads the library
 * holds until the process exits.
 *   Limits (PAULIB_ERR_UNSUPPORTED beyond them, before any device work):
 *   n_qubits <= 256, na and nb <= 16384, na*nb <= 65536.
 *   Inputs: device SoA arrays as in paulib_sum_create (word w of term t at
 *   [w*n + t], complex128 coefficients), all phases zero.
 *   Outputs: device arrays with room for out_capacity >= na*nb terms, SoA
 *   with stride out_capacity (word w of output term t at
 *   out_x[w*out_capacity + t]); *out_n (device int64) receives the number of
 *   distinct strings; terms are in ascending key order.
 *   The first call on a device looks up the scratch array's device address
 *   (and sets kernel attributes); make that first call before any stream
 *   capture on the device.  Every call shares the one scratch array, so
 *   calls that overlap on the GPU (on different streams, or from different
 *   host threads) race: serialise them.  Synchronises `stream` once, to
 *   report device-side errors.                                             */
#define PAULIB_NOALLOC_MAX_QUBITS 256
#define PAULIB_NOALLOC_MAX_TERMS 16384
#define PAULIB_NOALLOC_MAX_PRODUCTS 65536
#define PAULIB_NOALLOC_SCRATCH_BYTES 8995072 /* about 8.6 MiB per GPU */
paulib_status paulib_multiply_noalloc(int32_t n_qubits, int64_t na, const uint64_t* a_x,
                                      const uint64_t* a_z, const double* a_c, int64_t nb,
                                      const uint64_t* b_x, const uint64_t* b_z, const double* b_c,
                                      uint64_t* out_x, uint64_t* out_z, double* out_c,
                                      int64_t out_capacity, int64_t* out_n, void* stream);

/* Tuning of the canonicalisation pipeline for keys of `key_words` 64-bit
 * words (2*WP for products and compress, 2*WP + 2 for batched products; 0 =
 * every size).  No counterpart in the paper; results never depend on it.
 *   coarse_factor: a first-level key range targets coarse_factor x the
 *       shared-memory leaf capacity records (2..256, default 32);
 *   oversample: splitter sample size per first-level range (4..128, default 64);
 *   count_ctas_per_sm: CTAs per SM of the first-level counting kernel (1..16,
 *       default 8);
 *   range_ctas_per_sm: CTAs per SM of the range sort/merge kernel (1..2).
 * A value <= 0 keeps the current setting.  If the environment variable
 * PAULIB_TUNE_FILE names a file when the library first needs a setting, its
 * lines "key_words coarse_factor oversample count_ctas_per_sm
 * range_ctas_per_sm [method leaf_cap slot_target slot_oversample]" are
 * applied first (the file the autotuner writes); the four optional fields
 * are those of paulib_set_slot_tuning (0 = built-in default).               */
paulib_status paulib_set_tuning(int32_t key_words, int32_t coarse_factor, int32_t oversample,
                                int32_t count_ctas_per_sm, int32_t range_ctas_per_sm);

/* Canonicalisation method (no counterpart in the paper; results never
 * depend on it, up to the summation order of equal keys).
 *   method 1 (default): range sort.  Records stay 32-bit pair numbers, keys
 *     are recomputed from the factors in every pass, and the merged terms are
 *     compacted into an output sized exactly.
 *   method 0: slot sort.  Each record's term (key, and coefficient with i^k
 *     folded in) is formed once into a fine key range; runs of ranges are
 *     ordered in shared memory and merged straight into the output sum, whose
 *     storage is sized for one term per record (|A|*|B|, or |A|(|A|+1)/2
 *     when both operands are the same sum) and trimmed only in its term
 *     count.  It hands a call to the range sort when a device check fails
 *     (see paulib_last_canon_method).
 * leaf_cap: terms per slot-sort leaf (16..4096, at most the compiled
 * capacity: 1024 up to four key words per half, 8192/(2*WP) beyond);
 * slot_target: mean terms per fine range; slot_oversample: sample keys per
 * fine range.  method -1 keeps the method; for the other arguments -1 keeps
 * a setting and 0 restores its default.  Applies to keys of `key_words`
 * words (0 = every size).
 * Errors: INVALID_ARG for values outside these ranges.                      */
/* Sizes of the persistent batched kernel (paulib_multiply_batched and
 * batch plans made afterwards; no counterpart in the paper, results never
 * depend on them):
 *   leaf_cap: records a CTA sorts in shared memory at once (32..2048; at
 *       most the compiled capacity, 1,024 records up to 8-word keys, 512 for
 *       16-word, 256 for 32-word keys; 0 = that capacity);
 *   split_fan: a problem or range larger than a leaf is split into about
 *       split_fan x n / leaf_cap children (1..8; 0 = 2).
 * -1 keeps a value.  A tune-file line "batch leaf_cap split_fan" sets them
 * too.  Errors: INVALID_ARG for values out of range.                        */
paulib_status paulib_set_batch_tuning(int32_t leaf_cap, int32_t split_fan);

paulib_status paulib_set_slot_tuning(int32_t key_words, int32_t method, int32_t leaf_cap, int32_t slot_target,
                                     int32_t slot_oversample);

/* Which method produced the calling thread's last canonical product or
 * compress result: *method = 0 slot sort, 1 range sort, -1 none yet;
 * *fallback_bits = the device check bits that made the slot sort hand the
 * call to the range sort (64: an oversized range whose output could reach
 * its own terms, 128: a sub-range above a leaf, 256: a bounded wait expired,
 * 1024/2048: a leaf's or a sample's whole-key order check failed, which needs
 * a 64-bit key-hash collision), 0 otherwise.
 * Errors: INVALID_ARG for NULL pointers.                                    */
paulib_status paulib_last_canon_method(int32_t* method, int32_t* fallback_bits);

/* Measured rates of the pipes this path uses (no counterpart in the paper),
 * for roofline denominators; each from a microbenchmark of independent
 * dependency chains on every SM, timed with CUDA events on `stream`:
 *   out[0] FP64 fused multiply-adds/s, out[1] FP32 fused multiply-adds/s,
 *   out[2] 32-bit three-input logic operations/s (64-bit and-xor chains),
 *   out[3] 32-bit integer adds/s, out[4] population counts/s,
 *   out[5] bytes/s of random 64-byte reads from a 4 MiB (L2-resident) table,
 *   out[6] the same for 32-byte reads.
 * Writes min(n, 7) values; takes about a second.  Synchronises `stream`.
 * Errors: INVALID_ARG (NULL or n < 1), OOM, CUDA.                            */
paulib_status paulib_measure_peaks(double* out, int32_t n, void* stream);

/* Test settings (no counterpart in the paper; 0 turns a setting off, the
 * default).  Results never depend on them except as stated.
 *   knob 1, value 1..63: the range sort's warp leaves keep only the low
 *     `value` bits of their 64-bit key hashes, so different keys of a leaf
 *     share hashes and the leaf takes its whole-key path (the same result).
 *   knob 2, value 1..4096: a range CTA's worklist holds `value` entries; a
 *     split that needs more sets the device error word and returns, and the
 *     call fails with PAULIB_ERR_INTERNAL (no result).
 *   knob 3, value 1: batched products and batch plans made afterwards take
 *     the general multi-kernel pipeline even where the persistent kernel
 *     applies (the same result).
 *   knob 4, value 32..2048: leaf capacity of the persistent batched kernel
 *     for plans made afterwards (at most its compiled capacity: 1024 records
 *     up to 8-word keys, 512 for 16-word, 256 for 32-word keys); a small
 *     capacity makes small problems take its split path (the same result).
 * Errors: INVALID_ARG for an unknown knob or a value out of range.          */
paulib_status paulib_set_debug(int32_t knob, int64_t value);

/* Shape of the calling thread's last slot sort, for tuning/* Shape of the calling thread's last slot sort, for tuning: stats[0] coarse
 * ranges, [1] slot capacity per range, [2] leaves, [3] terms per leaf (the
 * capacity), [4] mean terms per slot aimed at.  All zero before the first
 * slot sort.  No counterpart in the paper.  Errors: INVALID_ARG (NULL).      */
paulib_status paulib_last_canon_stats(int64_t* stats);

/* Element-wise products: output term t = a_t * b_t, the paper's single
 * Pauli-string multiplication (Sec. III-A, III-E) applied to |a| pairs at
 * once.  Requires |a| == |b| and equal qubit counts.  The output is a new raw
 * sum (*out, owned by the caller): term t holds the product string, the
 * coefficient c_a c_b and the phase exponent k (both inputs' phases
 * included), exactly as a raw outer-product term.
 * Errors: INVALID_ARG (NULL, different lengths), QUBIT_MISMATCH, OOM, CUDA.
 * Asynchronous on `stream`.                                                  */
paulib_status paulib_multiply_pairwise(const paulib_sum* a, const paulib_sum* b, void* stream, paulib_sum** out);

/* ---- Gates and rotations (Sec. III-B; gate application of Sec. V-B).
 * A term is c * i^phase * P where P is a Hermitian Pauli string; a gate acts
 * by conjugation Q -> U Q U^dagger.                                          */
typedef enum {
    PAULIB_GATE_H = 0,    /* Hadamard on qubit q1: X <-> Z, Y -> -Y              */
    PAULIB_GATE_S = 1,    /* phase gate diag(1, i) on q1: X -> Y, Y -> -X        */
    PAULIB_GATE_CNOT = 2, /* control q1, target q2: X_1 -> X_1 X_2, Z_2 -> Z_1 Z_2 */
    PAULIB_GATE_CZ = 3    /* on q1, q2: X_1 -> X_1 Z_2, X_2 -> Z_1 X_2           */
} paulib_gate;

/* Conjugates every term of `s`, in place, by the Clifford gates of a gate
 * list applied in order (the first gate first).  `gates` is a HOST array of
 * n_gates triples (paulib_gate, q1, q2); q2 is ignored by one-qubit gates.
 * Each term keeps its place; strings are relabelled and coefficients change
 * sign where the image is -P, so the number of terms never changes (Sec.
 * III-B, Clifford case).  A canonical sum is no longer sorted afterwards and is
 * marked non-canonical (paulib_compress restores the order).  Every term is
 * read and written once per call, whatever the list's length.
 * Errors: PAULIB_ERR_INVALID_ARG for a NULL sum or list, an unknown gate, a
 * qubit outside [0, n_qubits), or q1 == q2 in a two-qubit gate; nothing is
 * changed then.  Asynchronous on `stream`.                                    */
paulib_status paulib_apply_clifford(paulib_sum* s, int32_t n_gates, const int32_t* gates, void* stream);

/* One step of Pauli propagation under the rotation U_P(theta) =
 * exp(-i theta P / 2) (Sec. III-B): every term Q of `s` that commutes with P
 * is kept; every term that anti-commutes becomes cos(theta) Q and
 * -i sin(theta) P Q (the non-Clifford case; theta = pi and pi/2 give the
 * Pauli and Clifford cases).  The result is returned in canonical form
 * (duplicates merged, Sec. III-H) in a new sum *out, after dropping merged
 * terms with |c| < threshold (truncation; threshold <= 0 keeps every term,
 * including exact zeros).
 *   p_x, p_z: the generator P as ceil(n/64) words each, host or device
 *     memory (bit q%64 of word q/64 = qubit q; bits >= n_qubits must be 0).
 *   precision: as for paulib_multiply (the merge's arithmetic).
 * Errors: INVALID_ARG (NULL arguments), TAIL_BITS (a generator bit at a
 * qubit >= n_qubits), UNSUPPORTED (2^32 or more terms after the split),
 * OOM, CUDA.  Synchronises `stream` (the output size is data dependent).     */
paulib_status paulib_rotate(const paulib_sum* s, const uint64_t* p_x, const uint64_t* p_z, double theta,
                            double threshold, int32_t precision, void* stream, paulib_sum** out);

/* Greedy commutation grouping (Sec. V-D; the sequential variant of Sec.
 * IV-C): partitions the terms of `s` into groups of mutually commuting
 * strings.  The terms are visited in their order; each joins the first group
 * (groups are numbered in the order they are opened) all of whose members
 * commute with it, or opens a new group when none qualifies.  Two strings
 * commute when their symplectic inner product is even (Sec. III-F);
 * coefficients and phases play no part, and repeated strings are fine.
 *   group_of_term: DEVICE int32[n_terms]; receives the group of every term
 *     (may be NULL for an empty sum).
 *   group_offsets: NULL, or DEVICE int32[n_groups + 1] (n_terms + 1 always
 *     suffices): the first member slot of each group, then n_terms.
 *   members: NULL, or DEVICE int32[n_terms]: the terms of group 0 in
 *     increasing order, then those of group 1, and so on (group g's are
 *     members[group_offsets[g] .. group_offsets[g+1])).
 *   n_groups: HOST; receives the number of groups.
 * Scratch: about n_terms^2 / 16 bytes of device memory for the
 * anti-commutation bits.
 * Errors: INVALID_ARG (NULL sum, group_of_term or n_groups), UNSUPPORTED
 * (more than 4,194,240 terms, or a partition into more than 32,704 groups),
 * OOM, CUDA.  Synchronises `stream` (n_groups is returned on the host).      */
paulib_status paulib_group_commuting(const paulib_sum* s, int32_t* group_of_term, int32_t* group_offsets,
                                     int32_t* members, int64_t* n_groups, void* stream);

/* Grouping tuning (no counterpart in the paper; results never depend on
 * it): the number of available groups, 1..4 (default 4), that each term
 * keeps when its 64-term block starts.  A term whose kept groups are all
 * taken by earlier anti-commuting terms of its block scans its whole
 * availability row instead.  Errors: INVALID_ARG outside 1..4.              */
paulib_status paulib_set_group_candidates(int32_t k);

/* Diagnostics (no counterpart in the paper): device time of the library's
 * stages measured with CUDA events recorded on the launching stream, and the
 * number of kernels launched per stage.  Stages:
 *   0 input conversion, 1 splitter sampling and selection, 2 coarse count,
 *   3 coarse scatter, 4 range splitting (the per-range worklist kernel),
 *   5 output compaction, 6 raw outer product, 7 export, 8 leaf sort + merge,
 *   9 commutation grouping, 10 fine splitting of the slot sort (sample,
 *   splitters, locating every record), 11 slot offsets, leaf packing and
 *   term placement of the slot sort.
 * paulib_timing_enable(1) starts recording (0 stops).  paulib_timing_read
 * waits for recorded events, adds their times to ms[PAULIB_STAGES] and the
 * launch counts to launches[PAULIB_STAGES] (either may be NULL), and clears
 * the totals when `reset` is nonzero.  Launch counts are kept even when
 * event timing is off.                                                      */
#define PAULIB_STAGES 12
paulib_status paulib_timing_enable(int32_t on);
paulib_status paulib_timing_read(double* ms, int64_t* launches, int32_t reset);

#ifdef __cplusplus
}
#endif
#endif /* PAULIB_H */
