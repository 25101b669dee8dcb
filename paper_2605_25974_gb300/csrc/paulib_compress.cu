// paulib_compress.cu -- canonical form of one sum (paulib_compress,
// PauLIB Sec. III-H sort_and_combine); the pipeline is in paulib_pipeline.cuh.
#include "paulib_slots.cuh"

namespace paulib {

paulib_sum* canon_terms(const paulib_sum* in, int mode, cudaStream_t st) {
    if (in->n_terms == 0) return empty_canonical(in->n_qubits, st);
    if (in->n_terms >= ((int64_t)1 << 32) - 1) fail(PAULIB_ERR_UNSUPPORTED, "compress needs < 2^32 terms");
#define L(WP)                                                    \
    {                                                            \
        if (mode == M_FP64) return terms_mode<WP, M_FP64>(in, st); \
        if (mode == M_F32_D64) return terms_mode<WP, M_F32_D64>(in, st); \
        return terms_mode<WP, M_F32_TWOSUM>(in, st);             \
    }
    PAULIB_DISPATCH_WP(in->WP, L);
#undef L
    return nullptr;
}

}  // namespace paulib
