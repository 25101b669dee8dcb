// paulib_peaks.cu -- microbenchmarks of the pipes the Pauli-product path uses
// (paulib_measure_peaks): FP64 and FP32 fused multiply-add, 64-bit logic and
// integer adds, population counts, and random gathers of 64- and 32-byte
// pieces from an L2-resident table.  They give the denominators of the
// roofline of a path that is not a dense contraction.  No counterpart in the
// paper.
#include "paulib_internal.h"

namespace paulib {
namespace {

constexpr int kChains = 8;  // independent dependency chains per thread

__global__ void k_peak_dfma(double* out, int iters) {
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 1e-3 * (threadIdx.x + c);
    const double b = 0.999999999, d = 1e-9;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], b, d);
    double s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == -1.0) out[0] = s;  // never true; keeps the chains alive
}

__global__ void k_peak_ffma(float* out, int iters) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 1e-3f * (threadIdx.x + c);
    const float b = 0.9999999f, d = 1e-7f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], b, d);
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == -1.0f) out[0] = s;
}

// x = (x & y) ^ z on 64-bit words: two 32-bit three-input logic operations
// per step.
__global__ void k_peak_lop(uint64_t* out, int iters) {
    uint64_t a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 0x9e3779b97f4a7c15ull * (threadIdx.x + c + 1);
    const uint64_t y = 0xf0f0f0f0f0f0f0f0ull ^ blockIdx.x, z = 0x0123456789abcdefull;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = (a[c] & (y ^ (uint64_t)c)) ^ (z + (uint64_t)i);
    uint64_t s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= a[c];
    if (s == 1ull) out[0] = s;
}

__global__ void k_peak_iadd(uint32_t* out, int iters) {
    uint32_t a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = threadIdx.x + c;
    const uint32_t y = blockIdx.x | 1u;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = a[c] + (y ^ (uint32_t)c);
    uint32_t s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= a[c];
    if (s == 1u) out[0] = s;
}

// x = x + popc(x ^ k): one population count and two simple integer
// operations per step.
__global__ void k_peak_popc(uint32_t* out, int iters) {
    uint32_t a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 0x9e3779b9u * (threadIdx.x + c + 1);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] += (uint32_t)__popc(a[c] ^ (uint32_t)i);
    uint32_t s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= a[c];
    if (s == 1u) out[0] = s;
}

// Random reads of PIECE-byte pieces (16-byte vector loads) from a table of
// `entries` pieces: each thread keeps 8 independent reads in flight.
template <int PIECE>
__global__ void k_peak_gather(const ulonglong2* __restrict__ tab, uint32_t entries, int iters, uint64_t* out) {
    constexpr int Q = PIECE / 16;
    uint64_t s = 0;
    uint64_t h = 0x9e3779b97f4a7c15ull * (blockIdx.x * blockDim.x + threadIdx.x + 1);
    for (int i = 0; i < iters; ++i) {
        uint32_t idx[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            h ^= h >> 29;
            h *= 0xbf58476d1ce4e5b9ull;
            idx[c] = (uint32_t)(h >> 32) % entries;
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c)
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const ulonglong2 v = __ldg(tab + (size_t)idx[c] * Q + q);
                s += v.x ^ v.y;
            }
    }
    if (s == 1ull) out[0] = s;
}

template <class F>
double time_kernel(F&& launch, cudaStream_t st) {
    cudaEvent_t a, b;
    check_cuda(cudaEventCreate(&a), "event");
    check_cuda(cudaEventCreate(&b), "event");
    launch();  // warm-up
    check_cuda(cudaEventRecord(a, st), "event record");
    launch();
    check_cuda(cudaEventRecord(b, st), "event record");
    check_cuda(cudaEventSynchronize(b), "event sync");
    float ms = 0;
    check_cuda(cudaEventElapsedTime(&ms, a, b), "elapsed");
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    check_cuda(cudaGetLastError(), "peak kernel");
    return ms * 1e-3;
}

}  // namespace

void measure_peaks(double* out, int n, cudaStream_t st) {
    const int sms = device_sm_count();
    const unsigned grid = (unsigned)sms * 8u, block = 256;
    const double threads = (double)grid * block;
    const int iters = 4096;
    Scratch sink(64, st);
    double r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    r[0] = threads * iters * kChains /
           time_kernel([&] { k_peak_dfma<<<grid, block, 0, st>>>(sink.as<double>(), iters); }, st);
    r[1] = threads * iters * kChains /
           time_kernel([&] { k_peak_ffma<<<grid, block, 0, st>>>(sink.as<float>(), iters); }, st);
    r[2] = threads * iters * kChains * 2 /
           time_kernel([&] { k_peak_lop<<<grid, block, 0, st>>>(sink.as<uint64_t>(), iters); }, st);
    r[3] = threads * iters * kChains /
           time_kernel([&] { k_peak_iadd<<<grid, block, 0, st>>>(sink.as<uint32_t>(), iters); }, st);
    r[4] = threads * iters * kChains /
           time_kernel([&] { k_peak_popc<<<grid, block, 0, st>>>(sink.as<uint32_t>(), iters); }, st);
    // a 4 MiB table (the size of the factor tables of a 30,000-term sum at
    // 200 qubits) stays in L2
    const size_t tab_bytes = (size_t)4 << 20;
    Scratch tab(tab_bytes, st);
    check_cuda(cudaMemsetAsync(tab.p, 1, tab_bytes, st), "memset table");
    const int giters = 64;
    r[5] = threads * giters * kChains * 64.0 /
           time_kernel([&] {
               k_peak_gather<64><<<grid, block, 0, st>>>(tab.as<ulonglong2>(), (uint32_t)(tab_bytes / 64), giters,
                                                         sink.as<uint64_t>());
           }, st);
    r[6] = threads * giters * kChains * 32.0 /
           time_kernel([&] {
               k_peak_gather<32><<<grid, block, 0, st>>>(tab.as<ulonglong2>(), (uint32_t)(tab_bytes / 32), giters,
                                                         sink.as<uint64_t>());
           }, st);
    for (int q = 0; q < n && q < 7; ++q) out[q] = r[q];
}

}  // namespace paulib
