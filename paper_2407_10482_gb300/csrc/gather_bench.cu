// gather_bench.cu -- measured ceiling of the render's dominant access: random
// gathers of whole 8-channel table entries (32 B in FP32 with one 256-bit load,
// 16 B in FP16 with one 128-bit load) from a table of a given footprint.  With a
// small table the rows stay in L1 and the rate is the L1 load-return bandwidth;
// with the hd table footprint it is the L2 / HBM random-gather rate.  Each thread
// draws rows from a counter-based hash of (seed, thread, step) and sums them into
// a sink so the loads cannot be dropped.
#include "common.cuh"

namespace ngprt {
namespace {

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

template <int DT>
__global__ void __launch_bounds__(256) gather_kernel(const void* table, uint32_t rows_mask, int per_thread,
                                                     uint32_t seed, float* sink) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    uint32_t h = mix32(seed ^ (tid * 0x9e3779b9u));
    for (int i = 0; i < per_thread; i += 8) {
        float e[8][8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            h = mix32(h + (uint32_t)k);
            load_entry<DT>(table, h & rows_mask, e[k]);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] += e[k][c];
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += acc[c];
    if (s == 1234.5678f) sink[0] = s;  // never true for the benches' tables; keeps the loads alive
}

}  // namespace
}  // namespace ngprt

using namespace ngprt;

extern "C" int32_t ngprt_gather_bench(const void* table, int32_t dtype, int64_t n_rows, int64_t n_threads,
                                      int32_t per_thread, uint32_t seed, float* sink, void* stream) {
    const char* fn = "ngprt_gather_bench";
    NGPRT_REQUIRE(table && sink, "%s: NULL buffer", fn);
    NGPRT_REQUIRE(n_rows >= 1 && (n_rows & (n_rows - 1)) == 0 && n_rows <= ((int64_t)1 << 31),
                  "%s: n_rows must be a power of two", fn);
    NGPRT_REQUIRE(n_threads >= 256 && n_threads % 256 == 0 && per_thread >= 8 && per_thread % 8 == 0,
                  "%s: n_threads a multiple of 256, per_thread a multiple of 8", fn);
    NGPRT_REQUIRE(dtype == NGPRT_F32 || dtype == NGPRT_F16, "%s: dtype F32 or F16", fn);
    NGPRT_REQUIRE(((uintptr_t)table & 31) == 0, "%s: table must be 32-byte aligned", fn);
    const unsigned blocks = (unsigned)(n_threads / 256);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (dtype == NGPRT_F32)
        gather_kernel<NGPRT_F32><<<blocks, 256, 0, st>>>(table, (uint32_t)(n_rows - 1), per_thread, seed, sink);
    else
        gather_kernel<NGPRT_F16><<<blocks, 256, 0, st>>>(table, (uint32_t)(n_rows - 1), per_thread, seed, sink);
    return cuda_status(fn);
}
