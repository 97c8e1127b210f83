// gather_bench.cu -- measured ceiling of the render's dominant access: random
// gathers of whole 8-channel table entries (32 B in FP32 with one 256-bit load,
// 16 B in FP16 with one 128-bit load) from a table of a given footprint.  With a
// small table the rows stay in L1 and the rate is the L1 load-return bandwidth;
// with the hd table footprint it is the L2 / HBM random-gather rate.  Each thread
// draws rows from a counter-based sequence of (seed, thread, step) and folds them into
// a sink so the loads cannot be dropped.  flags = 1 reads FP32 entries without L1
// allocation (the march's mode for its large levels).
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

// Row of gather j of a thread: a Weyl sequence (odd stride) scrambled by one
// multiply, so consecutive gathers of a thread and the lanes of a warp touch
// unrelated rows; the 8 gathers of a batch are independent (no serial chain).
__device__ __forceinline__ uint32_t row_of(uint32_t base, uint32_t j, uint32_t mask) {
    return ((base + j * 0x9e3779b9u) * 0x2c1b3c6du >> 7) & mask;
}

template <int DT, bool NA>
__global__ void __launch_bounds__(256) gather_kernel(const void* table, uint32_t rows_mask, int per_thread,
                                                     uint32_t seed, float* sink) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t base = mix32(seed ^ (tid * 0x85ebca6bu));
    uint32_t acc = 0;
    for (int i = 0; i < per_thread; i += 8) {
        float e[8][8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t row = row_of(base, (uint32_t)(i + k), rows_mask);
            if constexpr (NA && DT == NGPRT_F32) load_entry_f32_na(table, row, e[k]);
            else load_entry<DT>(table, row, e[k]);
        }
        // fold the loaded bits with three-way XORs (cheaper than summing 64 floats)
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int c = 0; c < 8; c += 2) acc ^= __float_as_uint(e[k][c]) ^ __float_as_uint(e[k][c + 1]);
    }
    if (acc == 0x7f7ff00du) sink[0] = __uint_as_float(acc);  // practically never; keeps the loads alive
}

}  // namespace
}  // namespace ngprt

using namespace ngprt;

extern "C" int32_t ngprt_gather_bench(const void* table, int32_t dtype, int64_t n_rows, int64_t n_threads,
                                      int32_t per_thread, uint32_t seed, int32_t flags, float* sink, void* stream) {
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
    NGPRT_REQUIRE(flags == 0 || (flags == 1 && dtype == NGPRT_F32), "%s: flags=%d (1: FP32 no-allocate loads)", fn,
                  flags);
    const uint32_t mask = (uint32_t)(n_rows - 1);
    if (dtype == NGPRT_F32 && flags == 1)
        gather_kernel<NGPRT_F32, true><<<blocks, 256, 0, st>>>(table, mask, per_thread, seed, sink);
    else if (dtype == NGPRT_F32)
        gather_kernel<NGPRT_F32, false><<<blocks, 256, 0, st>>>(table, mask, per_thread, seed, sink);
    else
        gather_kernel<NGPRT_F16, false><<<blocks, 256, 0, st>>>(table, mask, per_thread, seed, sink);
    return cuda_status(fn);
}
