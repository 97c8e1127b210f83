// coarse_sparse.cu -- the block-indexed sparse coarse grid (the baked 512^3 grid of
// Sec. 3.1 is stored sparse, about 2% occupied, Eq. S1).  Cells are grouped in 8^3
// blocks; a stored block keeps the 9^3 vertices of its cells, so a sample's 8
// corners always sit in the block of its cell (one index lookup, coarse_base in
// common.cuh).  The blocks kept are those a render can reach: every cell overlapped
// by an occupied voxel of the finest occupancy level, widened by one cell.
#include "common.cuh"

namespace ngprt {
namespace {

constexpr int kChunk = 1024;  // index entries per block of the count / index kernels

__host__ __device__ inline uint32_t blocks_per_axis(int R_C) {
    return (uint32_t)((R_C - 1 + NGPRT_COARSE_BLOCK - 1) / NGPRT_COARSE_BLOCK);
}

// One thread per word of the finest occupancy level: each occupied voxel marks the
// blocks of the coarse cells its u-range overlaps, one cell wider on each side.
__global__ void block_mask_kernel(const uint32_t* __restrict__ bits, int R_O, int R_C, uint32_t nb,
                                  uint8_t* __restrict__ mask) {
    const uint64_t n_vox = (uint64_t)R_O * R_O * R_O;
    const uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w * 32 >= n_vox) return;
    uint32_t word = bits[w];
    while (word) {
        const int bit = __ffs(word) - 1;
        word &= word - 1;
        const uint64_t i = w * 32 + (uint64_t)bit;
        if (i >= n_vox) break;
        const int v[3] = {(int)(i % R_O), (int)((i / R_O) % R_O), (int)(i / ((uint64_t)R_O * R_O))};
        int lo[3], hi[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int c0 = (int)(((int64_t)v[a] * (R_C - 1)) / R_O) - 1;
            const int c1 = (int)(((int64_t)(v[a] + 1) * (R_C - 1)) / R_O) + 1;
            lo[a] = max(c0, 0) >> 3;
            hi[a] = min(c1, R_C - 2) >> 3;
        }
        for (int z = lo[2]; z <= hi[2]; ++z)
            for (int y = lo[1]; y <= hi[1]; ++y)
                for (int x = lo[0]; x <= hi[0]; ++x) mask[(uint32_t)x + nb * ((uint32_t)y + nb * (uint32_t)z)] = 1;
    }
}

// Marked entries per chunk of kChunk index entries.
__global__ void count_kernel(const uint8_t* __restrict__ mask, uint64_t n, int32_t* __restrict__ counts) {
    int c = 0;
    for (int k = threadIdx.x; k < kChunk; k += blockDim.x) {
        const uint64_t i = (uint64_t)blockIdx.x * kChunk + k;
        c += (i < n && mask[i]) ? 1 : 0;
    }
    __shared__ int s[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s[k];
        counts[blockIdx.x] = t;
    }
}

// Exclusive prefix of the chunk counts (a few thousand at most) and the total.
__global__ void scan_counts_kernel(const int32_t* __restrict__ counts, int n_chunks, int32_t* __restrict__ offsets,
                                   int64_t* __restrict__ total) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t acc = 0;
    for (int k = 0; k < n_chunks; ++k) {
        offsets[k] = (int32_t)acc;
        acc += counts[k];
    }
    *total = acc;
}

// Slots in index order: marked entry j of the grid gets 1 + j, unmarked ones 0.
// Each of the 256 threads of a chunk owns 4 consecutive entries.
__global__ void __launch_bounds__(256) index_kernel(const uint8_t* __restrict__ mask, uint64_t n,
                                                    const int32_t* __restrict__ offsets, int32_t* __restrict__ index) {
    __shared__ int32_t part[256];
    const uint64_t i0 = (uint64_t)blockIdx.x * kChunk + 4 * threadIdx.x;
    int f[4], c = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        f[k] = (i0 + k < n && mask[i0 + k]) ? 1 : 0;
        c += f[k];
    }
    part[threadIdx.x] = c;
    __syncthreads();
    // Hillis-Steele inclusive scan over the 256 thread counts
    for (int o = 1; o < 256; o <<= 1) {
        const int32_t add = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += add;
        __syncthreads();
    }
    int32_t slot = 1 + offsets[blockIdx.x] + part[threadIdx.x] - c;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (i0 + k < n) index[i0 + k] = f[k] ? slot : 0;
        slot += f[k];
    }
}

// One CTA per index entry: a marked block copies its 9^3 vertex rows (4-byte words)
// from the dense grid, zero past the grid's last vertex.
__global__ void gather_blocks_kernel(const uint32_t* __restrict__ dense, int R_C, int row_words, uint32_t nb,
                                     const int32_t* __restrict__ index, uint32_t* __restrict__ blocks) {
    const uint32_t e = blockIdx.x;
    const int32_t s = index[e];
    if (s <= 0) return;
    const uint32_t bx = e % nb, by = (e / nb) % nb, bz = e / (nb * nb);
    const int n_words = NGPRT_COARSE_BLOCK_ROWS * row_words;
    uint32_t* out = blocks + (size_t)s * n_words;
    for (int k = threadIdx.x; k < n_words; k += blockDim.x) {
        const int r = k / row_words, c = k - r * row_words;
        const int li = r % 9, lj = (r / 9) % 9, lk = r / 81;
        const int x = (int)bx * NGPRT_COARSE_BLOCK + li, y = (int)by * NGPRT_COARSE_BLOCK + lj,
                  z = (int)bz * NGPRT_COARSE_BLOCK + lk;
        uint32_t v = 0;
        if (x < R_C && y < R_C && z < R_C)
            v = dense[((size_t)x + (size_t)R_C * ((size_t)y + (size_t)R_C * (size_t)z)) * row_words + c];
        out[k] = v;
    }
}

}  // namespace

int32_t make_occ(const ngprt_occ* o, OccView& v, const char* fn);

}  // namespace ngprt

using namespace ngprt;

extern "C" int32_t ngprt_coarse_block_mask(const ngprt_occ* occ, int32_t R_C, uint8_t* block_mask, void* stream) {
    const char* fn = "ngprt_coarse_block_mask";
    OccView v;
    int32_t rc;
    if ((rc = make_occ(occ, v, fn)) != NGPRT_OK) return rc;
    NGPRT_REQUIRE(R_C >= 2 && R_C <= 1024, "%s: R_C=%d not in [2, 1024]", fn, R_C);
    NGPRT_REQUIRE(block_mask != nullptr, "%s: block_mask is NULL", fn);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint32_t nb = blocks_per_axis(R_C);
    cudaMemsetAsync(block_mask, 0, (size_t)nb * nb * nb, st);
    const uint64_t n_words = ((uint64_t)v.R_O * v.R_O * v.R_O + 31) / 32;
    block_mask_kernel<<<(unsigned)((n_words + 255) / 256), 256, 0, st>>>(v.bits, v.R_O, R_C, nb, block_mask);
    return cuda_status(fn);
}

extern "C" size_t ngprt_coarse_sparsify_workspace_bytes(int32_t R_C) {
    if (R_C < 2 || R_C > 1024) return 0;
    const uint64_t nb = blocks_per_axis(R_C);
    const uint64_t n_chunks = (nb * nb * nb + kChunk - 1) / kChunk;
    return (size_t)(16 + ((2 * n_chunks * sizeof(int32_t) + 15) / 16) * 16);
}

extern "C" int32_t ngprt_coarse_sparsify(const void* dense, int32_t R_C, int32_t row_bytes, const uint8_t* block_mask,
                                         int32_t* index, void* blocks, int64_t max_blocks, int64_t* n_blocks,
                                         void* workspace, size_t ws_bytes, void* stream) {
    const char* fn = "ngprt_coarse_sparsify";
    NGPRT_REQUIRE(R_C >= 2 && R_C <= 1024, "%s: R_C=%d not in [2, 1024]", fn, R_C);
    NGPRT_REQUIRE(row_bytes > 0 && row_bytes % 4 == 0, "%s: row_bytes=%d must be a positive multiple of 4", fn,
                  row_bytes);
    NGPRT_REQUIRE(block_mask && index && n_blocks, "%s: NULL buffer", fn);
    NGPRT_REQUIRE(!blocks || (dense && ((uintptr_t)dense & 3) == 0 && ((uintptr_t)blocks & 3) == 0),
                  "%s: dense and blocks must be 4-byte aligned", fn);
    NGPRT_REQUIRE(((uintptr_t)index & 3) == 0, "%s: index must be 4-byte aligned", fn);
    const size_t need = ngprt_coarse_sparsify_workspace_bytes(R_C);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace & 15) != 0) {
        set_error("%s: workspace %zu bytes < %zu needed (16-byte aligned)", fn, ws_bytes, need);
        return NGPRT_ERR_WORKSPACE;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint32_t nb = blocks_per_axis(R_C);
    const uint64_t n = (uint64_t)nb * nb * nb;
    const int n_chunks = (int)((n + kChunk - 1) / kChunk);
    char* ws = static_cast<char*>(workspace);
    int64_t* total = reinterpret_cast<int64_t*>(ws);
    int32_t* counts = reinterpret_cast<int32_t*>(ws + 16);
    int32_t* offsets = counts + n_chunks;
    count_kernel<<<n_chunks, 256, 0, st>>>(block_mask, n, counts);
    scan_counts_kernel<<<1, 1, 0, st>>>(counts, n_chunks, offsets, total);
    index_kernel<<<n_chunks, 256, 0, st>>>(block_mask, n, offsets, index);
    int64_t marked = 0;
    cudaMemcpyAsync(&marked, total, sizeof marked, cudaMemcpyDeviceToHost, st);
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_error("%s: CUDA error %s (%s)", fn, cudaGetErrorName(e), cudaGetErrorString(e));
        return NGPRT_ERR_CUDA;
    }
    int32_t rc;
    if ((rc = cuda_status(fn)) != NGPRT_OK) return rc;
    *n_blocks = 1 + marked;
    if (!blocks) return NGPRT_OK;
    if (*n_blocks > max_blocks) {
        set_error("%s: %lld blocks needed, room for %lld", fn, (long long)*n_blocks, (long long)max_blocks);
        return NGPRT_ERR_WORKSPACE;
    }
    const int row_words = row_bytes / 4;
    cudaMemsetAsync(blocks, 0, (size_t)NGPRT_COARSE_BLOCK_ROWS * row_bytes, st);
    gather_blocks_kernel<<<(unsigned)n, 128, 0, st>>>(static_cast<const uint32_t*>(dense), R_C, row_words, nb, index,
                                                      static_cast<uint32_t*>(blocks));
    return cuda_status(fn);
}
