// occ_dist.cu -- occupancy pyramid and occupancy distance grid G (Sec. 3.3, Eq. 9;
// Sec. S2.5).  Integer work, bit-exact.
//
// G(p) = min(255, floor(sqrt(D2(p)))), D2(p) = min over occupied q of
// sum_a max(|p_a - q_a| - 1, 0)^2: the squared distance between voxel boxes.
// The sum is separable, so D2 is three exact 1-D minimisations, one per axis;
// each pass is one thread per voxel scanning its grid line (O(R) per voxel),
// with the line staged in shared memory.
#include <algorithm>

#include "common.cuh"

namespace ngprt {
namespace {

constexpr int32_t kInf = 0x3fffffff;

__device__ __forceinline__ int32_t gap2(int k) {
    int g = (k < 0 ? -k : k) - 1;
    return g > 0 ? g * g : 0;
}

// Level 0 of the pyramid: one thread packs 32 consecutive voxels into a word.
__global__ void pack_bits_kernel(const uint8_t* __restrict__ occ, size_t n_vox, uint32_t* __restrict__ bits,
                                 size_t n_words) {
    size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n_words) return;
    uint32_t v = 0;
    for (int b = 0; b < 32; ++b) {
        size_t i = w * 32 + b;
        if (i < n_vox && occ[i]) v |= 1u << b;
    }
    bits[w] = v;
}

// Level k+1 from level k: one thread per output word, OR of the 8 children of
// each of its 32 voxels.
__global__ void downsample_kernel(const uint32_t* __restrict__ fine, int rf, uint32_t* __restrict__ coarse, int rc,
                                  size_t n_words) {
    size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n_words) return;
    const size_t n_vox = (size_t)rc * rc * rc;
    uint32_t v = 0;
    for (int b = 0; b < 32; ++b) {
        size_t i = w * 32 + b;
        if (i >= n_vox) break;
        int x = (int)(i % rc), y = (int)((i / rc) % rc), z = (int)(i / ((size_t)rc * rc));
        uint32_t any = 0;
        for (int c = 0; c < 8; ++c) {
            size_t fx = 2 * x + (c & 1), fy = 2 * y + ((c >> 1) & 1), fz = 2 * z + ((c >> 2) & 1);
            size_t fi = fx + (size_t)rf * (fy + (size_t)rf * fz);
            any |= (fine[fi >> 5] >> (fi & 31)) & 1u;
        }
        v |= any << b;
    }
    coarse[w] = v;
}

// Pass along axis `axis` (0 = x, 1 = y, 2 = z).  Block = one grid line of R voxels
// along that axis (R threads); the line's input values sit in shared memory.
// Pass 0 reads occupancy (0 -> inf, else 0); the others read the previous pass.
__global__ void edt_pass_kernel(const uint8_t* __restrict__ occ, const int32_t* __restrict__ in,
                                int32_t* __restrict__ out, int R, int axis) {
    extern __shared__ int32_t line[];
    const int line_id = blockIdx.x;           // which line: the two other coordinates
    const int a = line_id % R, b = line_id / R;
    const size_t stride = axis == 0 ? 1 : (axis == 1 ? (size_t)R : (size_t)R * R);
    size_t base;
    if (axis == 0) base = (size_t)R * (a + (size_t)R * b);          // (y=a, z=b)
    else if (axis == 1) base = (size_t)a + (size_t)R * R * b;       // (x=a, z=b)
    else base = (size_t)a + (size_t)R * b;                          // (x=a, y=b)
    for (int i = threadIdx.x; i < R; i += blockDim.x) {
        size_t idx = base + stride * i;
        line[i] = in ? in[idx] : (occ[idx] ? 0 : kInf);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < R; i += blockDim.x) {
        int32_t best = kInf;
        for (int q = 0; q < R; ++q) {
            int32_t v = line[q];
            if (v < kInf) best = min(best, v + gap2(i - q));
        }
        out[base + stride * i] = best;
    }
}

// Unpack one pyramid level (n voxels) to one byte per voxel, the input of the
// distance transform when G sits on a coarser level than the finest.
__global__ void unpack_bits_kernel(const uint32_t* __restrict__ bits, size_t n, uint8_t* __restrict__ out) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = (uint8_t)((bits[i >> 5] >> (i & 31)) & 1u);
}

__global__ void finish_dist_kernel(const int32_t* __restrict__ d2, size_t n, uint8_t* __restrict__ dist) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t v = d2[i];
    int32_t g;
    if (v >= kInf) {
        g = 255;
    } else {
        int32_t s = (int32_t)sqrtf((float)v);
        while (s * s > v) --s;
        while ((s + 1) * (s + 1) <= v) ++s;
        g = s < 255 ? s : 255;
    }
    dist[i] = (uint8_t)g;
}

size_t words(size_t bits) { return (bits + 31) / 32; }

}  // namespace
}  // namespace ngprt

using namespace ngprt;

extern "C" size_t ngprt_occ_bits_words(int32_t R, int32_t n_levels) {
    if (R <= 0 || n_levels <= 0) return 0;
    size_t total = 0;
    for (int k = 0; k < n_levels; ++k) {
        size_t r = (size_t)(R >> k);
        total += words(r * r * r);
    }
    return total;
}

extern "C" size_t ngprt_build_occ_dist_workspace_bytes(int32_t R) {
    if (R <= 0) return 0;
    size_t n = (size_t)R * R * R;
    return 2 * ((n * sizeof(int32_t) + 255) / 256 * 256);
}

extern "C" int32_t ngprt_build_occ_dist(const uint8_t* occ, int32_t R, int32_t n_levels, int32_t dist_level,
                                        uint32_t* occ_bits_out, uint8_t* dist_out, void* workspace, size_t ws_bytes,
                                        void* stream) {
    NGPRT_REQUIRE(occ != nullptr, "ngprt_build_occ_dist: occ is NULL");
    NGPRT_REQUIRE(occ_bits_out != nullptr, "ngprt_build_occ_dist: occ_bits_out is NULL");
    NGPRT_REQUIRE(R >= 2 && R <= 1024 && (R & (R - 1)) == 0, "ngprt_build_occ_dist: R=%d must be a power of two in [2, 1024]", R);
    NGPRT_REQUIRE(n_levels >= 1 && n_levels <= kMaxOccLevels && (R >> (n_levels - 1)) >= 1,
                  "ngprt_build_occ_dist: n_levels=%d invalid for R=%d", n_levels, R);
    NGPRT_REQUIRE(dist_level >= 0 && dist_level < n_levels, "ngprt_build_occ_dist: dist_level=%d not in [0, %d)",
                  dist_level, n_levels);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t n = (size_t)R * R * R;
    // pyramid
    size_t w0 = words(n);
    pack_bits_kernel<<<(unsigned)((w0 + 255) / 256), 256, 0, st>>>(occ, n, occ_bits_out, w0);
    size_t off_prev = 0, off = w0, dist_off = 0;
    for (int k = 1; k < n_levels; ++k) {
        int rf = R >> (k - 1), rc = R >> k;
        size_t wk = words((size_t)rc * rc * rc);
        downsample_kernel<<<(unsigned)((wk + 127) / 128), 128, 0, st>>>(occ_bits_out + off_prev, rf,
                                                                         occ_bits_out + off, rc, wk);
        if (k == dist_level) dist_off = off;
        off_prev = off;
        off += wk;
    }
    if (dist_out) {
        size_t need = ngprt_build_occ_dist_workspace_bytes(R);
        if (workspace == nullptr || ws_bytes < need) {
            set_error("ngprt_build_occ_dist: workspace %zu bytes < %zu needed", ws_bytes, need);
            return NGPRT_ERR_WORKSPACE;
        }
        NGPRT_REQUIRE(((uintptr_t)workspace & 255) == 0, "ngprt_build_occ_dist: workspace not 256-byte aligned");
        // G on level dist_level: its voxels' occupancy (finest occ, or the level's
        // pyramid bits unpacked into the second half of the workspace)
        const int Rg = R >> dist_level;
        const size_t ng = (size_t)Rg * Rg * Rg;
        int32_t* a = static_cast<int32_t*>(workspace);
        int32_t* b = reinterpret_cast<int32_t*>(static_cast<char*>(workspace) + need / 2);
        const uint8_t* src = occ;
        if (dist_level > 0) {
            // (R/2)^3 bytes fit after a's (R/2)^3 ints in the first half (R^3 ints)
            uint8_t* u8 = reinterpret_cast<uint8_t*>(a + ng);
            unpack_bits_kernel<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(occ_bits_out + dist_off, ng, u8);
            src = u8;
        }
        const unsigned lines = (unsigned)((size_t)Rg * Rg);
        const int threads = std::min(Rg, 256);
        const size_t shm = (size_t)Rg * sizeof(int32_t);
        edt_pass_kernel<<<lines, threads, shm, st>>>(src, nullptr, b, Rg, 0);
        edt_pass_kernel<<<lines, threads, shm, st>>>(nullptr, b, a, Rg, 1);
        edt_pass_kernel<<<lines, threads, shm, st>>>(nullptr, a, b, Rg, 2);
        finish_dist_kernel<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(b, ng, dist_out);
    }
    return cuda_status("ngprt_build_occ_dist");
}
