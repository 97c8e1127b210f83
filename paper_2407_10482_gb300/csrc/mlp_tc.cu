// mlp_tc.cu -- the deferred MLP_psi (Eq. 5) in FP16 on the 5th-generation tensor
// cores (tcgen05), FP32 accumulation in tensor memory.
//
// Per CTA (128 threads, persistent over tiles of 128 rays): the weights are staged
// once in shared memory as FP16 K-major operands in the canonical no-swizzle
// layout (8 x 8 core matrices of 128 bytes; core matrices adjacent in K are 128 B
// apart, groups of 8 rows are K/8 * 128 B apart).  For each tile, thread r writes
// its ray's input row [C_d, F, SH16(d), 0...] (FP16) as row r of A; one thread
// issues tcgen05.mma (M = 128, N = hidden width, K = 16 per instruction) into TMEM
// and commits to an mbarrier; every warp then reads its 32 TMEM lanes (one row per
// thread) with tcgen05.ld, applies ReLU, and writes the next layer's A.  The last
// layer (N = 16, three used) feeds the colour sigmoid and the background.  Every
// mbarrier wait is bounded: on expiry the kernel records an error, frees its TMEM
// and returns.
#include "common.cuh"

namespace ngprt {

__device__ int g_tc_error = 0;  // set when a tensor-core wait expired

namespace {

constexpr int kTile = 128;
constexpr int kTmemCols = 128;
constexpr int kLastN = 16;

struct MlpTcParams {
    const float* state;
    const __half* w;
    float bg[3];
    int64_t n;
    float* rgb;
    float* depth;
    float* opacity;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (r, k) of an R x K FP16 K-major operand (canonical, no swizzle).
__device__ __forceinline__ uint32_t canon(int r, int k, int K) {
    return (uint32_t)((((r >> 3) * (K >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// Shared-memory matrix descriptor: start >> 4, leading byte offset (K direction)
// >> 4, stride byte offset (8-row groups) >> 4, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D = F32, A = B = F16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// Bounded wait for the mbarrier phase with the given parity; false on expiry.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, int limit = 1 << 24) {
    for (int i = 0; i < limit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

template <int WIDTH, int LAYERS>
struct TcLayout {
    static constexpr int w0 = 0;                                    // WIDTH x 32
    static constexpr int wm = w0 + WIDTH * kMlpIn * 2;              // WIDTH x WIDTH (3 layers)
    static constexpr int wl = wm + (LAYERS == 3 ? WIDTH * WIDTH * 2 : 0);  // 16 x WIDTH
    static constexpr int a0 = wl + kLastN * WIDTH * 2;              // 128 x 32
    static constexpr int a1 = a0 + kTile * kMlpIn * 2;              // 128 x WIDTH
    static constexpr int bar = a1 + kTile * WIDTH * 2;              // mbarrier (8 B) + TMEM slot (4 B)
    static constexpr int bytes = bar + 16;
};

// Issue C[128 x N] (TMEM) = A[128 x K] . B[N x K]^T from one thread, K in steps of 16.
__device__ __forceinline__ void issue_layer(uint32_t tmem_d, uint32_t a_addr, uint32_t b_addr, int K, int N,
                                            uint32_t mbar) {
    const uint32_t sbo = (uint32_t)(K >> 3) << 7;
    const uint32_t id = idesc(kTile, N);
    for (int ks = 0; ks < K / 16; ++ks) {
        const uint32_t off = (uint32_t)ks << 8;  // 16 elements of K = two core matrices
        mma_f16(tmem_d, sdesc(a_addr + off, 128, sbo), sdesc(b_addr + off, 128, sbo), id, ks > 0 ? 1u : 0u);
    }
    mma_commit(mbar);
}

template <int WIDTH, int LAYERS>
__global__ void __launch_bounds__(128) mlp_tc_kernel(const __grid_constant__ MlpTcParams p) {
    using Lay = TcLayout<WIDTH, LAYERS>;
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5;
    // weights -> canonical FP16 operands (rows of the last layer beyond 3 are zero)
    {
        const __half* w = p.w;
        for (int i = tid; i < WIDTH * kMlpIn; i += blockDim.x)
            *reinterpret_cast<__half*>(smem + Lay::w0 + canon(i / kMlpIn, i % kMlpIn, kMlpIn)) = w[i];
        w += WIDTH * kMlpIn;
        if constexpr (LAYERS == 3) {
            for (int i = tid; i < WIDTH * WIDTH; i += blockDim.x)
                *reinterpret_cast<__half*>(smem + Lay::wm + canon(i / WIDTH, i % WIDTH, WIDTH)) = w[i];
            w += WIDTH * WIDTH;
        }
        for (int i = tid; i < kLastN * WIDTH; i += blockDim.x) {
            const int r = i / WIDTH, k = i % WIDTH;
            *reinterpret_cast<__half*>(smem + Lay::wl + canon(r, k, WIDTH)) = r < 3 ? w[r * WIDTH + k] : __float2half(0.f);
        }
    }
    const uint32_t mbar = smem_u32(smem + Lay::bar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + Lay::bar + 8);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t my_lane = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t phase = 0;
    bool ok = true;
    const uint32_t a0 = smem_u32(smem + Lay::a0), a1 = smem_u32(smem + Lay::a1);
    for (int64_t tile = blockIdx.x; tile * kTile < p.n && ok; tile += gridDim.x) {
        const int64_t ray = tile * kTile + tid;
        const bool active = ray < p.n;
        float x[24], A = 0.f, depth = 0.f;
#pragma unroll
        for (int k = 0; k < 24; ++k) x[k] = 0.f;
        if (active) {
            const float4* s4 = reinterpret_cast<const float4*>(p.state + ray * NGPRT_STATE_FLOATS);
            const float4 q0 = s4[0], q1 = s4[1], q2 = s4[2];
            x[0] = q0.x; x[1] = q0.y; x[2] = q0.z; x[3] = q0.w;
            x[4] = q1.x; x[5] = q1.y; x[6] = q1.z;
            A = q1.w;
            depth = q2.x;
            sh16(q2.y, q2.z, q2.w, x + 7);
        }
        // row tid of A0: [x (23), 0 ...] in FP16, 16 bytes (8 elements) at a time
#pragma unroll
        for (int kc = 0; kc < kMlpIn / 8; ++kc) {
            __align__(16) __half h[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) h[e] = __float2half(kc * 8 + e < 24 ? x[(kc * 8 + e) % 24] : 0.f);
            *reinterpret_cast<uint4*>(smem + Lay::a0 + canon(tid, kc * 8, kMlpIn)) = *reinterpret_cast<uint4*>(h);
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        // hidden layers
#pragma unroll
        for (int layer = 0; layer < LAYERS - 1; ++layer) {
            if (tid == 0) {
                if (layer == 0) issue_layer(tmem, a0, smem_u32(smem + Lay::w0), kMlpIn, WIDTH, mbar);
                else issue_layer(tmem, a1, smem_u32(smem + Lay::wm), WIDTH, WIDTH, mbar);
            }
            ok = __syncthreads_and(mbar_wait(mbar, phase)) != 0;  // one decision for the whole block
            phase ^= 1u;
            fence_after();
            if (!ok) break;
#pragma unroll
            for (int c = 0; c < WIDTH / 16; ++c) {
                float v[16];
                tmem_ld16(my_lane + c * 16, v);
                __align__(16) __half h[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) h[e] = __float2half(fmaxf(v[e], 0.f));
                *reinterpret_cast<uint4*>(smem + Lay::a1 + canon(tid, c * 16, WIDTH)) = *reinterpret_cast<uint4*>(h);
                *reinterpret_cast<uint4*>(smem + Lay::a1 + canon(tid, c * 16 + 8, WIDTH)) =
                    *reinterpret_cast<uint4*>(h + 8);
            }
            fence_async_smem();
            fence_before();
            __syncthreads();
            fence_after();
        }
        if (!ok) break;
        // output layer (N = 16, columns WIDTH..WIDTH+15 of TMEM)
        if (tid == 0) issue_layer(tmem + WIDTH, a1, smem_u32(smem + Lay::wl), WIDTH, kLastN, mbar);
        ok = __syncthreads_and(mbar_wait(mbar, phase)) != 0;
        phase ^= 1u;
        fence_after();
        if (!ok) break;
        float out[16];
        tmem_ld16(my_lane + WIDTH, out);
        if (active) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float z = x[k] + out[k];
                p.rgb[3 * ray + k] = A * sigmoidf_(z) + (1.0f - A) * p.bg[k];
            }
            if (p.depth) p.depth[ray] = depth;
            if (p.opacity) p.opacity[ray] = A;
        }
        fence_before();
        __syncthreads();
        fence_after();
    }
    // An expired wait leaves the MMA it waited for possibly in flight, still writing
    // TMEM and reading the operand tiles: wait for that same phase once more (a
    // second bounded wait) before the tensor memory and shared memory are released.
    // If the MMA never completes the block keeps its TMEM (the dealloc would race
    // the MMA) and flags the context as suspect (2): the caller should stop using
    // the tensor-core forms.
    bool drained = true;
    if (!ok) drained = __syncthreads_and(mbar_wait(mbar, phase ^ 1u, 1 << 22)) != 0;
    if (!ok && tid == 0) atomicMax(&g_tc_error, drained ? 1 : 2);
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0 && drained)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

template <int WIDTH, int LAYERS>
void launch_tc(const MlpTcParams& p, cudaStream_t st) {
    using Lay = TcLayout<WIDTH, LAYERS>;
    const size_t shm = Lay::bytes;
    if (shm > 48 * 1024)
        cudaFuncSetAttribute(mlp_tc_kernel<WIDTH, LAYERS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    const int64_t tiles = (p.n + kTile - 1) / kTile;
    const int64_t grid = tiles < 152 * 2 ? tiles : 152 * 2;
    mlp_tc_kernel<WIDTH, LAYERS><<<(unsigned)grid, 128, shm, st>>>(p);
}

// A bounded wait that nothing completes: the MLP kernel's mbarrier wait with a
// caller-chosen poll limit on a barrier no thread arrives at.  When it gives up it
// sets the tensor-core error flag, which ngprt_sync_status then reports; the
// timeout path is exercised without the tensor cores and nothing is left running.
__global__ void wait_probe_kernel(int limit) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t mbar = smem_u32(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait(mbar, 0, limit);
    if (!ok && threadIdx.x == 0) atomicExch(&g_tc_error, 1);
}

}  // namespace

bool mlp_tc_supports(int width, int layers) {
    return (layers == 2 || layers == 3) && (width == 16 || width == 32 || width == 64);
}

void launch_mlp_tc(int width, int layers, const float* state, const void* w, const float bg[3], int64_t n, float* rgb,
                   float* depth, float* opacity, cudaStream_t st) {
    MlpTcParams p;
    p.state = state;
    p.w = static_cast<const __half*>(w);
    p.bg[0] = bg[0];
    p.bg[1] = bg[1];
    p.bg[2] = bg[2];
    p.n = n;
    p.rgb = rgb;
    p.depth = depth;
    p.opacity = opacity;
    if (layers == 2) {
        if (width == 16) launch_tc<16, 2>(p, st);
        else if (width == 32) launch_tc<32, 2>(p, st);
        else launch_tc<64, 2>(p, st);
    } else {
        if (width == 16) launch_tc<16, 3>(p, st);
        else if (width == 32) launch_tc<32, 3>(p, st);
        else launch_tc<64, 3>(p, st);
    }
}

}  // namespace ngprt

extern "C" int32_t ngprt_tensor_core_error(void) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, ngprt::g_tc_error, sizeof v) != cudaSuccess) return -1;
    return v;
}

extern "C" int32_t ngprt_sync_status(void* stream) {
    const cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        ngprt::set_error("ngprt_sync_status: %s", cudaGetErrorString(e));
        return NGPRT_ERR_CUDA;
    }
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, ngprt::g_tc_error, sizeof v) != cudaSuccess) return ngprt::cuda_status("ngprt_sync_status");
    if (v) {
        const int zero = 0;
        cudaMemcpyToSymbol(ngprt::g_tc_error, &zero, sizeof zero);  // reported once
        if (v >= 2)
            ngprt::set_error("ngprt_sync_status: a tensor-core MLP gave up waiting for its MMAs and they did not "
                             "complete: its tensor memory was not released, so stop using the tensor-core forms in "
                             "this context");
        else
            ngprt::set_error("ngprt_sync_status: a tensor-core MLP gave up waiting for its MMAs; its rays were not "
                             "shaded");
        return NGPRT_ERR_TIMEOUT;
    }
    return NGPRT_OK;
}

extern "C" int32_t ngprt_test_bounded_wait(int32_t limit, void* stream) {
    NGPRT_REQUIRE(limit >= 1 && limit <= (1 << 20), "ngprt_test_bounded_wait: limit=%d not in [1, 2^20]", limit);
    ngprt::wait_probe_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(limit);
    return ngprt::cuda_status("ngprt_test_bounded_wait");
}
