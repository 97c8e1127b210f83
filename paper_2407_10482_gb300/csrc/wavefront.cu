// wavefront.cu -- the render's march as alternating rounds over the unfinished rays.
//
// The fused march kernel keeps a ray per thread from start to end; lanes spend much
// of their time idle (some march empty space while others gather, rays end at
// different depths) and the per-ray state limits how many warps fit on an SM.
// Here every round has two kernels:
//   advance : one unfinished ray per thread walks empty space to its next K
//             occupied points and records them (position, delta, marching count);
//   gather  : K consecutive lanes per ray each gather and attend one of those points
//             (Eq. 6-8), then composite them (Eq. 2, 5) in order, every lane of
//             the group running the same sequence so that T, the accumulators and
//             the termination test (T < t_term) are exactly those of the fused
//             kernel; rays still going are appended to the next round's list.
// After the last round the fused kernel finishes the remaining rays from their
// stored state.  Results (values and counts) equal the fused kernel's bit for bit.
#include "march.cuh"

#ifndef NGPRT_WF_K
#define NGPRT_WF_K 4
#endif
#ifndef NGPRT_WF_ROUNDS
#define NGPRT_WF_ROUNDS 8
#endif

namespace ngprt {

constexpr int kWfK = NGPRT_WF_K;
constexpr int kWfRounds = NGPRT_WF_ROUNDS;
static_assert(32 % kWfK == 0, "K must divide the warp");

namespace {

struct WfParams {
    MarchParams m;
    float4* pos;      // [n] t, t_out, t_start, T
    int4* cnt;        // [n] lat_k, n_march, n_samp, -
    int* list[2];     // alive lists (ping-pong)
    int* counts;      // [kWfRounds + 1] list lengths per round
    float4* smp_u;    // [n * K] u0, u1, u2, t
    float2* smp_d;    // [n * K] delta, n_march (int bits)
    int* meta;        // [n] samples recorded | exhausted << 16
    int round;
};

// Warp-aggregated append of `ray` to list/count when `want` (lanes may be inactive).
__device__ __forceinline__ void append(bool want, int ray, int* list, int* count) {
    const unsigned active = __activemask();
    const unsigned mask = __ballot_sync(active, want);
    if (!mask) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(mask));
    base = __shfl_sync(active, base, leader);
    if (want) list[base + __popc(mask & ((1u << lane) - 1u))] = ray;
}

__global__ void __launch_bounds__(128) wf_init_kernel(const __grid_constant__ WfParams p) {
    int64_t ray;
    float o[3], d[3], t, t_out;
    bool hit;
    if (!ray_setup(p.m, ray, o, d, t, t_out, hit)) return;
    float4* s = reinterpret_cast<float4*>(p.m.state + ray * NGPRT_STATE_FLOATS);
    s[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    s[1] = make_float4(0.f, 0.f, 0.f, 0.f);
    s[2] = make_float4(0.f, d[0], d[1], d[2]);
    if (hit) {
        p.pos[ray] = make_float4(t, t_out, t, 1.0f);
        p.cnt[ray] = make_int4(0, 0, 0, 0);
    } else if (p.m.stats) {
        reinterpret_cast<int2*>(p.m.stats)[ray] = make_int2(0, 0);
    }
    append(hit, (int)ray, p.list[0], p.counts);
}

__global__ void __launch_bounds__(128) wf_advance_kernel(const __grid_constant__ WfParams p) {
    const int n = p.counts[p.round];
    const int* list = p.list[p.round & 1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ray = list[i];
        float o[3], d[3];
        ray_of(p.m, ray, o, d);
        normalize_dir(d);
        const float4 ps = p.pos[ray];
        const int4 cs = p.cnt[ray];
        MarchState st;
        st.t = ps.x;
        st.t_out = ps.y;
        st.t_start = ps.z;
        st.lat_k = cs.x;
        st.n_march = cs.y;
        st.n_samp = cs.z;
        int k = 0;
        bool exhausted = false;
        for (; k < kWfK; ++k) {
            float u[3], delta, dt;
            if (!march_advance(p.m, o, d, st, u, delta, dt)) {
                exhausted = true;
                break;
            }
            const size_t slot = (size_t)i * kWfK + k;
            p.smp_u[slot] = make_float4(u[0], u[1], u[2], st.t);
            p.smp_d[slot] = make_float2(delta, __int_as_float(st.n_march));
            march_after_sample(p.m, st, dt);
        }
        p.pos[ray] = make_float4(st.t, st.t_out, st.t_start, ps.w);
        p.cnt[ray] = make_int4(st.lat_k, st.n_march, st.n_samp, 0);
        p.meta[i] = k | (exhausted ? 1 << 16 : 0);
    }
}

template <int L, int DT>
__global__ void __launch_bounds__(128, 4) wf_gather_kernel(const __grid_constant__ WfParams p) {
    extern __shared__ float gate_smem[];
    const int n = p.counts[p.round];
    const int* list = p.list[p.round & 1];
    const int lane = threadIdx.x & 31;
    const int gbase = lane & ~(kWfK - 1);
    const int stride = gridDim.x * blockDim.x;
    // whole warps iterate together so that the group shuffles see all K lanes
    for (int j0 = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; j0 < n * kWfK; j0 += stride) {
        const int j = j0 + lane;
        const int i = j / kWfK, k = j % kWfK;
        const bool in = i < n;
        int ray = 0, meta = 0;
        if (in) {
            ray = list[i];
            meta = p.meta[i];
        }
        const int n_valid = meta & 0xffff;
        const bool valid = in && k < n_valid;
        float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float4 su = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 sd = make_float2(0.f, 0.f);
        if (valid) {
            su = p.smp_u[j];
            sd = p.smp_d[j];
            const float u[3] = {su.x, su.y, su.z};
            sample_features<L, DT>(p.m.g, u, p.m.opts.attn_mode, f, gate_smem + threadIdx.x, blockDim.x);
        }
        // composite the group's samples in order (every lane of the group alike)
        ForwardSampler<L, DT> fw(p.m.g, p.m.opts.attn_mode, p.m.opts.t_term, nullptr);
        float* s = p.m.state + (size_t)ray * NGPRT_STATE_FLOATS;
        float4 ps = make_float4(0.f, 0.f, 0.f, 1.f);
        int4 cs = make_int4(0, 0, 0, 0);
        if (in) {
            ps = p.pos[ray];
            cs = p.cnt[ray];
            fw.resume(s, ps.w);
        }
        bool done = false;
        int n_samp = cs.z - n_valid, n_march = cs.y;
#pragma unroll
        for (int kk = 0; kk < kWfK; ++kk) {
            const int src = gbase + kk;
            float fk[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) fk[c] = __shfl_sync(0xffffffffu, f[c], src);
            const float tk = __shfl_sync(0xffffffffu, su.w, src);
            const float dk = __shfl_sync(0xffffffffu, sd.x, src);
            const int mk = __float_as_int(__shfl_sync(0xffffffffu, sd.y, src));
            if (in && !done && kk < n_valid) {
                done = fw.composite(fk, tk, dk);
                ++n_samp;
                if (done) n_march = mk;
            }
        }
        if (!in) continue;
        const bool exhausted = (meta >> 16) & 1;
        const bool finished = done || exhausted;
        if (k == 0) {
            float4* s4 = reinterpret_cast<float4*>(s);
            s4[0] = make_float4(fw.Cd[0], fw.Cd[1], fw.Cd[2], fw.F[0]);
            s4[1] = make_float4(fw.F[1], fw.F[2], fw.F[3], fw.A);
            s[8] = fw.depth;
            if (finished) {
                if (p.m.stats) reinterpret_cast<int2*>(p.m.stats)[ray] = make_int2(n_march, n_samp);
            } else {
                p.pos[ray] = make_float4(ps.x, ps.y, ps.z, fw.T);
            }
        }
        if (p.round + 1 <= kWfRounds)
            append(k == 0 && !finished, ray, p.list[(p.round + 1) & 1], p.counts + p.round + 1);
    }
}

template <int L, int DT>
__global__ void __launch_bounds__(128, march_min_blocks<L, DT>()) wf_finish_kernel(const __grid_constant__ WfParams p) {
    extern __shared__ float gate_smem[];
    const int n = p.counts[kWfRounds];
    const int* list = p.list[kWfRounds & 1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ray = list[i];
        float o[3], d[3];
        ray_of(p.m, ray, o, d);
        normalize_dir(d);
        const float4 ps = p.pos[ray];
        const int4 cs = p.cnt[ray];
        MarchState st;
        st.t = ps.x;
        st.t_out = ps.y;
        st.t_start = ps.z;
        st.lat_k = cs.x;
        st.n_march = cs.y;
        st.n_samp = cs.z;
        float* s = p.m.state + (size_t)ray * NGPRT_STATE_FLOATS;
        ForwardSampler<L, DT> fw(p.m.g, p.m.opts.attn_mode, p.m.opts.t_term, gate_smem + threadIdx.x);
        fw.resume(s, ps.w);
        march_loop_from(p.m, o, d, st, fw);
        float4* s4 = reinterpret_cast<float4*>(s);
        s4[0] = make_float4(fw.Cd[0], fw.Cd[1], fw.Cd[2], fw.F[0]);
        s4[1] = make_float4(fw.F[1], fw.F[2], fw.F[3], fw.A);
        s[8] = fw.depth;
        if (p.m.stats) reinterpret_cast<int2*>(p.m.stats)[ray] = make_int2(st.n_march, st.n_samp);
    }
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

// Scratch of the wavefront engine for n rays (after the per-ray state).
size_t wavefront_bytes(int64_t n) {
    const size_t N = (size_t)n;
    return align256(N * sizeof(float4)) + align256(N * sizeof(int4)) + 2 * align256(N * sizeof(int)) +
           align256((kWfRounds + 1) * sizeof(int)) + align256(N * kWfK * sizeof(float4)) +
           align256(N * kWfK * sizeof(float2)) + align256(N * sizeof(int));
}

template <int L, int DT>
int32_t run_wavefront_t(const MarchParams& m, dim3 ray_grid, char* ws, cudaStream_t st) {
    WfParams p;
    memset(&p, 0, sizeof p);
    p.m = m;
    const size_t N = (size_t)m.n_rays;
    char* q = ws;
    p.pos = reinterpret_cast<float4*>(q); q += align256(N * sizeof(float4));
    p.cnt = reinterpret_cast<int4*>(q); q += align256(N * sizeof(int4));
    p.list[0] = reinterpret_cast<int*>(q); q += align256(N * sizeof(int));
    p.list[1] = reinterpret_cast<int*>(q); q += align256(N * sizeof(int));
    p.counts = reinterpret_cast<int*>(q); q += align256((kWfRounds + 1) * sizeof(int));
    p.smp_u = reinterpret_cast<float4*>(q); q += align256(N * kWfK * sizeof(float4));
    p.smp_d = reinterpret_cast<float2*>(q); q += align256(N * kWfK * sizeof(float2));
    p.meta = reinterpret_cast<int*>(q);
    if (cudaMemsetAsync(p.counts, 0, (kWfRounds + 1) * sizeof(int), st) != cudaSuccess) return cuda_status("wavefront");
    wf_init_kernel<<<ray_grid, 128, 0, st>>>(p);
    const size_t shm = (size_t)2 * L * 128 * sizeof(float);
    const unsigned blocks = 152 * 8;
    for (int r = 0; r < kWfRounds; ++r) {
        p.round = r;
        wf_advance_kernel<<<blocks, 128, 0, st>>>(p);
        wf_gather_kernel<L, DT><<<blocks, 128, shm, st>>>(p);
    }
    p.round = kWfRounds;
    wf_finish_kernel<L, DT><<<blocks, 128, shm, st>>>(p);
    return NGPRT_OK;
}

template <int L>
int32_t run_wavefront_l(int dt, const MarchParams& m, dim3 grid, char* ws, cudaStream_t st) {
    if (dt == NGPRT_F32) return run_wavefront_t<L, NGPRT_F32>(m, grid, ws, st);
    if (dt == NGPRT_F16) return run_wavefront_t<L, NGPRT_F16>(m, grid, ws, st);
    return run_wavefront_t<L, NGPRT_BF16>(m, grid, ws, st);
}

int32_t run_wavefront(int L, int dt, const MarchParams& m, dim3 grid, void* ws, cudaStream_t st) {
    char* w = static_cast<char*>(ws);
    switch (L) {
        case 1: return run_wavefront_l<1>(dt, m, grid, w, st);
        case 2: return run_wavefront_l<2>(dt, m, grid, w, st);
        case 3: return run_wavefront_l<3>(dt, m, grid, w, st);
        case 4: return run_wavefront_l<4>(dt, m, grid, w, st);
        case 8: return run_wavefront_l<8>(dt, m, grid, w, st);
        case 16: return run_wavefront_l<16>(dt, m, grid, w, st);
        default: set_error("wavefront: no kernel for L=%d", L); return NGPRT_ERR_UNSUPPORTED;
    }
}

}  // namespace ngprt
