// Learner-side memory-bound kernels of the PPO update: the per-epoch minibatch shuffle, the
// minibatch gather, Adam with the split-K / per-block gradient partials reduced on the fly,
// and the small scalar bookkeeping kernels that keep the iteration graph free of host syncs.
#include "common.cuh"
#include "kernels.cuh"

namespace rl {

namespace {

// ---------------------------------------------------------------- shuffle (Sec. 2.2.1)
// Permutation of [0, B) from a 4-round balanced Feistel network over 2h bits (2^(2h) >= B),
// round function = SplitMix64 finaliser of (key + (round + 1) 2^32 + R) masked to h bits, and
// cycle-walking back into [0, B).  A bijection by construction, so every sample appears in
// exactly one minibatch per epoch.
__device__ __forceinline__ uint64_t feistel(uint64_t x, uint64_t key, int half) {
    const uint64_t mask = (1ull << half) - 1ull;
    uint64_t L = x >> half, R = x & mask;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const uint64_t F = mix64(key + ((uint64_t)(r + 1) << 32) + R) & mask;
        const uint64_t nl = R;
        R = L ^ F;
        L = nl;
    }
    return (L << half) | R;
}

__global__ void permutation_kernel(int B, int half, uint64_t seed, const unsigned long long* iteration, int* idx,
                                   int* status) {
    pdl_wait();
    pdl_trigger();
    const int e = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    const uint64_t key = rng_key(seed, kStreamPerm, *iteration, (uint64_t)e, 0ull);
    uint64_t y = feistel((uint64_t)i, key, half);
    // A cycle of the permutation of [0, 2^(2h)) that starts in [0, B) returns to [0, B) in at
    // most 2^(2h) - B + 1 steps, so the walk always ends inside the bound; running out of it
    // would mean a broken network, which is recorded as RL_ERR_STATE (the slot then holds i, an
    // in-range index, so no later kernel reads outside the batch).
    const uint64_t limit = (1ull << (2 * half)) - (uint64_t)B + 2ull;
    for (uint64_t k = 0; y >= (uint64_t)B && k < limit; ++k) y = feistel(y, key, half);
    if (y >= (uint64_t)B) {
        set_status(status, RL_ERR_STATE);
        y = (uint64_t)i;
    }
    idx[(size_t)e * B + i] = (int)y;
}

// ---------------------------------------------------------------- gather
// One warp per four minibatch rows: the four sampled row indices are read first, then one
// 16-byte vector per lane of each of the four rollout observation rows is loaded before any is
// stored (few registers, so gather blocks fit beside a GEMM CTA on an SM and many warps keep
// loads in flight); Op * element size is a multiple of 128 bytes.
constexpr int GATHER_ROWS = 4;      // rows per warp
constexpr int GATHER_VPL = 1;       // 16-byte vectors per lane and row held in registers at once

template <bool BF16>
__global__ void __launch_bounds__(256, 6) gather_kernel(const void* __restrict__ obs, const int* __restrict__ idx, int M,
                                                     int Op, void* __restrict__ X) {
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int row0 = (blockIdx.x * 8 + (threadIdx.x >> 5)) * GATHER_ROWS;
    if (row0 >= M) return;
    constexpr int E = BF16 ? 2 : 4;
    const int nvec = Op * E / 16;                         // vectors per row (a multiple of 8)
    const uint8_t* src[GATHER_ROWS];
#pragma unroll
    for (int r = 0; r < GATHER_ROWS; ++r)
        src[r] = reinterpret_cast<const uint8_t*>(obs) + (size_t)(row0 + r < M ? __ldg(idx + row0 + r) : 0) * Op * E;
    for (int v0 = 0; v0 < nvec; v0 += 32 * GATHER_VPL) {
        uint4 val[GATHER_ROWS][GATHER_VPL];
#pragma unroll
        for (int r = 0; r < GATHER_ROWS; ++r)
#pragma unroll
            for (int k = 0; k < GATHER_VPL; ++k) {
                const int v = v0 + lane + 32 * k;
                if (row0 + r < M && v < nvec) val[r][k] = __ldg(reinterpret_cast<const uint4*>(src[r]) + v);
            }
#pragma unroll
        for (int r = 0; r < GATHER_ROWS; ++r)
#pragma unroll
            for (int k = 0; k < GATHER_VPL; ++k) {
                const int v = v0 + lane + 32 * k;
                if (row0 + r < M && v < nvec)
                    reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(X) + (size_t)(row0 + r) * Op * E)[v] = val[r][k];
            }
    }
}

// ---------------------------------------------------------------- Adam
// Kingma & Ba (2015) with bias correction: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
// p -= alpha m_hat / (sqrt(v_hat) + eps).  alpha and the step count come from the device
// scalars (Algorithm 1 has already updated alpha for this minibatch).  The gradient of each
// parameter is the sum of its partials (split-K slices or per-block head partials), read
// coalesced, four parameters per thread (float4) wherever the segment allows it, with eight
// loads in flight, and the parameter's own state (p, m, v) fetched after the partial sums (so
// that both are not live at once: four blocks fit per SM); bf16 copies of the GEMM weights are
// refreshed in the same pass.
template <int V>
struct Vec;
template <>
struct Vec<4> {
    using T = float4;
    __device__ static T zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ static T ld(const float* a) { return __ldg(reinterpret_cast<const float4*>(a)); }
    __device__ static T ld_rw(const float* a) { return *reinterpret_cast<const float4*>(a); }
    __device__ static void st(float* a, T v) { *reinterpret_cast<float4*>(a) = v; }
    __device__ static void add(T& a, T b) { a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w; }
    __device__ static float get(const T& v, int c) { return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w; }
    __device__ static void set(T& v, int c, float x) {
        if (c == 0) v.x = x; else if (c == 1) v.y = x; else if (c == 2) v.z = x; else v.w = x;
    }
};
template <>
struct Vec<1> {
    using T = float;
    __device__ static T zero() { return 0.f; }
    __device__ static T ld(const float* a) { return __ldg(a); }
    __device__ static T ld_rw(const float* a) { return *a; }
    __device__ static void st(float* a, T v) { *a = v; }
    __device__ static void add(T& a, T b) { a += b; }
    __device__ static float get(const T& v, int) { return v; }
    __device__ static void set(T& v, int, float x) { v = x; }
};

template <int V>
__device__ __forceinline__ void adam_segment(const AdamParams& p, const AdamSeg& sg, int s, float step_size,
                                             float inv_sqrt_bc2) {
    using O = Vec<V>;
    using T = typename O::T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // narrow segments (few partials): one thread per V parameters, each summing every partial;
    // wide segments (many partials): one warp per V parameters, lane l summing partials l, l + 32,
    // ..., then a fixed xor tree across the lanes (every lane ends with the same bits)
    const bool wide = sg.nsplit > ADAM_WIDE;
    const long long base = (long long)(blockIdx.x - sg.block_start) * adam_per_block(sg.nsplit, V == 4);
    const long long i = base + (long long)(wide ? warp : (int)threadIdx.x) * V;
    const bool in = i < sg.size;
    const bool owner = in && (!wide || lane == 0);          // the thread that applies the step
    const long long gi = sg.offset + i;
    // partial sums: eight independent accumulators, combined in a fixed order
    T g0 = O::zero(), g1 = g0, g2 = g0, g3 = g0, g4 = g0, g5 = g0, g6 = g0, g7 = g0;
    if (in) {
        const int dq = wide ? 32 : 1;
        int q = wide ? lane : 0;
        const float* src = sg.partials + i;
        const size_t st = (size_t)dq * sg.stride;
        for (; q + 7 * dq < sg.nsplit; q += 8 * dq) {
            const float* a = src + (size_t)q * sg.stride;
            O::add(g0, O::ld(a)); O::add(g1, O::ld(a + st)); O::add(g2, O::ld(a + 2 * st)); O::add(g3, O::ld(a + 3 * st));
            O::add(g4, O::ld(a + 4 * st)); O::add(g5, O::ld(a + 5 * st)); O::add(g6, O::ld(a + 6 * st));
            O::add(g7, O::ld(a + 7 * st));
        }
        for (; q < sg.nsplit; q += dq) O::add(g0, O::ld(src + (size_t)q * sg.stride));
    }
    O::add(g0, g4); O::add(g1, g5); O::add(g2, g6); O::add(g3, g7);
    O::add(g0, g1); O::add(g2, g3); O::add(g0, g2);
    T g = g0;
    if (wide) {
#pragma unroll
        for (int c = 0; c < V; ++c) {
            float x = O::get(g, c);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            O::set(g, c, x);
        }
    }
    if (!owner) return;
    if (p.grad_out) {
        O::st(p.grad_out + gi, g);
        return;
    }
    // the moments and weights are read after the partial sums, so that the sums' eight
    // accumulators and the moments are not live together
    T m = O::ld_rw(p.m + gi), v = O::ld_rw(p.v + gi), w = O::ld_rw(p.p + gi);
#pragma unroll
    for (int c = 0; c < V; ++c) {
        const float gc = O::get(g, c);
        const float mc = 0.9f * O::get(m, c) + 0.1f * gc;
        const float vc = 0.999f * O::get(v, c) + 0.001f * gc * gc;
        O::set(m, c, mc);
        O::set(v, c, vc);
        O::set(w, c, O::get(w, c) - step_size * mc / (sqrtf(vc) * inv_sqrt_bc2 + 1e-8f));
    }
    O::st(p.m + gi, m);
    O::st(p.v + gi, v);
    O::st(p.p + gi, w);
    if (p.wbf[s]) {
        __nv_bfloat16* d = reinterpret_cast<__nv_bfloat16*>(p.wbf[s]) + i;
        if (V == 4) {
            __nv_bfloat162 lo = __floats2bfloat162_rn(O::get(w, 0), O::get(w, 1));
            __nv_bfloat162 hi = __floats2bfloat162_rn(O::get(w, 2), O::get(w, 3));
            uint2 pk;
            pk.x = *reinterpret_cast<uint32_t*>(&lo);
            pk.y = *reinterpret_cast<uint32_t*>(&hi);
            *reinterpret_cast<uint2*>(d) = pk;
        } else {
            d[0] = f2bf(O::get(w, 0));
        }
    }
}

__global__ void __launch_bounds__(ADAM_THREADS, 4) adam_kernel(AdamParams p) {
    pdl_wait();
    pdl_trigger();
    int s = 0;
    while (s + 1 < p.nsegs && (int)blockIdx.x >= p.seg[s + 1].block_start) ++s;
    const AdamSeg sg = p.seg[s];
    // step size alpha / (1 - 0.9^t) and 1 / sqrt(1 - 0.999^t), computed once per minibatch by the
    // loss kernel together with Algorithm 1 and the step count
    const float step_size = p.scal ? p.scal[SC_STEPSIZE] : p.step_size_host;
    const float inv_sqrt_bc2 = p.scal ? p.scal[SC_INVSQRT_BC2] : p.inv_sqrt_bc2_host;
    if (sg.vec) adam_segment<4>(p, sg, s, step_size, inv_sqrt_bc2);
    else adam_segment<1>(p, sg, s, step_size, inv_sqrt_bc2);
}

__global__ void small_kernel(int op, float* scal, unsigned long long* iteration, const float* src, float* dst,
                             float nsamp) {
    pdl_wait();
    pdl_trigger();
    const int i = threadIdx.x;
    if (op == SMALL_ITER_INC) {
        if (i == 0) *iteration += 1ull;
    } else if (op == SMALL_ZERO_STATS) {
        if (i < RL_NSTATS) dst[i] = 0.f;
    } else if (op == SMALL_FINAL_STATS) {
        // dst = per-iteration summary from the accumulators (src = accumulators)
        if (i == 0) {
            const float nmb = src[12] > 0.f ? src[12] : 1.f;
            dst[0] = src[0] / nmb; dst[1] = src[1] / nmb; dst[2] = src[2] / nmb; dst[3] = src[3];
            dst[4] = src[4] / nmb; dst[5] = scal[SC_ALPHA]; dst[6] = src[6] / nmb;
            const float ns = nsamp > 0.f ? nsamp : 1.f;
            dst[7] = src[ACC_ENV] / ns; dst[8] = scal[SC_ADV_MEAN]; dst[9] = scal[SC_ADV_STD];
            dst[10] = src[ACC_ENV + 1]; dst[11] = src[ACC_ENV + 2] / ns;
            dst[12] = nmb; dst[13] = 0.f; dst[14] = 0.f; dst[15] = 0.f;
        }
    }
}

__global__ void to_bf16_kernel(const float* __restrict__ src, long long n, __nv_bfloat16* dst) {
    pdl_wait();
    pdl_trigger();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = f2bf(src[i]);
}

}  // namespace

cudaError_t launch_permutation(int B, int epochs, uint64_t seed, const unsigned long long* iteration, int* idx,
                               int* status, cudaStream_t s) {
    int bits = 2;
    while ((1ll << bits) < B) bits += 2;
    dim3 grid((B + 255) / 256, epochs);
    cudaError_t e = launch_pdl(permutation_kernel, grid, dim3(256), 0, s, B, bits / 2, seed, iteration, idx, status);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_gather(const void* obs, int bf16, const int* idx, int M, int Op, void* X, cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    if (Op % 64) return cudaErrorInvalidValue;
    const int grid = (M + 8 * GATHER_ROWS - 1) / (8 * GATHER_ROWS);
    cudaError_t e = bf16 ? launch_pdl(gather_kernel<true>, dim3(grid), dim3(256), 0, s, obs, idx, M, Op, X)
                         : launch_pdl(gather_kernel<false>, dim3(grid), dim3(256), 0, s, obs, idx, M, Op, X);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// One warp per sample: lane j writes field j of the sample's 128-byte record (lanes past the
// 2A + 4 fields write zeros), so every record leaves as one full line.
__global__ void __launch_bounds__(256) pack_records_kernel(int B, int A, const float* __restrict__ a_old,
                                                           const float* __restrict__ mu_old, const float* __restrict__ logp_old,
                                                           const float* __restrict__ adv, const float* __restrict__ v_old,
                                                           const float* __restrict__ ret, float* __restrict__ rec) {
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const long long s = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (s >= B) return;
    float f = 0.f;
    if (lane < A) f = a_old[s * A + lane];
    else if (lane < 2 * A) f = mu_old[s * A + lane - A];
    else if (lane == 2 * A) f = logp_old[s];
    else if (lane == 2 * A + 1) f = adv[s];
    else if (lane == 2 * A + 2) f = v_old[s];
    else if (lane == 2 * A + 3) f = ret[s];
    rec[s * REC_LD + lane] = f;
}

cudaError_t launch_pack_records(int B, int A, const float* a_old, const float* mu_old, const float* logp_old,
                                const float* adv, const float* v_old, const float* ret, float* rec, cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    if (A < 1 || 2 * A + 4 > REC_LD || !rec) return cudaErrorInvalidValue;
    cudaError_t e = launch_pdl(pack_records_kernel, dim3((B + 7) / 8), dim3(256), 0, s, B, A, a_old, mu_old, logp_old, adv,
                               v_old, ret, rec);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_adam(const AdamParams& p, cudaStream_t s) {
    if (p.nblocks <= 0) return cudaSuccess;
    cudaError_t e = launch_pdl(adam_kernel, dim3(p.nblocks), dim3(ADAM_THREADS), 0, s, p);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_small(int op, float* scal, unsigned long long* iteration, const float* stats_src, float* stats_dst,
                         float nsamp, cudaStream_t s) {
    cudaError_t e = launch_pdl(small_kernel, dim3(1), dim3(32), 0, s, op, scal, iteration, stats_src, stats_dst, nsamp);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* src, int rows, int cols, void* dst, cudaStream_t s) {
    const long long n = (long long)rows * cols;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    cudaError_t e = launch_pdl(to_bf16_kernel, dim3(blocks), dim3(256), 0, s, src, n, reinterpret_cast<__nv_bfloat16*>(dst));
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace rl
