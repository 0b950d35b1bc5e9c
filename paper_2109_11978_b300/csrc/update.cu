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

__global__ void permutation_kernel(int B, int half, uint64_t seed, const unsigned long long* iteration, int* idx) {
    const int e = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    const uint64_t key = rng_key(seed, kStreamPerm, *iteration, (uint64_t)e, 0ull);
    uint64_t y = feistel((uint64_t)i, key, half);
    // A cycle of the permutation of [0, 2^(2h)) that starts in [0, B) returns to [0, B) in at
    // most 2^(2h) - B + 1 steps; the bound only guards against a corrupted key.
    const uint64_t limit = (1ull << (2 * half)) - (uint64_t)B + 2ull;
    for (uint64_t k = 0; y >= (uint64_t)B && k < limit; ++k) y = feistel(y, key, half);
    idx[(size_t)e * B + i] = (int)(y < (uint64_t)B ? y : (uint64_t)i);
}

// ---------------------------------------------------------------- gather
// One warp per minibatch row: the sampled row of the rollout observations is copied with
// 16-byte vector loads and stores (Op * element size is a multiple of 128 bytes).
template <bool BF16>
__global__ void __launch_bounds__(256) gather_kernel(const void* __restrict__ obs, const int* __restrict__ idx, int M,
                                                     int Op, void* X) {
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= M) return;
    constexpr int E = BF16 ? 2 : 4;
    const int nvec = Op * E / 16;
    const uint4* src = reinterpret_cast<const uint4*>(reinterpret_cast<const uint8_t*>(obs) + (size_t)__ldg(idx + row) * Op * E);
    uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(X) + (size_t)row * Op * E);
    for (int v = lane; v < nvec; v += 32) dst[v] = __ldg(src + v);
}

// ---------------------------------------------------------------- Adam
// Kingma & Ba (2015) with bias correction: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
// p -= alpha m_hat / (sqrt(v_hat) + eps).  alpha and the step count come from the device
// scalars (Algorithm 1 has already updated alpha for this minibatch).  The gradient of each
// parameter is the sum of its partials (split-K slices or per-block head partials), read
// coalesced; bf16 copies of the GEMM weights (and their transposes) are refreshed in the
// same pass.
__global__ void __launch_bounds__(256) adam_kernel(AdamParams p) {
    int s = 0;
    while (s + 1 < p.nsegs && (int)blockIdx.x >= p.seg[s + 1].block_start) ++s;
    const AdamSeg sg = p.seg[s];
    // step size alpha / (1 - 0.9^t) and 1 / sqrt(1 - 0.999^t), computed once per minibatch by the
    // loss kernel together with Algorithm 1 and the step count
    const float step_size = p.scal ? p.scal[SC_STEPSIZE] : 0.f;
    const float inv_sqrt_bc2 = p.scal ? p.scal[SC_INVSQRT_BC2] : 1.f;
    // Segments with many partials: 32 parameters per block, the 8 warps split the partials
    // (warp w sums partials w, w + 8, ...) and the warp sums are added in warp order.
    const bool wide = sg.nsplit > ADAM_WIDE;
    __shared__ float red[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long base = (long long)(blockIdx.x - sg.block_start) * (wide ? 32 : ADAM_CHUNK);
    for (int k = wide ? lane : (int)threadIdx.x; k < (wide ? 32 : ADAM_CHUNK); k += wide ? 32 : blockDim.x) {
        const long long i = base + k;
        const bool in = i < sg.size;
        const float* src = sg.partials + (in ? i : 0);
        float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f, g4 = 0.f, g5 = 0.f, g6 = 0.f, g7 = 0.f;
        const int q0 = wide ? warp : 0, dq = wide ? 8 : 1;
        int q = q0;
        if (in) {
            // eight independent loads in flight, fixed order
            const size_t st = (size_t)dq * sg.stride;
            for (; q + 7 * dq < sg.nsplit; q += 8 * dq) {
                const float* a = src + (size_t)q * sg.stride;
                g0 += __ldg(a); g1 += __ldg(a + st); g2 += __ldg(a + 2 * st); g3 += __ldg(a + 3 * st);
                g4 += __ldg(a + 4 * st); g5 += __ldg(a + 5 * st); g6 += __ldg(a + 6 * st); g7 += __ldg(a + 7 * st);
            }
            for (; q < sg.nsplit; q += dq) g0 += __ldg(src + (size_t)q * sg.stride);
        }
        g0 += g4; g1 += g5; g2 += g6; g3 += g7;
        float g = (g0 + g1) + (g2 + g3);
        if (wide) {
            red[warp][lane] = g;
            __syncthreads();
            g = 0.f;
#pragma unroll
            for (int w = 0; w < 8; ++w) g += red[w][lane];
            if (warp != 0) break;           // warp 0 applies the step for the 32 parameters
        }
        if (!in) continue;
        const long long gi = sg.offset + i;
        if (p.grad_out) {
            p.grad_out[gi] = g;
            continue;
        }
        const float m = 0.9f * p.m[gi] + 0.1f * g;
        const float v = 0.999f * p.v[gi] + 0.001f * g * g;
        p.m[gi] = m;
        p.v[gi] = v;
        const float w = p.p[gi] - step_size * m / (sqrtf(v) * inv_sqrt_bc2 + 1e-8f);
        p.p[gi] = w;
        if (p.wbf[s]) {
            const int cols = p.cols[s];
            const int r = (int)(i / cols), c = (int)(i % cols);
            const __nv_bfloat16 b = f2bf(w);
            reinterpret_cast<__nv_bfloat16*>(p.wbf[s])[i] = b;
            if (p.wbf_t[s]) reinterpret_cast<__nv_bfloat16*>(p.wbf_t[s])[(size_t)c * p.rows[s] + r] = b;
        }
    }
}

__global__ void small_kernel(int op, float* scal, unsigned long long* iteration, const float* src, float* dst,
                             float nsamp) {
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

__global__ void to_bf16_kernel(const float* __restrict__ src, int rows, int cols, __nv_bfloat16* dst, __nv_bfloat16* dst_t) {
    const long long n = (long long)rows * cols;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const __nv_bfloat16 b = f2bf(src[i]);
        if (dst) dst[i] = b;
        if (dst_t) dst_t[(size_t)(i % cols) * rows + i / cols] = b;
    }
}

}  // namespace

cudaError_t launch_permutation(int B, int epochs, uint64_t seed, const unsigned long long* iteration, int* idx,
                               cudaStream_t s) {
    int bits = 2;
    while ((1ll << bits) < B) bits += 2;
    dim3 grid((B + 255) / 256, epochs);
    permutation_kernel<<<grid, 256, 0, s>>>(B, bits / 2, seed, iteration, idx);
    return cudaGetLastError();
}

cudaError_t launch_gather(const void* obs, int bf16, const int* idx, int M, int Op, void* X, cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    if (Op % 64) return cudaErrorInvalidValue;
    const int grid = (M + 7) / 8;
    if (bf16) gather_kernel<true><<<grid, 256, 0, s>>>(obs, idx, M, Op, X);
    else gather_kernel<false><<<grid, 256, 0, s>>>(obs, idx, M, Op, X);
    return cudaGetLastError();
}

cudaError_t launch_adam(const AdamParams& p, cudaStream_t s) {
    if (p.nblocks <= 0) return cudaSuccess;
    adam_kernel<<<p.nblocks, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_small(int op, float* scal, unsigned long long* iteration, const float* stats_src, float* stats_dst,
                         float nsamp, cudaStream_t s) {
    small_kernel<<<1, 32, 0, s>>>(op, scal, iteration, stats_src, stats_dst, nsamp);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* src, int rows, int cols, void* dst, void* dst_t, cudaStream_t s) {
    const long long n = (long long)rows * cols;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    to_bf16_kernel<<<blocks, 256, 0, s>>>(src, rows, cols, reinterpret_cast<__nv_bfloat16*>(dst),
                                          reinterpret_cast<__nv_bfloat16*>(dst_t));
    return cudaGetLastError();
}

}  // namespace rl
