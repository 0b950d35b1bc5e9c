// Generalized advantage estimation (Sec. 2.2.1, Table 3) as a reverse-time scan per robot,
// plus the batch normalisation of the advantages.
//
// Layout: rewards, values, dones, advantages and returns are [T][N] (robot index
// contiguous), so at every step t a warp touches 32 consecutive robots: 128-byte coalesced
// loads and stores.  One thread owns one robot and keeps its running A_{t+1}, V_{t+1} in
// registers; the T steps are processed newest first in chunks of 8 whose loads are issued
// together.  Each block also leaves the fp64 sum and sum of squares of its advantages in a
// scratch slot; the normalising kernel reduces those few hundred partials (every block
// redundantly, which avoids a third launch) and rescales the advantages in place.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace rl {

// Scratch of rl_gae_noalloc: the per-block fp64 (sum, sum of squares) pairs of the advantage
// statistics, in a file-scope device array instead of caller- or library-allocated memory.
// 4096 blocks of 64 robots = at most 262,144 robots; 64 KiB held by every device that loads
// the library, until the process exits.
constexpr int NOALLOC_MAX_PARTS = 4096;
static __device__ __align__(256) double g_gae_noalloc_scratch[2 * NOALLOC_MAX_PARTS];

namespace {

constexpr int GAE_THREADS = 64;
constexpr int CHUNK = 8;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(GAE_THREADS) gae_scan_kernel(int T, int N, float gamma, float lam,
                                                               const float* __restrict__ rew,
                                                               const float* __restrict__ val,
                                                               const float* __restrict__ last_val,
                                                               const uint8_t* __restrict__ done,
                                                               float* __restrict__ adv, float* __restrict__ ret,
                                                               double* __restrict__ partials) {
    pdl_wait();
    pdl_trigger();
    const int n = blockIdx.x * GAE_THREADS + threadIdx.x;
    double s1 = 0.0, s2 = 0.0;
    if (n < N) {
        float next_v = last_val[n];
        float next_a = 0.f;
        const float gl = gamma * lam;
        for (int t1 = T; t1 > 0; t1 -= CHUNK) {
            const int t0 = t1 - CHUNK > 0 ? t1 - CHUNK : 0;
            float r[CHUNK], v[CHUNK], d[CHUNK];
#pragma unroll
            for (int i = 0; i < CHUNK; ++i) {
                const int t = t1 - 1 - i;
                if (t >= t0) {
                    const size_t o = (size_t)t * N + n;
                    r[i] = __ldg(rew + o);
                    v[i] = __ldg(val + o);
                    d[i] = (float)__ldg(done + o);
                }
            }
#pragma unroll
            for (int i = 0; i < CHUNK; ++i) {
                const int t = t1 - 1 - i;
                if (t >= t0) {
                    const float nonterm = 1.0f - d[i];
                    const float delta = r[i] + gamma * nonterm * next_v - v[i];
                    next_a = delta + gl * nonterm * next_a;
                    const size_t o = (size_t)t * N + n;
                    adv[o] = next_a;
                    ret[o] = next_a + v[i];
                    next_v = v[i];
                    s1 += (double)next_a;
                    s2 += (double)next_a * (double)next_a;
                }
            }
        }
    }
    if (partials) {
        __shared__ double red[2][GAE_THREADS / 32];
        s1 = warp_sum(s1);
        s2 = warp_sum(s2);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) { red[0][warp] = s1; red[1][warp] = s2; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < GAE_THREADS / 32; ++w) { a += red[0][w]; b += red[1][w]; }
            partials[2 * blockIdx.x] = a;
            partials[2 * blockIdx.x + 1] = b;
        }
    }
}

__global__ void gae_normalize_kernel(size_t total, int nparts, const double* __restrict__ partials,
                                     float* __restrict__ adv, int normalize, float* __restrict__ stats) {
    pdl_wait();
    pdl_trigger();
    __shared__ double red[2][32];
    __shared__ float ms[2];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        a += partials[2 * i];
        b += partials[2 * i + 1];
    }
    a = warp_sum(a);
    b = warp_sum(b);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { red[0][warp] = a; red[1][warp] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) { sa += red[0][w]; sb += red[1][w]; }
        const double mean = sa / (double)total;
        double var = sb / (double)total - mean * mean;
        var = var > 0.0 ? var : 0.0;
        ms[0] = (float)mean;
        ms[1] = (float)sqrt(var);
        if (blockIdx.x == 0 && stats) { stats[0] = ms[0]; stats[1] = ms[1]; }
    }
    __syncthreads();
    if (!normalize) return;
    const float mean = ms[0];
    const float inv = 1.0f / (ms[1] + 1e-8f);
    const size_t n4 = total / 4;
    float4* a4 = reinterpret_cast<float4*>(adv);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        float4 x = a4[i];
        x.x = (x.x - mean) * inv; x.y = (x.y - mean) * inv; x.z = (x.z - mean) * inv; x.w = (x.w - mean) * inv;
        a4[i] = x;
    }
    for (size_t i = n4 * 4 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
        adv[i] = (adv[i] - mean) * inv;
}

}  // namespace

int gae_num_partials(int T, int N) { return (N + GAE_THREADS - 1) / GAE_THREADS; }

int gae_noalloc_max_envs() { return NOALLOC_MAX_PARTS * GAE_THREADS; }

// Device address of the scratch array on the current device.  In host code the array's name is
// only a host-side stand-in, so the address is looked up with the device current.  Outside stream
// capture it is looked up on every call (so it stays right after a cudaDeviceReset, which loads
// the module afresh) and remembered per device; during capture the remembered address is used,
// since the lookup may load the module, which a capturing stream does not allow.
cudaError_t gae_noalloc_scratch(cudaStream_t s, void** out) {
    static std::mutex mu;
    static void* addr[128] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_gae_noalloc_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = p;
    } else if (!addr[dev]) {
        return cudaErrorStreamCaptureUnsupported;   // first call on this device inside a capture
    }
    *out = addr[dev];
    return cudaSuccess;
}

cudaError_t launch_gae(int T, int N, float gamma, float lam, const float* rew, const float* val,
                       const float* last_val, const uint8_t* done, float* adv, float* ret, int normalize,
                       float* adv_stats, float* partials, int nparts, cudaStream_t s) {
    if (T <= 0 || N <= 0) return cudaSuccess;
    const bool need = normalize || adv_stats;
    double* part = need ? reinterpret_cast<double*>(partials) : nullptr;
    cudaError_t e0 = launch_pdl(gae_scan_kernel, dim3(gae_num_partials(T, N)), dim3(GAE_THREADS), 0, s, T, N, gamma, lam,
                                rew, val, last_val, done, adv, ret, part);
    if (e0 != cudaSuccess) return e0;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !need) return e;
    const size_t total = (size_t)T * N;
    int blocks = (int)((total / 4 + 255) / 256);
    if (blocks < 1) blocks = 1;
    if (blocks > 1184) blocks = 1184;   // 8 x 148 SMs
    e = launch_pdl(gae_normalize_kernel, dim3(blocks), dim3(256), 0, s, total, nparts, (const double*)part, adv, normalize,
                   adv_stats);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace rl
