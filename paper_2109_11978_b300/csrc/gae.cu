// Generalized advantage estimation (Sec. 2.2.1, Table 3) as a reverse-time scan per robot,
// plus the batch normalisation of the advantages.
//
// Layout: rewards, values, dones, advantages and returns are [T][N] (robot index
// contiguous), so at every step t a warp touches consecutive robots: coalesced loads and
// stores.  A thread owns four consecutive robots (16-byte accesses, 512 bytes per warp request;
// one robot when N is not a multiple of 4 or an array is not 16-byte aligned) and keeps their
// running A_{t+1}, V_{t+1} in registers; the T steps are processed newest first in chunks whose
// loads are issued together.  Each 256-thread block also leaves the sum and the sum of squares
// of its advantages in a 16-byte scratch slot as compensated fp32 pairs (value, rounding error:
// Neumaier's two-sum at every addition, a fixed xor tree across the lanes, the warps in order),
// so that no fp64 arithmetic runs per element (fp64 is slow on this part).  One block then
// reduces the slots in a fixed order and writes (mean, std) to the scratch's first slot (the last
// additions and the variance in fp64, a handful of operations); the normalising kernel reads
// those two numbers and rescales the advantages in place with 16-byte vectors.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace rl {

// Scratch of rl_gae_noalloc: the (mean, std) slot and the per-block (sum, error, sum of squares,
// error) slots of the advantage statistics, in a file-scope device array instead of caller- or
// library-allocated memory.  4096 slots of 16 bytes = the statistics slot and 4095 blocks of 256
// robots (the one-robot-per-thread form; the four-robot form needs fewer), so at most 1,048,320
// robots; 64 KiB held by every device that loads the library, until the process exits.
constexpr int NOALLOC_MAX_SLOTS = 4096;
static __device__ __align__(256) float4 g_gae_noalloc_scratch[NOALLOC_MAX_SLOTS];

namespace {

constexpr int GAE_THREADS = 256;
constexpr int GAE_V4_MIN_N = 262144;   // robots from which the scan takes four per thread
constexpr int CHUNK = 8;

__device__ __forceinline__ void two_sum(float& sum, float& err, float x) {
    const float t = sum + x;
    err += fabsf(sum) >= fabsf(x) ? (sum - t) + x : (x - t) + sum;
    sum = t;
}

// (value, error) pairs of two quantities combined across the lanes by a fixed xor tree (the
// lower lane's value first, so both partners form the same sum)
__device__ __forceinline__ void warp_pairs(float (&v)[4], int lane) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const float os = __shfl_xor_sync(0xffffffffu, v[2 * q], o), oe = __shfl_xor_sync(0xffffffffu, v[2 * q + 1], o);
            const bool lo = (lane & o) == 0;
            float a = lo ? v[2 * q] : os, e = lo ? v[2 * q + 1] : oe;
            two_sum(a, e, lo ? os : v[2 * q]);
            v[2 * q] = a;
            v[2 * q + 1] = e + (lo ? oe : v[2 * q + 1]);
        }
}

// R robots per thread (R = 4: 16-byte loads and stores of four consecutive robots, used when N is
// a multiple of 4 and the arrays are 16-byte aligned, so that each warp request moves 512 bytes;
// R = 1 otherwise); the T steps newest first in chunks whose loads are issued together.
template <int R>
struct GaeIO;
template <>
struct GaeIO<1> {
    static constexpr int CH = 8;
    __device__ static void ldf(const float* p, size_t o, float (&x)[1]) { x[0] = __ldg(p + o); }
    __device__ static void ldd(const uint8_t* p, size_t o, float (&x)[1]) { x[0] = (float)__ldg(p + o); }
    __device__ static void stf(float* p, size_t o, const float (&x)[1]) { p[o] = x[0]; }
};
template <>
struct GaeIO<4> {
    static constexpr int CH = 4;
    __device__ static void ldf(const float* p, size_t o, float (&x)[4]) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p + o));
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    }
    __device__ static void ldd(const uint8_t* p, size_t o, float (&x)[4]) {
        const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(p + o));
        x[0] = (float)(w & 0xFFu); x[1] = (float)((w >> 8) & 0xFFu); x[2] = (float)((w >> 16) & 0xFFu); x[3] = (float)(w >> 24);
    }
    __device__ static void stf(float* p, size_t o, const float (&x)[4]) {
        *reinterpret_cast<float4*>(p + o) = make_float4(x[0], x[1], x[2], x[3]);
    }
};

template <int R>
__global__ void __launch_bounds__(GAE_THREADS, R == 4 ? 3 : 4) gae_scan_kernel(int T, int N, float gamma, float lam,
                                                                const float* __restrict__ rew,
                                                                const float* __restrict__ val,
                                                                const float* __restrict__ last_val,
                                                                const uint8_t* __restrict__ done,
                                                                float* __restrict__ adv, float* __restrict__ ret,
                                                                float4* __restrict__ partials) {
    using IO = GaeIO<R>;
    constexpr int CH = IO::CH;
    pdl_wait();
    pdl_trigger();
    const int n = (blockIdx.x * GAE_THREADS + threadIdx.x) * R;
    float st[4] = {0.f, 0.f, 0.f, 0.f};     // sum, its error, sum of squares, its error
    if (n < N) {
        float next_v[R], next_a[R];
        IO::ldf(last_val, (size_t)n, next_v);
#pragma unroll
        for (int k = 0; k < R; ++k) next_a[k] = 0.f;
        const float gl = gamma * lam;
        for (int t1 = T; t1 > 0; t1 -= CH) {
            const int t0 = t1 - CH > 0 ? t1 - CH : 0;
            float r[CH][R], v[CH][R], d[CH][R];
#pragma unroll
            for (int i = 0; i < CH; ++i) {
                const int t = t1 - 1 - i;
                if (t >= t0) {
                    const size_t o = (size_t)t * N + n;
                    IO::ldf(rew, o, r[i]);
                    IO::ldf(val, o, v[i]);
                    IO::ldd(done, o, d[i]);
                }
            }
#pragma unroll
            for (int i = 0; i < CH; ++i) {
                const int t = t1 - 1 - i;
                if (t >= t0) {
                    float a[R], rt[R];
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        const float nonterm = 1.0f - d[i][k];
                        const float delta = r[i][k] + gamma * nonterm * next_v[k] - v[i][k];
                        next_a[k] = delta + gl * nonterm * next_a[k];
                        a[k] = next_a[k];
                        rt[k] = next_a[k] + v[i][k];
                        next_v[k] = v[i][k];
                        two_sum(st[0], st[1], next_a[k]);
                        // the square's own rounding error (exact by fma) joins the error term, so
                        // the sums carry A and A^2 to about twice fp32's precision
                        const float sq = next_a[k] * next_a[k];
                        two_sum(st[2], st[3], sq);
                        st[3] += fmaf(next_a[k], next_a[k], -sq);
                    }
                    const size_t o = (size_t)t * N + n;
                    IO::stf(adv, o, a);
                    IO::stf(ret, o, rt);
                }
            }
        }
    }
    if (partials) {
        __shared__ float ws[GAE_THREADS / 32][4];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        warp_pairs(st, lane);
        if (lane == 0)
#pragma unroll
            for (int i = 0; i < 4; ++i) ws[warp][i] = st[i];
        __syncthreads();
        if (threadIdx.x == 0) {
            float b[4] = {ws[0][0], ws[0][1], ws[0][2], ws[0][3]};
            for (int w = 1; w < GAE_THREADS / 32; ++w) {
                two_sum(b[0], b[1], ws[w][0]);
                b[1] += ws[w][1];
                two_sum(b[2], b[3], ws[w][2]);
                b[3] += ws[w][3];
            }
            partials[blockIdx.x] = make_float4(b[0], b[1], b[2], b[3]);
        }
    }
}

// One block: the blocks' slots in a fixed order (thread t takes slots t, t + 256, ...; adding a
// zero slot changes no sum), then the xor tree and the warps in order; mean and population std
// into ms_slot (and adv_stats).
__global__ void __launch_bounds__(GAE_THREADS) gae_stats_kernel(int nparts, double total, const float4* __restrict__ partials,
                                                                float4* __restrict__ ms_slot, float* __restrict__ adv_stats) {
    pdl_wait();
    pdl_trigger();
    __shared__ float ws[GAE_THREADS / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float st[4] = {0.f, 0.f, 0.f, 0.f};
    // eight slots' loads in flight per thread before any is added
    for (int i0 = threadIdx.x; i0 < nparts; i0 += 8 * GAE_THREADS) {
        float4 q[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int i = i0 + k * GAE_THREADS;
            q[k] = i < nparts ? partials[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            two_sum(st[0], st[1], q[k].x);
            st[1] += q[k].y;
            two_sum(st[2], st[3], q[k].z);
            st[3] += q[k].w;
        }
    }
    warp_pairs(st, lane);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < 4; ++i) ws[warp][i] = st[i];
    __syncthreads();
    if (threadIdx.x != 0) return;
    double s1 = 0.0, s2 = 0.0;
    for (int w = 0; w < GAE_THREADS / 32; ++w) {
        s1 += (double)ws[w][0] + (double)ws[w][1];
        s2 += (double)ws[w][2] + (double)ws[w][3];
    }
    const double mean = s1 / total;
    double var = s2 / total - mean * mean;
    var = var > 0.0 ? var : 0.0;
    const float m = (float)mean, sd = (float)sqrt(var);
    ms_slot[0] = make_float4(m, sd, 0.f, 0.f);
    if (adv_stats) {
        adv_stats[0] = m;
        adv_stats[1] = sd;
    }
}

__global__ void gae_normalize_kernel(size_t total, const float4* __restrict__ ms, float* __restrict__ adv) {
    pdl_wait();
    pdl_trigger();
    const float4 q = ms[0];
    const float mean = q.x;
    const float inv = 1.0f / (q.y + 1e-8f);
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

// one slot per block of 256 robots plus the (mean, std) slot
int gae_noalloc_max_envs() { return (NOALLOC_MAX_SLOTS - 1) * GAE_THREADS; }

size_t gae_workspace_bytes(int T, int N) {
    if (T <= 0 || N <= 0) return 0;
    return (size_t)(gae_num_partials(T, N) + 1) * sizeof(float4);
}

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
    if (need && (!partials || nparts != gae_num_partials(T, N))) return cudaErrorInvalidValue;
    // slot 0: (mean, std); slots 1 ..: one per block of the scan
    float4* ms = need ? reinterpret_cast<float4*>(partials) : nullptr;
    float4* part = need ? ms + 1 : nullptr;
    // four robots per thread (16-byte accesses) where the scan is bandwidth-bound; below that the
    // launch is a single latency-bound wave, and one robot per thread gives four times the blocks
    // and half the dependent load rounds (chunks of 8 steps instead of 4)
    const bool v4 = N >= GAE_V4_MIN_N && N % 4 == 0 && ((reinterpret_cast<uintptr_t>(rew) | reinterpret_cast<uintptr_t>(val) |
                                    reinterpret_cast<uintptr_t>(last_val) | reinterpret_cast<uintptr_t>(adv) |
                                    reinterpret_cast<uintptr_t>(ret)) & 15u) == 0 &&
                    (reinterpret_cast<uintptr_t>(done) & 3u) == 0;
    const int robots_per_block = GAE_THREADS * (v4 ? 4 : 1);
    const int blocks = (N + robots_per_block - 1) / robots_per_block;
    cudaError_t e = v4 ? launch_pdl(gae_scan_kernel<4>, dim3(blocks), dim3(GAE_THREADS), 0, s, T, N, gamma, lam, rew, val,
                                    last_val, done, adv, ret, part)
                       : launch_pdl(gae_scan_kernel<1>, dim3(blocks), dim3(GAE_THREADS), 0, s, T, N, gamma, lam, rew, val,
                                    last_val, done, adv, ret, part);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess || !need) return e;
    const size_t total = (size_t)T * N;
    e = launch_pdl(gae_stats_kernel, dim3(1), dim3(GAE_THREADS), 0, s, blocks, (double)total, (const float4*)part, ms,
                   adv_stats);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess || !normalize) return e;
    int nb = (int)((total / 4 + 255) / 256);
    if (nb < 1) nb = 1;
    if (nb > 4 * 148) nb = 4 * 148;     // four blocks of 256 per SM, grid-stride
    e = launch_pdl(gae_normalize_kernel, dim3(nb), dim3(256), 0, s, total, (const float4*)ms, adv);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace rl
