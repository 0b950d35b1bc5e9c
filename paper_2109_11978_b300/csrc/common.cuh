// Device helpers shared by the kernels of the library: the counter-based generator, exact
// fp32 arithmetic for the physics stand-in, bf16 conversion, the device status word.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "../../include/rl_b300.h"

namespace rl {

// ---------------------------------------------------------------------------------------
// Counter-based random numbers.  SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014;
// constants of Vigna's public reference implementation).  A key chains the finaliser over
// (seed, stream, a, b, env) adding (counter + 1) * GAMMA; the slot-th word of a key is
// SplitMix64's slot-th output mix64(key + (slot + 1) * GAMMA).
// ---------------------------------------------------------------------------------------
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr int kStreamEnv = 1, kStreamAct = 2, kStreamPerm = 3, kStreamInit = 4, kStreamTerrain = 5;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t rng_key(uint64_t seed, uint64_t stream, uint64_t a,
                                                     uint64_t b, uint64_t env) {
    uint64_t h = mix64(seed + (stream + 1) * kGamma);
    h = mix64(h + (a + 1) * kGamma);
    h = mix64(h + (b + 1) * kGamma);
    return mix64(h + (env + 1) * kGamma);
}

__host__ __device__ __forceinline__ uint64_t rng_word(uint64_t key, uint32_t slot) {
    return mix64(key + (uint64_t)(slot + 1) * kGamma);
}

__device__ __forceinline__ uint32_t hi32(uint64_t w) { return (uint32_t)(w >> 32); }
__device__ __forceinline__ uint32_t lo32(uint64_t w) { return (uint32_t)w; }

// (u >> 8) * 2^-24, exact in fp32.
__device__ __forceinline__ float uniform01(uint32_t u) {
    return __fmul_rn(__uint2float_rn(u >> 8), 5.9604644775390625e-08f);
}
// 2 * uniform01 - 1, exact in fp32.
__device__ __forceinline__ float uniform_pm1(uint32_t u) {
    return __fsub_rn(__fmul_rn(2.0f, uniform01(u)), 1.0f);
}
// floor(u * n / 2^32), uniform on {0..n-1}.
__device__ __forceinline__ uint32_t mulhi_n(uint32_t u, uint32_t n) {
    return (uint32_t)(((uint64_t)u * n) >> 32);
}
// Irwin-Hall(4) normal: the four 16-bit fields summed, centred, times 1/sqrt((2^32-1)/3).
// The centred sum is an integer below 2^24 in magnitude, so only the product rounds.
__device__ __forceinline__ float irwin_hall(uint64_t w) {
    int s = (int)(w & 0xFFFF) + (int)((w >> 16) & 0xFFFF) + (int)((w >> 32) & 0xFFFF) +
            (int)((w >> 48) & 0xFFFF);
    return __fmul_rn(__int2float_rn(s - 131070), 0x1.bb67aep-16f);
}
// Box-Muller (cos branch): u1 in (0, 1] from the high word, u2 in [0, 1) from the low word.
__device__ __forceinline__ float box_muller(uint64_t w) {
    float u1 = __fmul_rn(__uint2float_rn((hi32(w) >> 8) + 1u), 5.9604644775390625e-08f);
    float u2 = uniform01(lo32(w));
    return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

// ---------------------------------------------------------------------------------------
// Programmatic dependent launch.  The kernels of an iteration are launched with programmatic
// stream serialization: a kernel's blocks may be scheduled while its predecessor drains, run
// their set-up, and wait in pdl_wait() until the predecessor grid has completed and its memory
// is visible; pdl_trigger() lets the successor be scheduled early.  Every kernel calls
// pdl_trigger() only after pdl_wait(), so when a kernel starts, every kernel before its
// predecessor has completed: it may read what those wrote before its own pdl_wait() (weights,
// state, records), but reads its predecessor's results and writes global memory only after it.
// Without the launch attribute both are no-ops.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------------------------------
// Device status word (first failure wins).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void set_status(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

__device__ __forceinline__ float elu(float x) { return x > 0.f ? x : expm1f(x); }
// d ELU / dx from y = ELU(x): 1 for x > 0, y + 1 otherwise.
__device__ __forceinline__ float elu_grad_y(float y) { return y > 0.f ? 1.f : y + 1.f; }

__device__ __forceinline__ float bf2f(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ __nv_bfloat16 f2bf(float x) { return __float2bfloat16_rn(x); }

}  // namespace rl
