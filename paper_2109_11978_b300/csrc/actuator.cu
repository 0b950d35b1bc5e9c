// Batched LSTM actuator network (Sec. 3.3): one recurrent cell per joint maps the joint's current
// measurements (position error q* - q, velocity qd) to a torque, stepped once per simulation
// substep (four per 50 Hz policy step).  Standard cell with a forget gate, gate order input,
// forget, cell, output; hidden width 32, so a warp runs four joints at a time with lane j owning
// hidden unit j: the recurrent product takes h from the lanes by shuffle, the weights sit transposed in
// shared memory (lane-contiguous, conflict-free), and the torque is a warp sum over the units.
// Weights: [W_ih (4H x 2) | W_hh (4H x H) | b (4H) | w_out (H) | b_out], row-major.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace rl {

namespace {

constexpr int AI = ACT_INPUTS, AH = ACT_HIDDEN, AG = 4 * ACT_HIDDEN;

__device__ __forceinline__ float sigmoid(float x) { return 1.f / (1.f + expf(-x)); }

__global__ void __launch_bounds__(256) actuator_lstm_kernel(int n, const float* __restrict__ w, const float* __restrict__ x,
                                                            float* __restrict__ h, float* __restrict__ c,
                                                            float* __restrict__ tau) {
    pdl_wait();
    pdl_trigger();
    __shared__ float whh[AH][AG];   // [m][gate row]: W_hh transposed
    __shared__ float wih[AI][AG];
    __shared__ float bias[AG];
    __shared__ float wout[AH];
    __shared__ float bout;
    constexpr int O_HH = AG * AI, O_B = O_HH + AG * AH, O_OUT = O_B + AG;
    // transposed by destination index (consecutive threads, consecutive banks)
    for (int i = threadIdx.x; i < AG * AH; i += blockDim.x) whh[i / AG][i % AG] = __ldg(w + O_HH + (i % AG) * AH + i / AG);
    for (int i = threadIdx.x; i < AG * AI; i += blockDim.x) wih[i / AG][i % AG] = __ldg(w + (i % AG) * AI + i / AG);
    for (int i = threadIdx.x; i < AG; i += blockDim.x) bias[i] = w[O_B + i];
    if (threadIdx.x < AH) wout[threadIdx.x] = w[O_OUT + threadIdx.x];
    if (threadIdx.x == 0) bout = w[O_OUT + AH];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    // JPW joints per warp at a time: each weight read from shared memory serves all of them, and
    // their independent chains overlap the shuffle and FMA latencies
    constexpr int JPW = 4;
    for (int j0 = (blockIdx.x * wpb + (threadIdx.x >> 5)) * JPW; j0 < n; j0 += gridDim.x * wpb * JPW) {
        float hj[JPW], cj[JPW], a[JPW][4];
#pragma unroll
        for (int q = 0; q < JPW; ++q) {
            const int j = min(j0 + q, n - 1);          // a tail warp repeats the last joint, writes nothing
            hj[q] = h[(size_t)j * AH + lane];
            cj[q] = c[(size_t)j * AH + lane];
            const float x0 = x[(size_t)j * AI], x1 = x[(size_t)j * AI + 1];
#pragma unroll
            for (int g = 0; g < 4; ++g)
                a[q][g] = fmaf(wih[1][g * AH + lane], x1, fmaf(wih[0][g * AH + lane], x0, bias[g * AH + lane]));
        }
#pragma unroll 8
        for (int m = 0; m < AH; ++m) {
            float wm[4];
#pragma unroll
            for (int g = 0; g < 4; ++g) wm[g] = whh[m][g * AH + lane];
#pragma unroll
            for (int q = 0; q < JPW; ++q) {
                const float hm = __shfl_sync(0xffffffffu, hj[q], m);
#pragma unroll
                for (int g = 0; g < 4; ++g) a[q][g] = fmaf(wm[g], hm, a[q][g]);
            }
        }
#pragma unroll
        for (int q = 0; q < JPW; ++q) {
            const int j = j0 + q;
            const float c2 = sigmoid(a[q][1]) * cj[q] + sigmoid(a[q][0]) * tanhf(a[q][2]);
            const float h2 = sigmoid(a[q][3]) * tanhf(c2);
            float t = wout[lane] * h2;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (j < n) {
                h[(size_t)j * AH + lane] = h2;
                c[(size_t)j * AH + lane] = c2;
                if (lane == 0) tau[j] = t + bout;
            }
        }
    }
}

}  // namespace

cudaError_t launch_actuator_lstm(int n, const float* w, const float* x, float* h, float* c, float* tau, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    // one wave of four blocks per SM (63 registers a thread), each block's warps striding over joints
    const int grid = std::min((n + 31) / 32, 148 * 4);
    cudaError_t e = launch_pdl(actuator_lstm_kernel, dim3(grid), dim3(256), 0, s, n, w, x, h, c, tau);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace rl
