// Batched LSTM actuator network (Sec. 3.3): one recurrent cell per joint maps the joint's current
// measurements (position error q* - q, velocity qd) to a torque, stepped once per simulation
// substep (four per 50 Hz policy step).  Standard cell with a forget gate, gate order input,
// forget, cell, output; hidden width 32, so a warp runs four joints at a time with lane j owning
// hidden unit j: the recurrent product reads the joints' h rows from shared memory by broadcast and
// the weights as 16-byte vectors (both four units per load), and the torque is a warp sum over the
// units.
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
    constexpr int JPW = 4;                       // joints per warp at a time
    // W_hh as [m / 4][gate row][m % 4]: lane j reads its row's four consecutive m with one 16-byte
    // load (consecutive lanes, consecutive 16 bytes); each warp's joints' h rows sit in shared
    // memory and are read four units at a time by broadcast
    __shared__ __align__(16) float whh[AH / 4][AG][4];
    __shared__ float wih[AI][AG];
    __shared__ float bias[AG];
    __shared__ float wout[AH];
    __shared__ float bout;
    __shared__ __align__(16) float hs[8][JPW][AH];
    constexpr int O_HH = AG * AI, O_B = O_HH + AG * AH, O_OUT = O_B + AG;
    for (int i = threadIdx.x; i < AG * AH; i += blockDim.x) {
        const int mg = i / (AG * 4), r = (i / 4) % AG, k = i % 4;   // destination order
        whh[mg][r][k] = __ldg(w + O_HH + r * AH + 4 * mg + k);
    }
    for (int i = threadIdx.x; i < AG * AI; i += blockDim.x) wih[i / AG][i % AG] = __ldg(w + (i % AG) * AI + i / AG);
    for (int i = threadIdx.x; i < AG; i += blockDim.x) bias[i] = w[O_B + i];
    if (threadIdx.x < AH) wout[threadIdx.x] = w[O_OUT + threadIdx.x];
    if (threadIdx.x == 0) bout = w[O_OUT + AH];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    for (int j0 = (blockIdx.x * wpb + wid) * JPW; j0 < n; j0 += gridDim.x * wpb * JPW) {
        float cj[JPW], a[JPW][4];
        __syncwarp();                            // the previous group's h rows are read
#pragma unroll
        for (int q = 0; q < JPW; ++q) {
            const int j = min(j0 + q, n - 1);          // a tail warp repeats the last joint, writes nothing
            hs[wid][q][lane] = h[(size_t)j * AH + lane];
            cj[q] = c[(size_t)j * AH + lane];
            const float x0 = x[(size_t)j * AI], x1 = x[(size_t)j * AI + 1];
#pragma unroll
            for (int g = 0; g < 4; ++g)
                a[q][g] = fmaf(wih[1][g * AH + lane], x1, fmaf(wih[0][g * AH + lane], x0, bias[g * AH + lane]));
        }
        __syncwarp();
#pragma unroll 2
        for (int mg = 0; mg < AH / 4; ++mg) {
            float4 wv[4];
#pragma unroll
            for (int g = 0; g < 4; ++g) wv[g] = *reinterpret_cast<const float4*>(&whh[mg][g * AH + lane][0]);
#pragma unroll
            for (int q = 0; q < JPW; ++q) {
                const float4 hv = *reinterpret_cast<const float4*>(&hs[wid][q][4 * mg]);
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    a[q][g] = fmaf(wv[g].x, hv.x, a[q][g]);
                    a[q][g] = fmaf(wv[g].y, hv.y, a[q][g]);
                    a[q][g] = fmaf(wv[g].z, hv.z, a[q][g]);
                    a[q][g] = fmaf(wv[g].w, hv.w, a[q][g]);
                }
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
    // one wave of three blocks per SM (80 registers a thread), each block's warps striding over joints
    const int grid = std::min((n + 31) / 32, 148 * 3);
    cudaError_t e = launch_pdl(actuator_lstm_kernel, dim3(grid), dim3(256), 0, s, n, w, x, h, c, tau);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace rl
