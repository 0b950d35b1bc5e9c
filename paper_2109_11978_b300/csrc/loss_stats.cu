// Minibatch statistics of the loss head and the learning-rate step (Sec. 2.2, Algorithm 1):
// one block sums the per-block statistics the loss head left in its partials (surrogate, value
// loss, KL, clip count) in a fixed order in compensated fp32, takes the minibatch means, applies
// Algorithm 1 to the device learning rate and prepares Adam's step size and bias corrections for
// the step that follows.  It runs after the loss head, beside the first input-gradient GEMM
// (nothing but Adam reads what it writes), so it stays off the update's critical path.
#include "common.cuh"
#include "kernels.cuh"

namespace rl {

namespace {

constexpr int ST_THREADS = 256;
constexpr float HALF_LOG_2PI_F = 0.91893853320467274f;

// Neumaier's two-sum: the rounding error of every addition is carried in a second float
__device__ __forceinline__ void two_sum(float& sum, float& err, float x) {
    const float t = sum + x;
    err += fabsf(sum) >= fabsf(x) ? (sum - t) + x : (x - t) + sum;
    sum = t;
}

// (sum, err) pairs of four values combined across the lanes of a warp by a fixed xor tree (the
// lower lane's value first, so both partners form the same sum)
__device__ __forceinline__ void warp_two_sum(float (&st)[4], float (&ce)[4], int lane) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float os = __shfl_xor_sync(0xffffffffu, st[i], o), oc = __shfl_xor_sync(0xffffffffu, ce[i], o);
            const bool lo = (lane & o) == 0;
            float a = lo ? st[i] : os, ca = lo ? ce[i] : oc;
            two_sum(a, ca, lo ? os : st[i]);
            st[i] = a;
            ce[i] = ca + (lo ? oc : ce[i]);
        }
}

__global__ void __launch_bounds__(ST_THREADS) loss_stats_kernel(HeadParams p) {
    pdl_wait();
    pdl_trigger();
    const int A = p.A;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const HeadPart hp = head_part(A, p.H);
    const int PF = hp.PF, O_ST = hp.ST;
    __shared__ float ws[ST_THREADS / 32][8];
    // thread t sums blocks t, t + 256, ... in that order (their loads issued together)
    float st[4] = {0.f, 0.f, 0.f, 0.f}, ce[4] = {0.f, 0.f, 0.f, 0.f};
    for (int b0 = tid; b0 < p.nblocks; b0 += ST_THREADS * 4) {
        float v[4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int b = b0 + ST_THREADS * k;
            const float* q = p.part + (size_t)(b < p.nblocks ? b : 0) * PF + O_ST;
#pragma unroll
            for (int i = 0; i < 4; ++i) v[k][i] = __ldg(q + i);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (b0 + ST_THREADS * k < p.nblocks)
#pragma unroll
                for (int i = 0; i < 4; ++i) two_sum(st[i], ce[i], v[k][i]);
    }
    warp_two_sum(st, ce, lane);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            ws[warp][i] = st[i];
            ws[warp][4 + i] = ce[i];
        }
    __syncthreads();
    if (warp != 0) return;
    // the warps' pairs in warp order, then the same tree over the first eight lanes
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        st[i] = lane < ST_THREADS / 32 ? ws[lane][i] : 0.f;
        ce[i] = lane < ST_THREADS / 32 ? ws[lane][4 + i] : 0.f;
    }
    warp_two_sum(st, ce, lane);
#pragma unroll
    for (int i = 0; i < 4; ++i) st[i] += ce[i];
    if (lane != 0) return;
    float* sc = p.scal;
    float alpha = sc[SC_ALPHA];
    const float step = sc[SC_STEP];
    float acc[6] = {};
    if (p.stats) {
        acc[0] = p.stats[0]; acc[1] = p.stats[1]; acc[2] = p.stats[2]; acc[3] = p.stats[4];
        acc[4] = p.stats[6]; acc[5] = p.stats[12];
    }
    const float inv_M = 1.0f / (float)p.M;
    float ent = 0.f;
    for (int j = 0; j < A; ++j) ent += p.log_std[j] + HALF_LOG_2PI_F + 0.5f;
    const float kl = (float)st[2] * inv_M;
    const float surr = -(float)st[0] * inv_M, vloss = (float)st[1] * inv_M;
    const float loss = surr + p.value_coef * vloss - p.entropy_coef * ent;
    sc[SC_KL] = kl;
    sc[SC_LOSS] = loss;
    sc[SC_SURR] = surr;
    sc[SC_VLOSS] = vloss;
    sc[SC_ENT] = ent;
    sc[SC_CLIPFRAC] = (float)st[3] * inv_M;
    if (p.kl_target > 0.f) {
        if (kl > 2.f * p.kl_target) alpha = fmaxf(p.lr_min, alpha / 1.5f);
        else if (kl < 0.5f * p.kl_target) alpha = fminf(p.lr_max, alpha * 1.5f);
        sc[SC_ALPHA] = alpha;
    }
    if (p.trace) {
        p.trace[0] = kl;
        p.trace[1] = alpha;
    }
    const float t = step + 1.f;
    sc[SC_STEP] = t;
    const float bc1 = -expm1f(t * log1pf(-0.1f));
    const float bc2 = -expm1f(t * log1pf(-0.001f));
    sc[SC_STEPSIZE] = alpha / bc1;
    sc[SC_INVSQRT_BC2] = 1.0f / sqrtf(bc2);
    if (p.stats) {
        p.stats[0] = acc[0] + loss; p.stats[1] = acc[1] + surr; p.stats[2] = acc[2] + vloss; p.stats[3] = ent;
        p.stats[4] = acc[3] + kl; p.stats[5] = alpha; p.stats[6] = acc[4] + (float)st[3] * inv_M;
        p.stats[12] = acc[5] + 1.f;
    }
}

}  // namespace

cudaError_t launch_loss_stats(const HeadParams& p, cudaStream_t s) {
    if (p.nblocks < 1 || !p.part || !p.scal) return cudaErrorInvalidValue;
    cudaError_t e = launch_pdl(loss_stats_kernel, dim3(1), dim3(ST_THREADS), 0, s, p);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace rl
