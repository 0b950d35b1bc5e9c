// Output heads of the actor and critic and the per-sample PPO loss with its hand-written
// backward through the heads (Sec. 2.2, Table 3, Algorithm 1).
//
// One warp per sample row: the lanes split the last hidden layer (coalesced row loads), the
// 12 actor outputs and the value are finished with xor-shuffle reductions, so every lane holds
// the whole per-sample state (mu, V, ratio, gradients) and the backward into the hidden layer
// is written back coalesced.  Reductions over the minibatch (head weight / bias gradients,
// log-std gradient, bias gradient of the last hidden layer, loss terms, KL) accumulate per
// warp in registers, then per block in shared memory, then as one partial per block; the
// last block to finish (a counter, no spin-wait) reduces the statistics, takes the KL mean and
// applies Algorithm 1 to the device-side learning rate before Adam runs.
#include "common.cuh"
#include "kernels.cuh"

namespace rl {

namespace {

constexpr int HEAD_WARPS = 8;
constexpr int MAX_A = 12;         // action dims (12 joint targets)
constexpr float HALF_LOG_2PI = 0.91893853320467274f;

template <bool BF16>
__device__ __forceinline__ float ld_act(const void* base, size_t i) {
    if (BF16) return bf2f(reinterpret_cast<const __nv_bfloat16*>(base)[i]);
    return reinterpret_cast<const float*>(base)[i];
}

template <bool BF16, int NK>
__global__ void __launch_bounds__(HEAD_WARPS * 32) act_head_kernel(HeadParams p) {
    extern __shared__ float sm[];
    float* Wa = sm;                 // [A][H]
    float* Wc = sm + p.A * p.H;     // [H]
    const bool actor = p.mu != nullptr || p.actions != nullptr || p.logp != nullptr;
    for (int i = threadIdx.x; i < p.A * p.H; i += blockDim.x) Wa[i] = actor ? p.Wa[i] : 0.f;
    for (int i = threadIdx.x; i < p.H; i += blockDim.x) Wc[i] = p.Wc[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nk = NK;
    const unsigned long long it = p.iteration ? *p.iteration : 0ull;
    for (int m = blockIdx.x * HEAD_WARPS + warp; m < p.M; m += gridDim.x * HEAD_WARPS) {
        float hc[NK];
        float v = 0.f;
#pragma unroll
        for (int i = 0; i < NK; ++i)
            if (i < nk) {
                hc[i] = ld_act<BF16>(p.hc, (size_t)m * p.H + lane + 32 * i);
                v += hc[i] * Wc[lane + 32 * i];
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) p.values[m] = v + p.bc[0];
        if (!actor) continue;
        float ha[NK];
#pragma unroll
        for (int i = 0; i < NK; ++i)
            if (i < nk) ha[i] = ld_act<BF16>(p.ha, (size_t)m * p.H + lane + 32 * i);
        float mine = 0.f;   // mu of action dim == lane
        for (int j = 0; j < p.A; ++j) {
            float s = 0.f;
#pragma unroll
            for (int i = 0; i < NK; ++i)
                if (i < nk) s += ha[i] * Wa[j * p.H + lane + 32 * i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == j) mine = s + p.ba[j];
        }
        float lp = 0.f;
        if (lane < p.A) {
            const float ls = p.log_std[lane];
            const uint64_t key = rng_key(p.seed, kStreamAct, it, (uint64_t)p.t, (uint64_t)m);
            const float eps = box_muller(rng_word(key, (uint32_t)lane));
            const float a = mine + expf(ls) * eps;
            lp = -0.5f * eps * eps - ls - HALF_LOG_2PI;
            if (p.mu) p.mu[(size_t)m * p.A + lane] = mine;
            if (p.actions) p.actions[(size_t)m * p.A + lane] = a;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lp += __shfl_xor_sync(0xffffffffu, lp, o);
        if (lane == 0 && p.logp) p.logp[m] = lp;
    }
}

template <bool BF16, int NK>
__global__ void __launch_bounds__(HEAD_WARPS * 32) loss_head_kernel(HeadParams p) {
    extern __shared__ float sm[];
    const int A = p.A, H = p.H;
    constexpr int nk = NK;
    float* Wa = sm;                       // [A][H]
    float* Wc = Wa + A * H;               // [H]
    const int PF = head_part_floats(A, H);
    float* accw = Wc + H;                 // per-warp partial records [HEAD_WARPS][PF]
    for (int i = threadIdx.x; i < A * H; i += blockDim.x) Wa[i] = p.Wa[i];
    for (int i = threadIdx.x; i < H; i += blockDim.x) Wc[i] = p.Wc[i];
    __syncthreads();
    // offsets inside a partial record
    const int O_WA = 0, O_BA = A * H, O_LS = O_BA + A, O_WC = O_LS + A, O_BC = O_WC + H, O_DBA = O_BC + 1,
              O_DBC = O_DBA + H, O_ST = O_DBC + H;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float inv_M = 1.0f / (float)p.M;
    float ls[MAX_A], var[MAX_A], lso[MAX_A];
#pragma unroll
    for (int j = 0; j < MAX_A; ++j)
        if (j < A) {
            ls[j] = p.log_std[j];
            var[j] = expf(2.f * ls[j]);
            lso[j] = p.log_std_old[j];
        }
    float gWa[MAX_A][NK], gWc[NK], dba[NK], dbc[NK];
#pragma unroll
    for (int i = 0; i < NK; ++i) {
        gWc[i] = dba[i] = dbc[i] = 0.f;
#pragma unroll
        for (int j = 0; j < MAX_A; ++j) gWa[j][i] = 0.f;
    }
    float gba = 0.f, gls = 0.f, gbc = 0.f;     // lane j < A owns action dim j
    float st_surr = 0.f, st_vl = 0.f, st_kl = 0.f, st_clip = 0.f;

    for (int m = blockIdx.x * HEAD_WARPS + warp; m < p.M; m += gridDim.x * HEAD_WARPS) {
        const int s = p.idx ? p.idx[m] : m;
        float ha[NK], hc[NK];
        float v = 0.f;
#pragma unroll
        for (int i = 0; i < NK; ++i)
            if (i < nk) {
                ha[i] = ld_act<BF16>(p.ha, (size_t)m * H + lane + 32 * i);
                hc[i] = ld_act<BF16>(p.hc, (size_t)m * H + lane + 32 * i);
                v += hc[i] * Wc[lane + 32 * i];
            }
        float mu[MAX_A];
#pragma unroll
        for (int j = 0; j < MAX_A; ++j)
            if (j < A) {
                float t = 0.f;
#pragma unroll
                for (int i = 0; i < NK; ++i)
                    if (i < nk) t += ha[i] * Wa[j * H + lane + 32 * i];
                mu[j] = t;
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v += __shfl_xor_sync(0xffffffffu, v, o);
#pragma unroll
            for (int j = 0; j < MAX_A; ++j)
                if (j < A) mu[j] += __shfl_xor_sync(0xffffffffu, mu[j], o);
        }
        v += p.bc[0];
        // per-sample loss terms (every lane computes the same scalars)
        float logp = 0.f, kl = 0.f;
        float diff[MAX_A];
#pragma unroll
        for (int j = 0; j < MAX_A; ++j)
            if (j < A) {
                mu[j] += p.ba[j];
                diff[j] = __ldg(p.a_old + (size_t)s * A + j) - mu[j];
                logp += -diff[j] * diff[j] / (2.f * var[j]) - ls[j] - HALF_LOG_2PI;
                const float dm = __ldg(p.mu_old + (size_t)s * A + j) - mu[j];
                kl += ls[j] - lso[j] + (expf(2.f * lso[j]) + dm * dm) / (2.f * var[j]) - 0.5f;
            }
        const float ratio = expf(logp - __ldg(p.logp_old + s));
        const float adv = __ldg(p.adv + s);
        const float s1 = ratio * adv;
        const float s2 = fminf(fmaxf(ratio, 1.f - p.clip), 1.f + p.clip) * adv;
        const float g_logp = -(s1 <= s2 ? adv : 0.f) * inv_M * ratio;
        const float vo = __ldg(p.v_old + s), R = __ldg(p.ret + s);
        const float dv = v - vo;
        const float vclip = vo + fminf(fmaxf(dv, -p.clip), p.clip);
        const float u = (v - R) * (v - R), w = (vclip - R) * (vclip - R);
        const float g_v = p.value_coef * inv_M *
                          (u >= w ? 2.f * (v - R) : ((dv > -p.clip && dv < p.clip) ? 2.f * (vclip - R) : 0.f));
        if (lane == 0) {
            st_surr += fminf(s1, s2);
            st_vl += fmaxf(u, w);
            st_kl += kl;
            st_clip += fabsf(ratio - 1.f) > p.clip ? 1.f : 0.f;
        }
        float gmu[MAX_A];
#pragma unroll
        for (int j = 0; j < MAX_A; ++j)
            if (j < A) {
                gmu[j] = g_logp * diff[j] / var[j];
                if (lane == j) {
                    gba += gmu[j];
                    gls += g_logp * (diff[j] * diff[j] / var[j] - 1.f);
                }
            }
        if (lane == 0) gbc += g_v;
        // backward into the last hidden layer and the head weight gradients
#pragma unroll
        for (int i = 0; i < NK; ++i)
            if (i < nk) {
                const int k = lane + 32 * i;
                float da = 0.f;
#pragma unroll
                for (int j = 0; j < MAX_A; ++j)
                    if (j < A) {
                        da += gmu[j] * Wa[j * H + k];
                        gWa[j][i] += gmu[j] * ha[i];
                    }
                da *= elu_grad_y(ha[i]);
                const float dc = g_v * Wc[k] * elu_grad_y(hc[i]);
                gWc[i] += g_v * hc[i];
                dba[i] += da;
                dbc[i] += dc;
                if (BF16) {
                    const __nv_bfloat16 ba16 = f2bf(da), bc16 = f2bf(dc);
                    reinterpret_cast<__nv_bfloat16*>(p.dya)[(size_t)m * H + k] = ba16;
                    reinterpret_cast<__nv_bfloat16*>(p.dyc)[(size_t)m * H + k] = bc16;
                    reinterpret_cast<__nv_bfloat16*>(p.dya_t)[(size_t)k * p.ldt + m] = ba16;
                    reinterpret_cast<__nv_bfloat16*>(p.dyc_t)[(size_t)k * p.ldt + m] = bc16;
                } else {
                    reinterpret_cast<float*>(p.dya)[(size_t)m * H + k] = da;
                    reinterpret_cast<float*>(p.dyc)[(size_t)m * H + k] = dc;
                }
            }
    }
    // warp -> shared record of this warp (every slot written exactly once)
    float* acc = accw + (size_t)warp * PF;
#pragma unroll
    for (int i = 0; i < NK; ++i) {
        const int k = lane + 32 * i;
#pragma unroll
        for (int j = 0; j < MAX_A; ++j)
            if (j < A) acc[O_WA + j * H + k] = gWa[j][i];
        acc[O_WC + k] = gWc[i];
        acc[O_DBA + k] = dba[i];
        acc[O_DBC + k] = dbc[i];
    }
    if (lane < A) {
        acc[O_BA + lane] = gba;
        acc[O_LS + lane] = gls;
    }
    if (lane == 0) {
        acc[O_BC] = gbc;
        acc[O_ST + 0] = st_surr;
        acc[O_ST + 1] = st_vl;
        acc[O_ST + 2] = st_kl;
        acc[O_ST + 3] = st_clip;
        for (int i = 4; i < 8; ++i) acc[O_ST + i] = 0.f;
    }
    __syncthreads();
    // block record = sum of the warp records in warp order (deterministic)
    float* out = p.part + (size_t)blockIdx.x * PF;
    for (int i = threadIdx.x; i < PF; i += blockDim.x) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < HEAD_WARPS; ++w) v += accw[(size_t)w * PF + i];
        if (blockIdx.x == 0 && i >= O_LS && i < O_LS + A) v -= p.entropy_coef;   // d(-c_e H)/d log sigma
        out[i] = v;
    }

    // Last block: statistics, KL mean and Algorithm 1 on the device learning rate.
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(p.counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        double su = 0.0, vl = 0.0, klsum = 0.0, cl = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) {
            const float* q = p.part + (size_t)b * PF + O_ST;
            su += __ldcg(q); vl += __ldcg(q + 1); klsum += __ldcg(q + 2); cl += __ldcg(q + 3);
        }
        float ent = 0.f;
        for (int j = 0; j < A; ++j) ent += ls[j] + HALF_LOG_2PI + 0.5f;
        const float kl = (float)(klsum / p.M);
        const float surr = (float)(-su / p.M), vloss = (float)(vl / p.M);
        const float loss = surr + p.value_coef * vloss - p.entropy_coef * ent;
        float* sc = p.scal;
        sc[SC_KL] = kl;
        sc[SC_LOSS] = loss;
        sc[SC_SURR] = surr;
        sc[SC_VLOSS] = vloss;
        sc[SC_ENT] = ent;
        sc[SC_CLIPFRAC] = (float)(cl / p.M);
        if (p.kl_target > 0.f) {
            // Algorithm 1 (App. A.4), then the Adam step count for the step that follows.
            float alpha = sc[SC_ALPHA];
            if (kl > 2.f * p.kl_target) alpha = fmaxf(p.lr_min, alpha / 1.5f);
            else if (kl < 0.5f * p.kl_target) alpha = fminf(p.lr_max, alpha * 1.5f);
            sc[SC_ALPHA] = alpha;
            sc[SC_STEP] = sc[SC_STEP] + 1.f;
        }
        if (p.stats) {
            p.stats[0] += loss; p.stats[1] += surr; p.stats[2] += vloss; p.stats[3] = ent;
            p.stats[4] += kl; p.stats[5] = sc[SC_ALPHA]; p.stats[6] += sc[SC_CLIPFRAC]; p.stats[12] += 1.f;
        }
        *p.counter = 0u;
    }
}

}  // namespace

int loss_head_blocks(int M) {
    int b = (M + HEAD_WARPS * 8 - 1) / (HEAD_WARPS * 8);
    return b < 1 ? 1 : (b > 296 ? 296 : b);
}

template <bool BF16, int NK>
static cudaError_t act_dispatch(const HeadParams& p, int blocks, size_t smem, cudaStream_t s) {
    act_head_kernel<BF16, NK><<<blocks, HEAD_WARPS * 32, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_act_head(const HeadParams& p, cudaStream_t s) {
    if (p.M <= 0) return cudaSuccess;
    if (p.A > MAX_A || !(p.H == 64 || p.H == 128 || p.H == 256)) return cudaErrorInvalidValue;
    int blocks = (p.M + HEAD_WARPS - 1) / HEAD_WARPS;
    if (blocks > 148 * 16) blocks = 148 * 16;
    const size_t smem = (size_t)(p.A * p.H + p.H) * sizeof(float);
    const int nk = p.H / 32;
    if (p.bf16) {
        if (nk == 2) return act_dispatch<true, 2>(p, blocks, smem, s);
        if (nk == 4) return act_dispatch<true, 4>(p, blocks, smem, s);
        return act_dispatch<true, 8>(p, blocks, smem, s);
    }
    if (nk == 2) return act_dispatch<false, 2>(p, blocks, smem, s);
    if (nk == 4) return act_dispatch<false, 4>(p, blocks, smem, s);
    return act_dispatch<false, 8>(p, blocks, smem, s);
}

template <bool BF16, int NK>
static cudaError_t loss_dispatch(const HeadParams& p, size_t smem, cudaStream_t s) {
    loss_head_kernel<BF16, NK><<<p.nblocks, HEAD_WARPS * 32, smem, s>>>(p);
    return cudaGetLastError();
}

// Largest dynamic shared memory of the loss head (A = 12, H = 256), set once before any
// launch (and so before any stream capture).
void heads_prepare() {
    const int smem = (12 * 256 + 256 + HEAD_WARPS * head_part_floats(12, 256)) * (int)sizeof(float);
    cudaFuncSetAttribute(loss_head_kernel<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(loss_head_kernel<true, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(loss_head_kernel<true, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(loss_head_kernel<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(loss_head_kernel<false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(loss_head_kernel<false, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_loss_head(const HeadParams& p, cudaStream_t s) {
    if (p.M <= 0) return cudaSuccess;
    if (p.A > MAX_A || !(p.H == 64 || p.H == 128 || p.H == 256)) return cudaErrorInvalidValue;
    const size_t smem = (size_t)(p.A * p.H + p.H + HEAD_WARPS * head_part_floats(p.A, p.H)) * sizeof(float);
    const int nk = p.H / 32;
    if (p.bf16) {
        if (nk == 2) return loss_dispatch<true, 2>(p, smem, s);
        if (nk == 4) return loss_dispatch<true, 4>(p, smem, s);
        return loss_dispatch<true, 8>(p, smem, s);
    }
    if (nk == 2) return loss_dispatch<false, 2>(p, smem, s);
    if (nk == 4) return loss_dispatch<false, 4>(p, smem, s);
    return loss_dispatch<false, 8>(p, smem, s);
}

}  // namespace rl
