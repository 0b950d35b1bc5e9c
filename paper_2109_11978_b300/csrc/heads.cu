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

// Loss head: 4 warps per block, each warp owns chunks of 16 consecutive minibatch rows, whose
// per-sample data (old actions, old means, log pi_old, advantage, V_old, return) it gathers into
// shared memory once per chunk with independent loads.  The
// gradient rows leave row-major straight from the lanes; in the bf16 form they are also staged
// in shared memory and written transposed (the K-major operand of the weight-gradient GEMM)
// as 64-byte runs, one per hidden unit.
constexpr int LH_WARPS = 4;
constexpr int LH_ROWS = 16;
constexpr int LH_SD = 28;           // per-row sample record: a_old[12], mu_old[12], logp_old, adv, v_old, ret

template <bool BF16, int NK>
__global__ void __launch_bounds__(LH_WARPS * 32) loss_head_kernel(HeadParams p) {
    extern __shared__ float sm[];
    const int A = p.A, H = p.H;
    float* Wa = sm;                       // [A][H]
    float* Wc = Wa + A * H;               // [H]
    float* cst = Wc + H;                  // [4][16]: log sigma, 1 / sigma^2, sigma_old^2, log sigma_old
    const int PF = head_part_floats(A, H);
    float* accw = cst + 64;               // per-warp partial records [LH_WARPS][PF]
    float* sdat = accw + LH_WARPS * PF;   // per-warp sample records [LH_WARPS][LH_ROWS][LH_SD]
    __nv_bfloat16* stage = reinterpret_cast<__nv_bfloat16*>(sdat + LH_WARPS * LH_ROWS * LH_SD);   // [LH_WARPS][2][LH_ROWS][H + 2]
    const int SP = H + 2;
    for (int i = threadIdx.x; i < A * H; i += blockDim.x) Wa[i] = p.Wa[i];
    for (int i = threadIdx.x; i < H; i += blockDim.x) Wc[i] = p.Wc[i];
    if (threadIdx.x < A) {
        const float ls = p.log_std[threadIdx.x], lso = p.log_std_old[threadIdx.x];
        cst[threadIdx.x] = ls;
        cst[16 + threadIdx.x] = expf(-2.f * ls);
        cst[32 + threadIdx.x] = expf(2.f * lso);
        cst[48 + threadIdx.x] = lso;
    }
    __syncthreads();
    const int O_WA = 0, O_BA = A * H, O_LS = O_BA + A, O_WC = O_LS + A, O_BC = O_WC + H, O_DBA = O_BC + 1,
              O_DBC = O_DBA + H, O_ST = O_DBC + H;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float inv_M = 1.0f / (float)p.M;
    float gWa[MAX_A][NK], gWc[NK], dba[NK], dbc[NK];
#pragma unroll
    for (int i = 0; i < NK; ++i) {
        gWc[i] = dba[i] = dbc[i] = 0.f;
#pragma unroll
        for (int j = 0; j < MAX_A; ++j) gWa[j][i] = 0.f;
    }
    float gba = 0.f, gls = 0.f, gbc = 0.f;     // lane j < A owns action dim j
    float st_surr = 0.f, st_vl = 0.f, st_kl = 0.f, st_clip = 0.f;
    __nv_bfloat16* stA = stage + (size_t)warp * 2 * LH_ROWS * SP;
    __nv_bfloat16* stC = stA + LH_ROWS * SP;

    float* sd = sdat + (size_t)warp * LH_ROWS * LH_SD;
    const int nchunks = (p.M + LH_ROWS - 1) / LH_ROWS;
    for (int ch = blockIdx.x * LH_WARPS + warp; ch < nchunks; ch += gridDim.x * LH_WARPS) {
        const int m0 = ch * LH_ROWS;
        const int rows = min(LH_ROWS, p.M - m0);
        // the chunk's per-sample data, gathered once (two lanes per row, independent loads)
        __syncwarp();
        {
            const int r = lane >> 1, h = lane & 1;
            if (r < rows) {
                const int s = p.idx ? __ldg(p.idx + m0 + r) : m0 + r;
                float* d = sd + r * LH_SD;
                const float* src = h ? p.mu_old : p.a_old;
#pragma unroll
                for (int j = 0; j < MAX_A; ++j)
                    if (j < A) d[h * 12 + j] = __ldg(src + (size_t)s * A + j);
                if (h == 0) {
                    d[24] = __ldg(p.logp_old + s);
                    d[25] = __ldg(p.adv + s);
                } else {
                    d[26] = __ldg(p.v_old + s);
                    d[27] = __ldg(p.ret + s);
                }
            }
        }
        __syncwarp();
        for (int r = 0; r < rows; ++r) {
            const int m = m0 + r;
            const float* d = sd + r * LH_SD;
            float ha[NK], hc[NK];
            float v = 0.f;
#pragma unroll
            for (int i = 0; i < NK; ++i) {
                ha[i] = ld_act<BF16>(p.ha, (size_t)m * H + lane + 32 * i);
                hc[i] = ld_act<BF16>(p.hc, (size_t)m * H + lane + 32 * i);
                v += hc[i] * Wc[lane + 32 * i];
            }
            float mu[MAX_A];
#pragma unroll
            for (int j = 0; j < MAX_A; ++j) {
                float t = 0.f;
                if (j < A) {
#pragma unroll
                    for (int i = 0; i < NK; ++i) t += ha[i] * Wa[j * H + lane + 32 * i];
                }
                mu[j] = t;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                v += __shfl_xor_sync(0xffffffffu, v, o);
#pragma unroll
                for (int j = 0; j < MAX_A; ++j) mu[j] += __shfl_xor_sync(0xffffffffu, mu[j], o);
            }
            v += p.bc[0];
            // per-sample loss terms (every lane computes the same scalars)
            float logp = 0.f, kl = 0.f;
#pragma unroll
            for (int j = 0; j < MAX_A; ++j) {
                if (j < A) {
                    mu[j] += p.ba[j];
                    const float ls = cst[j], iv = cst[16 + j];
                    const float diff = d[j] - mu[j];
                    logp += -0.5f * diff * diff * iv - ls - HALF_LOG_2PI;
                    const float dm = d[12 + j] - mu[j];
                    kl += ls - cst[48 + j] + 0.5f * (cst[32 + j] + dm * dm) * iv - 0.5f;
                    mu[j] = diff;          // keep a - mu for the gradient
                }
            }
            const float ratio = expf(logp - d[24]);
            const float adv = d[25];
            const float s1 = ratio * adv;
            const float s2 = fminf(fmaxf(ratio, 1.f - p.clip), 1.f + p.clip) * adv;
            const float g_logp = -(s1 <= s2 ? adv : 0.f) * inv_M * ratio;
            const float vo = d[26], R = d[27];
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
                gbc += g_v;
            }
            float gmu[MAX_A];
#pragma unroll
            for (int j = 0; j < MAX_A; ++j) {
                gmu[j] = 0.f;
                if (j < A) {
                    const float iv = cst[16 + j];
                    gmu[j] = g_logp * mu[j] * iv;
                    if (lane == j) {
                        gba += gmu[j];
                        gls += g_logp * (mu[j] * mu[j] * iv - 1.f);
                    }
                }
            }
            // backward into the last hidden layer and the head weight gradients
#pragma unroll
            for (int i = 0; i < NK; ++i) {
                const int k = lane + 32 * i;
                float da = 0.f;
#pragma unroll
                for (int j = 0; j < MAX_A; ++j) {
                    if (j < A) {
                        da += gmu[j] * Wa[j * H + k];
                        gWa[j][i] += gmu[j] * ha[i];
                    }
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
                    stA[r * SP + k] = ba16;
                    stC[r * SP + k] = bc16;
                } else {
                    reinterpret_cast<float*>(p.dya)[(size_t)m * H + k] = da;
                    reinterpret_cast<float*>(p.dyc)[(size_t)m * H + k] = dc;
                }
            }
        }
        if (BF16) {
            // transposed copies: hidden unit k -> rows m0 .. m0 + rows - 1, 64 contiguous bytes
            __syncwarp();
            __nv_bfloat16* ta = reinterpret_cast<__nv_bfloat16*>(p.dya_t);
            __nv_bfloat16* tc = reinterpret_cast<__nv_bfloat16*>(p.dyc_t);
            if (lane < rows) {
                for (int k = 0; k < H; ++k) {
                    ta[(size_t)k * p.ldt + m0 + lane] = stA[lane * SP + k];
                    tc[(size_t)k * p.ldt + m0 + lane] = stC[lane * SP + k];
                }
            }
            __syncwarp();
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
        for (int w = 0; w < LH_WARPS; ++w) v += accw[(size_t)w * PF + i];
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
    // all threads of the last block sum the per-block statistics (strided, then in thread order)
    __shared__ float red[4][LH_WARPS * 32];
    {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
            const float* q = p.part + (size_t)b * PF + O_ST;
            a0 += __ldcg(q); a1 += __ldcg(q + 1); a2 += __ldcg(q + 2); a3 += __ldcg(q + 3);
        }
        red[0][threadIdx.x] = a0; red[1][threadIdx.x] = a1; red[2][threadIdx.x] = a2; red[3][threadIdx.x] = a3;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double su = 0.0, vl = 0.0, klsum = 0.0, cl = 0.0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            su += red[0][t]; vl += red[1][t]; klsum += red[2][t]; cl += red[3][t];
        }
        float ent = 0.f;
        for (int j = 0; j < A; ++j) ent += cst[j] + HALF_LOG_2PI + 0.5f;
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
            const float t = sc[SC_STEP] + 1.f;
            sc[SC_STEP] = t;
            // Adam's bias corrections for this step, once (float64 is slow on this part):
            // step size alpha / (1 - 0.9^t) and 1 / sqrt(1 - 0.999^t)
            sc[SC_STEPSIZE] = (float)((double)alpha / (1.0 - pow(0.9, (double)t)));
            sc[SC_INVSQRT_BC2] = (float)(1.0 / sqrt(1.0 - pow(0.999, (double)t)));
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
    const int chunks = (M + LH_ROWS - 1) / LH_ROWS;
    int b = (chunks + LH_WARPS - 1) / LH_WARPS;
    return b < 1 ? 1 : (b > 3 * 148 ? 3 * 148 : b);
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
    loss_head_kernel<BF16, NK><<<p.nblocks, LH_WARPS * 32, smem, s>>>(p);
    return cudaGetLastError();
}

static size_t loss_head_smem(int A, int H, bool bf16) {
    return (size_t)(A * H + H + 64 + LH_WARPS * head_part_floats(A, H) + LH_WARPS * LH_ROWS * LH_SD) * sizeof(float) +
           (bf16 ? (size_t)LH_WARPS * 2 * LH_ROWS * (H + 2) * 2 : 0);
}

// Largest dynamic shared memory of the loss head (A = 12, H = 256), set once before any
// launch (and so before any stream capture).
void heads_prepare() {
    const int smem = (int)loss_head_smem(12, 256, true);
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
    const size_t smem = loss_head_smem(p.A, p.H, p.bf16 != 0);
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
