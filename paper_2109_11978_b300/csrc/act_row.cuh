// Output heads of one rollout row (Sec. 2.2), shared by the action-head kernel and the env step
// that fuses it: a warp per row, the lanes split the last hidden layer (coalesced row loads) and
// finish the actor outputs with one reduce-scatter and the value with an xor-shuffle reduction; the Gaussian policy
// samples a = mu + exp(log_std) eps with eps from the counter-based generator keyed by
// (seed, iteration, t, row), and logp is the sum of the per-dimension log densities.
#pragma once
#include "common.cuh"
#include "kernels.cuh"

namespace rl {

constexpr float HALF_LOG_2PI = 0.91893853320467274f;

template <bool BF16>
__device__ __forceinline__ float ld_act(const void* base, size_t i) {
    if (BF16) return bf2f(reinterpret_cast<const __nv_bfloat16*>(base)[i]);
    return reinterpret_cast<const float*>(base)[i];
}

// Row m by the calling warp.  Wa [A][H] and Wc [H] in shared memory (fp32).  Writes p.values[m]
// and, with actor, p.mu / p.actions / p.logp where non-null; a_sm [A] / v_sm (shared memory,
// optional) receive the sampled action and the value too.
template <bool BF16, int NK>
__device__ __forceinline__ void act_row(const HeadParams& p, const float* Wa, const float* Wc, int m, unsigned long long it,
                                        bool actor, int lane, float* a_sm, float* v_sm) {
    float hc[NK];
    float v = 0.f;
#pragma unroll
    for (int i = 0; i < NK; ++i) {
        hc[i] = ld_act<BF16>(p.hc, (size_t)m * p.H + lane + 32 * i);
        v += hc[i] * Wc[lane + 32 * i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) {
        p.values[m] = v + p.bc[0];
        if (v_sm) *v_sm = v + p.bc[0];
    }
    if (!actor) return;
    float ha[NK];
#pragma unroll
    for (int i = 0; i < NK; ++i) ha[i] = ld_act<BF16>(p.ha, (size_t)m * p.H + lane + 32 * i);
    // the A (<= 16) per-lane partial dot products, summed over the warp by a reduce-scatter:
    // each xor step (16, 8, 4, 2) hands half of the lane's values to its partner and keeps the
    // other half, so that after four steps lane l holds the 16-lane sum of output (l >> 1) and the
    // xor-1 step completes it (16 shuffles for all outputs instead of 5 per output)
    float s[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        s[j] = 0.f;
        if (j < p.A) {
#pragma unroll
            for (int i = 0; i < NK; ++i) s[j] += ha[i] * Wa[j * p.H + lane + 32 * i];
        }
    }
#pragma unroll
    for (int st = 0; st < 4; ++st) {
        const int o = 16 >> st, n = 8 >> st;          // partner offset, values kept after the step
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < n; ++k) {
            const float send = up ? s[k] : s[k + n];
            const float keep = up ? s[k + n] : s[k];
            s[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    s[0] += __shfl_xor_sync(0xffffffffu, s[0], 1);
    // output j sits on lanes 2j and 2j + 1
    const float tot = __shfl_sync(0xffffffffu, s[0], (2 * lane) & 31);
    const float mine = lane < p.A ? tot + p.ba[lane] : 0.f;   // mu of action dim == lane
    float lp = 0.f;
    if (lane < p.A) {
        const float ls = p.log_std[lane];
        const uint64_t key = rng_key(p.seed, kStreamAct, it, (uint64_t)p.t, (uint64_t)m);
        const float eps = box_muller(rng_word(key, (uint32_t)lane));
        const float a = mine + expf(ls) * eps;
        lp = -0.5f * eps * eps - ls - HALF_LOG_2PI;
        if (p.mu) p.mu[(size_t)m * p.A + lane] = mine;
        if (p.actions) p.actions[(size_t)m * p.A + lane] = a;
        if (a_sm) a_sm[lane] = a;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lp += __shfl_xor_sync(0xffffffffu, lp, o);
    if (lane == 0 && p.logp) p.logp[m] = lp;
}

}  // namespace rl
