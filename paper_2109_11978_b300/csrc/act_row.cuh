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

// Rows m[0..R) by the calling warp, processed together so that the loads and shuffle chains of
// one row overlap those of the other (the same operations per row as one at a time).  Rows with
// ok[r] false are computed on row m[0] and write nothing.  Wa [A][H] and Wc [H] in shared memory
// (fp32).  Writes p.values[m] and, with actor, p.mu / p.actions / p.logp where non-null;
// a_sm[r] [A] / v_sm[r] (shared memory, optional) receive the sampled action and the value too.
// The rows' last hidden activations (lane l: units l, l + 32, ...), loaded by act_rows or ahead
// of it (the fused env step issues them before it stages the head weights).
template <bool BF16, int NK, int R>
__device__ __forceinline__ void act_rows_load(const HeadParams& p, const int (&m_in)[R], const bool (&ok)[R], bool actor,
                                              int lane, float (&hc)[R][NK], float (&ha)[R][NK]) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int m = ok[r] ? m_in[r] : m_in[0];
#pragma unroll
        for (int i = 0; i < NK; ++i) {
            hc[r][i] = ld_act<BF16>(p.hc, (size_t)m * p.H + lane + 32 * i);
            if (actor) ha[r][i] = ld_act<BF16>(p.ha, (size_t)m * p.H + lane + 32 * i);
        }
    }
}

// act_rows on rows already loaded by act_rows_load.
template <bool BF16, int NK, int R>
__device__ __forceinline__ void act_rows_loaded(const HeadParams& p, const float* Wa, const float* Wc, const int (&m_in)[R],
                                                const bool (&ok)[R], unsigned long long it, bool actor, int lane,
                                                float* const (&a_sm)[R], float* const (&v_sm)[R], const float (&hc)[R][NK],
                                                const float (&ha)[R][NK]) {
    int m[R];
#pragma unroll
    for (int r = 0; r < R; ++r) m[r] = ok[r] ? m_in[r] : m_in[0];
    float v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        v[r] = 0.f;
#pragma unroll
        for (int i = 0; i < NK; ++i) v[r] += hc[r][i] * Wc[lane + 32 * i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] += __shfl_xor_sync(0xffffffffu, v[r], o);
    if (lane == 0)
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (ok[r]) {
                p.values[m[r]] = v[r] + p.bc[0];
                if (v_sm[r]) *v_sm[r] = v[r] + p.bc[0];
            }
    if (!actor) return;
    // the A (<= 16) per-lane partial dot products, summed over the warp by a reduce-scatter:
    // each xor step (16, 8, 4, 2) hands half of the lane's values to its partner and keeps the
    // other half, so that after four steps lane l holds the 16-lane sum of output (l >> 1) and the
    // xor-1 step completes it (16 shuffles for all outputs instead of 5 per output)
    float s[R][16];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            s[r][j] = 0.f;
            if (j < p.A) {
#pragma unroll
                for (int i = 0; i < NK; ++i) s[r][j] += ha[r][i] * Wa[j * p.H + lane + 32 * i];
            }
        }
#pragma unroll
    for (int st = 0; st < 4; ++st) {
        const int o = 16 >> st, n = 8 >> st;          // partner offset, values kept after the step
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float send = up ? s[r][k] : s[r][k + n];
                const float keep = up ? s[r][k + n] : s[r][k];
                s[r][k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
    }
    float lp[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        s[r][0] += __shfl_xor_sync(0xffffffffu, s[r][0], 1);
        // output j sits on lanes 2j and 2j + 1
        const float tot = __shfl_sync(0xffffffffu, s[r][0], (2 * lane) & 31);
        const float mine = lane < p.A ? tot + p.ba[lane] : 0.f;   // mu of action dim == lane
        lp[r] = 0.f;
        if (lane < p.A) {
            const float ls = p.log_std[lane];
            const uint64_t key = rng_key(p.seed, kStreamAct, it, (uint64_t)p.t, (uint64_t)m[r]);
            const float eps = box_muller(rng_word(key, (uint32_t)lane));
            const float a = mine + expf(ls) * eps;
            lp[r] = -0.5f * eps * eps - ls - HALF_LOG_2PI;
            if (ok[r]) {
                if (p.mu) p.mu[(size_t)m[r] * p.A + lane] = mine;
                if (p.actions) p.actions[(size_t)m[r] * p.A + lane] = a;
                if (a_sm[r]) a_sm[r][lane] = a;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int r = 0; r < R; ++r) lp[r] += __shfl_xor_sync(0xffffffffu, lp[r], o);
    if (lane == 0 && p.logp)
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (ok[r]) p.logp[m[r]] = lp[r];
}

template <bool BF16, int NK, int R>
__device__ __forceinline__ void act_rows(const HeadParams& p, const float* Wa, const float* Wc, const int (&m_in)[R],
                                         const bool (&ok)[R], unsigned long long it, bool actor, int lane,
                                         float* const (&a_sm)[R], float* const (&v_sm)[R]) {
    float hc[R][NK], ha[R][NK];
    act_rows_load<BF16, NK, R>(p, m_in, ok, actor, lane, hc, ha);
    act_rows_loaded<BF16, NK, R>(p, Wa, Wc, m_in, ok, it, actor, lane, a_sm, v_sm, hc, ha);
}

// One row m by the calling warp (act_rows with R = 1).
template <bool BF16, int NK>
__device__ __forceinline__ void act_row(const HeadParams& p, const float* Wa, const float* Wc, int m, unsigned long long it,
                                        bool actor, int lane, float* a_sm, float* v_sm) {
    const int mm[1] = {m};
    const bool ok[1] = {true};
    float* const as[1] = {a_sm};
    float* const vs[1] = {v_sm};
    act_rows<BF16, NK, 1>(p, Wa, Wc, mm, ok, it, actor, lane, as, vs);
}

}  // namespace rl
