// Output heads of the actor and critic and the per-sample PPO loss with its hand-written
// backward through the heads (Sec. 2.2, Table 3, Algorithm 1).
//
// One warp per sample row: the lanes split the last hidden layer (coalesced row loads), the
// 12 actor outputs and the value are finished with xor-shuffle reductions, so every lane holds
// the whole per-sample state (mu, V, ratio, gradients) and the backward into the hidden layer
// is written back coalesced.  Reductions over the minibatch (head weight / bias gradients,
// log-std gradient, bias gradient of the last hidden layer, loss terms, KL) accumulate per
// warp in registers, then per block in shared memory, then as one partial per block;
// loss_stats_kernel then reduces the statistics, takes the KL mean and applies Algorithm 1 to the
// device-side learning rate before Adam runs.
#include <type_traits>

#include "act_row.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace rl {

namespace {

constexpr int HEAD_WARPS = 8;
constexpr int MAX_A = 12;         // action dims (12 joint targets)

template <bool BF16, int NK>
__global__ void __launch_bounds__(HEAD_WARPS * 32) act_head_kernel(HeadParams p) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ float sm[];
    float* Wa = sm;                 // [A][H]
    float* Wc = sm + p.A * p.H;     // [H]
    const bool actor = p.mu != nullptr || p.actions != nullptr || p.logp != nullptr;
    for (int i = threadIdx.x; i < p.A * p.H; i += blockDim.x) Wa[i] = actor ? p.Wa[i] : 0.f;
    for (int i = threadIdx.x; i < p.H; i += blockDim.x) Wc[i] = p.Wc[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long it = p.iteration ? *p.iteration : 0ull;
    for (int m = blockIdx.x * HEAD_WARPS + warp; m < p.M; m += gridDim.x * HEAD_WARPS)
        act_row<BF16, NK>(p, Wa, Wc, m, it, actor, lane, nullptr, nullptr);
}

// Loss head: four threads per minibatch row, LR rows per block.  The rows' last hidden
// activations (actor and critic) are staged in shared memory with a padded pitch (reads across
// the rows of a warp are then conflict-free); each of a row's four threads takes a quarter of
// the hidden units for the head outputs and for the backward into the hidden layer, and the
// quarter sums are combined in a fixed order by the row's first thread, which computes the
// per-sample loss terms and their gradients.  The head weight gradients are computed by
// (hidden unit, row range) threads whose partials are combined in a fixed order, and the
// gradient rows are written back from shared memory by whole warps.  Every reduction runs in a
// fixed order, so the result does not depend on scheduling.
template <typename T>
struct Tile;
template <>
struct Tile<float> {
    static constexpr int PAD = 1;       // words
    __device__ static float ld(const float* t, int i) { return t[i]; }
    __device__ static void st(float* t, int i, float v) { t[i] = v; }
};
template <>
struct Tile<__nv_bfloat16> {
    static constexpr int PAD = 2;       // elements (one word)
    __device__ static float ld(const __nv_bfloat16* t, int i) { return bf2f(t[i]); }
    __device__ static void st(__nv_bfloat16* t, int i, float v) { t[i] = f2bf(v); }
};

constexpr int LH_TPR = 4;           // threads per row (each owns H / 4 hidden units of the row)
constexpr int LH_GP = 13;           // pitch of the [12 g_mu, g_v] rows (odd: conflict-free)
constexpr int LH_RP = 17;           // pitch of the per-row records (surr, vloss, kl, clip, g_ls[12])

template <int H, int LR>
struct LossShape {
    static constexpr int NT = LR * LH_TPR;         // threads
    static constexpr int QW = NT / H;              // threads per hidden unit in the weight gradient
    static constexpr int FWD = (LH_TPR - 1) * LR * LH_GP;   // forward partials of quarters 1..3
    static constexpr int WG = (QW - 1) * H * LH_GP;          // weight-gradient partials of ranges 1..
    static constexpr int SCR = FWD > WG ? FWD : WG;
    // floats: WaT, Wc, constants, g rows, records, scratch
    static constexpr int FLOATS = H * MAX_A + H + 64 + LR * LH_GP + LR * LH_RP + SCR;
    static_assert(NT % H == 0 && QW >= 1 && LR % QW == 0, "loss head shape");
};

template <bool BF16, int H, int LR>
__global__ void __launch_bounds__(LR * LH_TPR, 2) loss_head_kernel(HeadParams p) {
    pdl_wait();
    pdl_trigger();
    using T = typename std::conditional<BF16, __nv_bfloat16, float>::type;
    using S = LossShape<H, LR>;
    constexpr int SP = H + Tile<T>::PAD;           // tile pitch (elements)
    constexpr int NT = S::NT;
    constexpr int HQ = H / LH_TPR;                 // hidden units per thread of a row
    constexpr int QW = S::QW;
    constexpr int RQ = LR / QW;                    // rows per weight-gradient range
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int A = p.A;
    float* WaT = reinterpret_cast<float*>(sm_raw);          // [H][12] (transposed head weights)
    float* Wc = WaT + H * MAX_A;                            // [H]
    float* cst = Wc + H;                                    // [64]
    float* gmu_s = cst + 64;                                // [LR][13]: g_mu (12) and g_v
    float* recs = gmu_s + LR * LH_GP;                       // [LR][17]
    float* scr = recs + LR * LH_RP;                         // scratch (partials)
    T* ta = reinterpret_cast<T*>(scr + S::SCR);             // [LR][SP] actor h rows, then d/dh
    T* tc = ta + LR * SP;                                   // [LR][SP] critic
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r = tid % LR, part = tid / LR;                // row of the block, quarter of the units
    const int m0 = blockIdx.x * LR;
    const int rows = max(0, min(LR, p.M - m0));   // blocks past M leave zero records
    for (int i = tid; i < H * MAX_A; i += NT) {
        const int k = i / MAX_A, j = i % MAX_A;
        WaT[i] = j < A ? p.Wa[j * H + k] : 0.f;
    }
    for (int i = tid; i < H; i += NT) Wc[i] = p.Wc[i];
    if (tid < A) {
        const float ls = p.log_std[tid], lso = p.log_std_old[tid];
        cst[tid] = ls;
        cst[16 + tid] = expf(-2.f * ls);
        // KL(pi_old || pi) per dimension = (ls - lso) + (sigma_old^2 / sigma^2 - 1) / 2 + dm^2 / (2 sigma^2);
        // its sample-independent part, with d = lso - ls, is expm1(2 d) / 2 - d: written this way it
        // has no cancellation between terms near 1/2 (the KL of a small policy change is small)
        const float dls = lso - ls;
        cst[32 + tid] = 0.5f * expm1f(2.f * dls) - dls;
    }
    // stage the rows (coalesced 4-byte words)
    {
        const T* ga = reinterpret_cast<const T*>(p.ha) + (size_t)m0 * H;
        const T* gc = reinterpret_cast<const T*>(p.hc) + (size_t)m0 * H;
        constexpr int EPW = 4 / sizeof(T);                  // elements per word
        for (int w = tid; w < rows * (H / EPW); w += NT) {
            const int rr = w / (H / EPW), c = (w % (H / EPW)) * EPW;
            if (BF16) {
                *reinterpret_cast<uint32_t*>(ta + rr * SP + c) = *reinterpret_cast<const uint32_t*>(ga + (size_t)rr * H + c);
                *reinterpret_cast<uint32_t*>(tc + rr * SP + c) = *reinterpret_cast<const uint32_t*>(gc + (size_t)rr * H + c);
            } else {
                ta[rr * SP + c] = ga[(size_t)rr * H + c];
                tc[rr * SP + c] = gc[(size_t)rr * H + c];
            }
        }
    }
    const bool live = r < rows;
    __syncthreads();

    // ---- forward of the heads over this thread's quarter of the hidden units
    float mu[MAX_A], v = 0.f;
#pragma unroll
    for (int j = 0; j < MAX_A; ++j) mu[j] = 0.f;
    if (live) {
        const T* hr = ta + r * SP;
        const T* cr = tc + r * SP;
#pragma unroll 4
        for (int k = part * HQ; k < (part + 1) * HQ; ++k) {
            const float h = Tile<T>::ld(hr, k);
            const float4* w4 = reinterpret_cast<const float4*>(WaT + k * MAX_A);
            const float4 w0 = w4[0], w1 = w4[1], w2 = w4[2];
            mu[0] += h * w0.x; mu[1] += h * w0.y; mu[2] += h * w0.z; mu[3] += h * w0.w;
            mu[4] += h * w1.x; mu[5] += h * w1.y; mu[6] += h * w1.z; mu[7] += h * w1.w;
            mu[8] += h * w2.x; mu[9] += h * w2.y; mu[10] += h * w2.z; mu[11] += h * w2.w;
            v += Tile<T>::ld(cr, k) * Wc[k];
        }
    }
    if (part > 0) {
        float* d = scr + ((size_t)(part - 1) * LR + r) * LH_GP;
#pragma unroll
        for (int j = 0; j < MAX_A; ++j) d[j] = mu[j];
        d[12] = v;
    }
    __syncthreads();
    // ---- per row (the row's first thread): loss terms and gradients w.r.t. mu and V
    if (part == 0) {
        const int m = m0 + r;
        const int s = live ? (p.idx ? __ldg(p.idx + m) : m) : 0;
        // quarter sums in order 0, 1, 2, 3, then the bias
#pragma unroll
        for (int q = 1; q < LH_TPR; ++q) {
            const float* d = scr + ((size_t)(q - 1) * LR + r) * LH_GP;
#pragma unroll
            for (int j = 0; j < MAX_A; ++j) mu[j] += d[j];
            v += d[12];
        }
#pragma unroll
        for (int j = 0; j < MAX_A; ++j) mu[j] += j < A ? p.ba[j] : 0.f;
        v += p.bc[0];
        float logp = 0.f, kl = 0.f, diff[MAX_A];
#pragma unroll
        for (int j = 0; j < MAX_A; ++j) {
            diff[j] = 0.f;
            if (j < A && live) {
                const float ls = cst[j], iv = cst[16 + j];
                diff[j] = __ldg(p.a_old + (size_t)s * A + j) - mu[j];
                logp += -0.5f * diff[j] * diff[j] * iv - ls - HALF_LOG_2PI;
                const float dm = __ldg(p.mu_old + (size_t)s * A + j) - mu[j];
                kl += cst[32 + j] + 0.5f * dm * dm * iv;
            }
        }
        const float lpo = live ? __ldg(p.logp_old + s) : 0.f;
        const float adv = live ? __ldg(p.adv + s) : 0.f;
        const float vo = live ? __ldg(p.v_old + s) : 0.f;
        const float R = live ? __ldg(p.ret + s) : 0.f;
        const float inv_M = 1.0f / (float)p.M;
        const float ratio = expf(logp - lpo);
        const float s1 = ratio * adv;
        const float s2 = fminf(fmaxf(ratio, 1.f - p.clip), 1.f + p.clip) * adv;
        const float g_logp = -(s1 <= s2 ? adv : 0.f) * inv_M * ratio;
        const float dv = v - vo;
        const float vclip = vo + fminf(fmaxf(dv, -p.clip), p.clip);
        const float u = (v - R) * (v - R), w = (vclip - R) * (vclip - R);
        float g_v = p.value_coef * inv_M * (u >= w ? 2.f * (v - R) : ((dv > -p.clip && dv < p.clip) ? 2.f * (vclip - R) : 0.f));
        if (!live) g_v = 0.f;
        float* rc = recs + r * LH_RP;
        rc[0] = live ? fminf(s1, s2) : 0.f;
        rc[1] = live ? fmaxf(u, w) : 0.f;
        rc[2] = live ? kl : 0.f;
        rc[3] = (live && fabsf(ratio - 1.f) > p.clip) ? 1.f : 0.f;
#pragma unroll
        for (int j = 0; j < MAX_A; ++j) {
            const float iv = j < A ? cst[16 + j] : 0.f;
            gmu_s[r * LH_GP + j] = (live && j < A) ? g_logp * diff[j] * iv : 0.f;
            rc[4 + j] = (live && j < A) ? g_logp * (diff[j] * diff[j] * iv - 1.f) : 0.f;
        }
        gmu_s[r * LH_GP + 12] = g_v;
    }
    __syncthreads();

    // ---- head weight gradients: thread (unit k, row range q); ranges combined by q = 0 in order
    const HeadPart hp = head_part(A, H);
    const int PF = hp.PF, O_WA = hp.WA, O_BA = hp.BA, O_LS = hp.LS, O_WC = hp.WC, O_BC = hp.BC, O_DBA = hp.DBA,
              O_DBC = hp.DBC, O_ST = hp.ST;
    float* out = p.part + (size_t)blockIdx.x * PF;
    const int k = tid % H, q = tid / H;
    float acc[MAX_A], accc = 0.f;
#pragma unroll
    for (int j = 0; j < MAX_A; ++j) acc[j] = 0.f;
    for (int rr = q * RQ; rr < min(rows, (q + 1) * RQ); ++rr) {
        const float h = Tile<T>::ld(ta + rr * SP, k);
        const float* g = gmu_s + rr * LH_GP;
#pragma unroll
        for (int j = 0; j < MAX_A; ++j) acc[j] += g[j] * h;
        accc += g[12] * Tile<T>::ld(tc + rr * SP, k);
    }
    if (q > 0) {
        float* d = scr + ((size_t)(q - 1) * H + k) * LH_GP;
#pragma unroll
        for (int j = 0; j < MAX_A; ++j) d[j] = acc[j];
        d[12] = accc;
    }
    __syncthreads();
    if (q == 0) {
        for (int qq = 1; qq < QW; ++qq) {
            const float* d = scr + ((size_t)(qq - 1) * H + k) * LH_GP;
#pragma unroll
            for (int j = 0; j < MAX_A; ++j) acc[j] += d[j];
            accc += d[12];
        }
#pragma unroll
        for (int j = 0; j < MAX_A; ++j)
            if (j < A) out[O_WA + j * H + k] = acc[j];
        out[O_WC + k] = accc;
    }

    // ---- backward into the last hidden layer (in place in the tiles)
    if (live) {
        T* hr = ta + r * SP;
        T* cr = tc + r * SP;
        float gmu[MAX_A];
#pragma unroll
        for (int j = 0; j < MAX_A; ++j) gmu[j] = gmu_s[r * LH_GP + j];
        const float g_v = gmu_s[r * LH_GP + 12];
#pragma unroll 4
        for (int kk = part * HQ; kk < (part + 1) * HQ; ++kk) {
            const float4* w4 = reinterpret_cast<const float4*>(WaT + kk * MAX_A);
            const float4 w0 = w4[0], w1 = w4[1], w2 = w4[2];
            float da = gmu[0] * w0.x + gmu[1] * w0.y + gmu[2] * w0.z + gmu[3] * w0.w + gmu[4] * w1.x + gmu[5] * w1.y +
                       gmu[6] * w1.z + gmu[7] * w1.w + gmu[8] * w2.x + gmu[9] * w2.y + gmu[10] * w2.z + gmu[11] * w2.w;
            da *= elu_grad_y(Tile<T>::ld(hr, kk));
            const float dc = g_v * Wc[kk] * elu_grad_y(Tile<T>::ld(cr, kk));
            Tile<T>::st(hr, kk, da);
            Tile<T>::st(cr, kk, dc);
        }
    }
    __syncthreads();

    // ---- bias gradient of the last hidden layer (column sums) and the block's statistics:
    // items [0, H) actor columns, [H, 2H) critic columns, [2H, 2H + 29) record columns
    for (int i = tid; i < 2 * H + 29; i += NT) {
        if (i < 2 * H) {
            const T* t = i < H ? ta : tc;
            const int kk = i < H ? i : i - H;
            float sum = 0.f;
            for (int rr = 0; rr < rows; ++rr) sum += Tile<T>::ld(t + rr * SP, kk);
            out[(i < H ? O_DBA : O_DBC) + kk] = sum;
        } else {
            // record column c: 0..3 loss terms, 4 g_v, 5..16 g_mu, 17..28 g_log_std
            const int c = i - 2 * H;
            const float* col = c < 4 ? recs + c : c == 4 ? gmu_s + 12 : c < 17 ? gmu_s + (c - 5) : recs + 4 + (c - 17);
            const int pitch = (c >= 4 && c < 17) ? LH_GP : LH_RP;
            float sum = 0.f;
            for (int rr = 0; rr < LR; ++rr) sum += col[rr * pitch];
            if (c < 4) out[O_ST + c] = sum;
            else if (c == 4) out[O_BC] = sum;
            else if (c < 17) { if (c - 5 < A) out[O_BA + c - 5] = sum; }
            else if (c - 17 < A) out[O_LS + c - 17] = sum - (blockIdx.x == 0 ? p.entropy_coef : 0.f);
        }
    }
    if (tid >= 4 && tid < 8) out[O_ST + tid] = 0.f;
    // ---- gradient rows out (row-major)
    {
        T* gda = reinterpret_cast<T*>(p.dya);
        T* gdc = reinterpret_cast<T*>(p.dyc);
        for (int rr = warp; rr < rows; rr += NT / 32)
            for (int kk = lane; kk < H; kk += 32) {
                gda[(size_t)(m0 + rr) * H + kk] = ta[rr * SP + kk];
                gdc[(size_t)(m0 + rr) * H + kk] = tc[rr * SP + kk];
            }
    }

    // the minibatch statistics and Algorithm 1 follow in loss_stats_kernel
}

}  // namespace

template <bool BF16, int NK>
static cudaError_t act_dispatch(const HeadParams& p, int blocks, size_t smem, cudaStream_t s) {
    cudaError_t e = launch_pdl(act_head_kernel<BF16, NK>, dim3(blocks), dim3(HEAD_WARPS * 32), smem, s, p);
    if (e != cudaSuccess) return e;
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

template <bool BF16, int H, int LR>
static size_t loss_head_smem_t() {
    using T = typename std::conditional<BF16, __nv_bfloat16, float>::type;
    return (size_t)LossShape<H, LR>::FLOATS * sizeof(float) + (size_t)2 * LR * (H + Tile<T>::PAD) * sizeof(T);
}

template <bool BF16, int H, int LR>
static cudaError_t loss_dispatch(const HeadParams& p, cudaStream_t s) {
    cudaError_t e = launch_pdl(loss_head_kernel<BF16, H, LR>, dim3(p.nblocks), dim3(LR * LH_TPR), loss_head_smem_t<BF16, H, LR>(), s, p);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <bool BF16, int H, int LR>
static void loss_prepare() {
    cudaFuncSetAttribute(loss_head_kernel<BF16, H, LR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)loss_head_smem_t<BF16, H, LR>());
}

// Dynamic shared-memory limits of every loss-head instantiation, set once before any launch
// (and so before any stream capture).
void heads_prepare() {
    loss_mma_prepare();
    loss_prepare<false, 64, 128>();
    loss_prepare<false, 128, 128>();
    loss_prepare<false, 256, 64>();
}

// 128 rows per block (64 when the last hidden layer is 256 wide, to fit the tiles).
int loss_head_rows(int H) { return H >= 256 ? 64 : 128; }

int loss_head_blocks(int M, int H, int bf16) {
    const int rows = bf16 ? loss_mma_rows() : loss_head_rows(H);
    return (M + rows - 1) / rows;
}

cudaError_t launch_loss_head(const HeadParams& p, cudaStream_t s) {
    if (p.M <= 0) return cudaSuccess;
    if (p.A > MAX_A || !(p.H == 64 || p.H == 128 || p.H == 256)) return cudaErrorInvalidValue;
    // blocks past the rows leave zero partials, so a launch may have more blocks than its rows
    // need (the context sizes them for the full minibatch)
    if (p.nblocks < loss_head_blocks(p.M, p.H, p.bf16)) return cudaErrorInvalidValue;
    if (p.bf16) return launch_loss_mma(p, s);    // tensor-core form (loss_mma.cu)
    if (p.H == 64) return loss_dispatch<false, 64, 128>(p, s);
    if (p.H == 128) return loss_dispatch<false, 128, 128>(p, s);
    return loss_dispatch<false, 256, 64>(p, s);
}

}  // namespace rl
