// BF16 form of the loss head (Sec. 2.2, Table 3, Algorithm 1): the heads' forward, the
// per-sample clipped-surrogate / clipped-value loss, and the backward through the heads, with
// the three small products on the warp-level tensor-core MMA
// (mma.sync m16n8k16, bf16 operands, fp32 accumulation), 64 rows per block (4 warps x 16):
//
//   mu  = H_a Wa^T + ba        [64 x 12]    (actor; V = H_c Wc^T + bc the same way, one column)
//   dWa = G^T H_a              [12 x H]     G = d loss / d mu, per row
//   dH_a = (G Wa) * ELU'(H_a)  [64 x H]     (critic: dH_c = g_v Wc * ELU'(H_c), elementwise)
//
// The last hidden activations are bf16 already; the fp32 operands (head weights, G) are split
// into a bf16 high part and a bf16 remainder, and the products hi*hi + hi*lo + lo*hi (weights:
// hi + lo against exact bf16 activations) carry about 16 bits of each operand, which keeps the
// result at fp32 level.  Per-row work (log pi, ratio, clipping, KL) runs one thread per row in
// fp32.  The per-block partials follow the same layout as the FP32 kernel's; the minibatch
// statistics and Algorithm 1 run afterwards in loss_stats_kernel.
#include "common.cuh"
#include "kernels.cuh"

namespace rl {

namespace {

constexpr int MAX_A = 12;
constexpr float HALF_LOG_2PI = 0.91893853320467274f;
constexpr int ROWS = 64;                  // rows per block (4 warps x 16)
// warps per block: eight for H >= 128 (the products split by output columns too), four for
// H = 64; the 64 rows of a block are four 16-row MMA fragments
template <int H>
constexpr int warps_of() { return H >= 128 ? 8 : 4; }
constexpr int GP = 24;                    // bf16 pitch of the [row][16] G tiles and [H][16] WaT tiles
constexpr int FP = 17;                    // fp32 pitch of the [row][16] mu / G tiles
constexpr int RP = 17;                    // per-row records: surr, vloss, kl, clip, g_ls[12]

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(const void* p, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x4_t(const void* p, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x2(const void* p, uint32_t& r0, uint32_t& r1) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(smem_addr(p)));
}

// D += A B, A 16 x 16 (row-major fragments), B 16 x 8 (column-major fragments), fp32 accumulators.
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// 16-byte asynchronous global -> shared copy; src_bytes 0 fills the 16 bytes with zeros
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// fp32 -> bf16 high part and bf16 remainder (x - hi rounded again)
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

template <int H>
struct Smem {
    static constexpr int HP = H + 8;                          // bf16 pitch of the [row][H] tiles
    // bf16 regions (element offsets)
    static constexpr int HA = 0;                              // [ROWS][HP] actor h, then dY_a
    static constexpr int HC = HA + ROWS * HP;                 // [ROWS][HP] critic h, then dY_c
    static constexpr int WA_HI = HC + ROWS * HP;              // [16][HP] Wa (rows j >= A zero)
    static constexpr int WA_LO = WA_HI + 16 * HP;
    static constexpr int WC_HI = WA_LO + 16 * HP;             // [8][HP] Wc in row 0
    static constexpr int WC_LO = WC_HI + 8 * HP;
    static constexpr int WAT_HI = WC_LO + 8 * HP;             // [H][GP] Wa^T
    static constexpr int WAT_LO = WAT_HI + H * GP;
    static constexpr int G_HI = WAT_LO + H * GP;              // [ROWS][GP] G
    static constexpr int G_LO = G_HI + ROWS * GP;
    static constexpr int BF16_END = G_LO + ROWS * GP;
    // fp32 regions (float offsets from the end of the bf16 part, 16-byte aligned)
    static constexpr int F0 = (BF16_END * 2 + 15) / 16 * 4;
    // mu / V rows and the per-row records share one [ROWS][17] area: the row's thread reads
    // its mu row before it writes its record row
    static constexpr int MU = F0;                             // [ROWS][FP]: mu (12) and V at 12
    static constexpr int REC = MU;                            // [ROWS][RP]
    static constexpr int G = MU + ROWS * FP;                  // [ROWS][FP]: g_mu (12) and g_v at 12
    static constexpr int WCF = G + ROWS * FP;                 // [H] Wc fp32
    static constexpr int CST = WCF + H;                       // [64] log-std constants, ba at 48, bc at 60
    static constexpr int FLOATS = CST + 64;
    static constexpr int BYTES = FLOATS * 4;
};

template <int H>
__global__ void __launch_bounds__(32 * warps_of<H>(), H >= 128 ? 3 : 4) loss_mma_kernel(HeadParams p) {
    constexpr int NW = warps_of<H>(), THREADS = 32 * NW;
    // Everything staged before the wait for the preceding kernel (the forward GEMM that writes the
    // last hidden rows) was written by kernels that have completed when this one starts: the
    // packed records and permutation (written once per iteration before the update), the head
    // weights and log-std (Adam of the previous minibatch, which precedes the forward layers).  The
    // hidden rows are copied after the wait.
    using S = Smem<H>;
    constexpr int HP = S::HP;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    __nv_bfloat16* sb = reinterpret_cast<__nv_bfloat16*>(sm_raw);
    float* sf = reinterpret_cast<float*>(sm_raw);
    __nv_bfloat16* ha = sb + S::HA;
    __nv_bfloat16* hc = sb + S::HC;
    float* mu_s = sf + S::MU;
    float* g_s = sf + S::G;
    float* recs = sf + S::REC;
    float* wcf = sf + S::WCF;
    float* cst = sf + S::CST;
    const int A = p.A;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gq = lane >> 2, tq = lane & 3;                  // mma fragment row group / column pair
    const int m0 = blockIdx.x * ROWS;
    const int rows = max(0, min(ROWS, p.M - m0));

    // ---- per-row inputs of the loss, issued first (their latency overlaps the staging): TPR
    // consecutive threads per row, thread q of a row holding dimensions q, q + TPR, ...
    constexpr int TPR = THREADS / ROWS;                       // 4 (2 with four warps)
    constexpr int DPT = MAX_A / TPR;                          // dimensions per thread
    static_assert(TPR * ROWS == THREADS && DPT * TPR == MAX_A && 32 % TPR == 0, "row threads");
    const int rr_ = tid / TPR, qq = tid % TPR;                // the thread's row and quarter
    const bool live = rr_ < rows;
    float aold[DPT], muold[DPT], lpo = 0.f, adv = 0.f, vo = 0.f, R = 0.f;
#pragma unroll
    for (int u = 0; u < DPT; ++u) aold[u] = muold[u] = 0.f;
    if (live) {
        const int m = m0 + rr_;
        const int s = p.idx ? __ldg(p.idx + m) : m;
        if (p.rec) {
            // the sample's packed 128-byte record [a_old A][mu_old A][logp_old][adv][V_old][R]
            const float* rc = p.rec + (size_t)s * p.rec_ld;
#pragma unroll
            for (int u = 0; u < DPT; ++u) {
                const int jj = qq + TPR * u;
                if (jj < A) {
                    aold[u] = __ldg(rc + jj);
                    muold[u] = __ldg(rc + A + jj);
                }
            }
            lpo = __ldg(rc + 2 * A);
            adv = __ldg(rc + 2 * A + 1);
            vo = __ldg(rc + 2 * A + 2);
            R = __ldg(rc + 2 * A + 3);
        } else {
#pragma unroll
            for (int u = 0; u < DPT; ++u) {
                const int jj = qq + TPR * u;
                if (jj < A) {
                    aold[u] = __ldg(p.a_old + (size_t)s * A + jj);
                    muold[u] = __ldg(p.mu_old + (size_t)s * A + jj);
                }
            }
            lpo = __ldg(p.logp_old + s);
            adv = __ldg(p.adv + s);
            vo = __ldg(p.v_old + s);
            R = __ldg(p.ret + s);
        }
    }
    // ---- the critic head's fp32 weights (asynchronous 16-byte copies)
    for (int v = tid; v < H / 4; v += THREADS) cp_async16(wcf + 4 * v, p.Wc + 4 * v, 16);
    // head weights -> bf16 hi / lo tiles (Wa rows j >= A and Wc rows 1..7 zero), read straight from
    // global memory while the row copies are in flight
    {
        constexpr int NWA = 16 * H / THREADS;
#pragma unroll
        for (int u = 0; u < NWA; ++u) {
            const int i = tid + u * THREADS;
            const int j = i / H, k = i % H;
            const float w = j < A ? __ldg(p.Wa + j * H + k) : 0.f;
            __nv_bfloat16 hi, lo;
            split_bf16(w, hi, lo);
            sb[S::WA_HI + j * HP + k] = hi;
            sb[S::WA_LO + j * HP + k] = lo;
            sb[S::WAT_HI + k * GP + j] = hi;
            sb[S::WAT_LO + k * GP + j] = lo;
        }
        for (int i = tid; i < 8 * H; i += THREADS) {
            const int j = i / H, k = i % H;
            const float w = j == 0 ? __ldg(p.Wc + k) : 0.f;
            __nv_bfloat16 hi, lo;
            split_bf16(w, hi, lo);
            sb[S::WC_HI + j * HP + k] = hi;
            sb[S::WC_LO + j * HP + k] = lo;
        }
    }
    if (tid < A) {
        const float ls = p.log_std[tid], lso = p.log_std_old[tid];
        cst[tid] = ls;
        cst[16 + tid] = expf(-2.f * ls);
        // KL(pi_old || pi) per dimension = (ls - lso) + (sigma_old^2 / sigma^2 - 1) / 2 + dm^2 / (2 sigma^2);
        // its sample-independent part, with d = lso - ls, is expm1(2 d) / 2 - d: written this way it
        // has no cancellation between terms near 1/2 (the KL of a small policy change is small)
        const float dls = lso - ls;
        cst[32 + tid] = 0.5f * expm1f(2.f * dls) - dls;
        cst[48 + tid] = p.ba[tid];                           // the heads' biases, with the constants
    }
    if (tid == 0) cst[60] = p.bc[0];
    // the preceding kernel's results (the hidden rows), then the next kernel may be placed
    pdl_wait();
    pdl_trigger();
    // ---- h tiles (asynchronous 16-byte copies, zeros past M)
    {
        const __nv_bfloat16* ga = reinterpret_cast<const __nv_bfloat16*>(p.ha) + (size_t)m0 * H;
        const __nv_bfloat16* gc = reinterpret_cast<const __nv_bfloat16*>(p.hc) + (size_t)m0 * H;
        constexpr int VPR = H / 8;                            // 16-byte vectors per row
        for (int v = tid; v < ROWS * VPR; v += THREADS) {
            const int r = v / VPR, c = (v % VPR) * 8;
            const int rr = r < rows ? r : 0;                  // a valid address; zero-filled
            cp_async16(ha + r * HP + c, ga + (size_t)rr * H + c, r < rows ? 16 : 0);
            cp_async16(hc + r * HP + c, gc + (size_t)rr * H + c, r < rows ? 16 : 0);
        }
    }
    cp_async_wait_all();
    __syncthreads();

    static_assert(FP == RP, "mu rows and records share their rows");
    // ---- heads forward: rows 16 (w % 4) .. + 15; with eight warps the first four take the actor
    // head and the other four the critic head, with four each warp both
    {
        const int r0 = 16 * (warp & 3);
        const bool do_a = NW == 4 || warp < 4, do_c = NW == 4 || warp >= 4;
        float acc[2][4] = {}, accv[4] = {};
#pragma unroll
        for (int ks = 0; ks < H / 16; ++ks) {
            const int k0 = 16 * ks;
            if (do_a) {
                uint32_t a[4];
                ldsm_x4(ha + (r0 + (lane & 15)) * HP + k0 + 8 * (lane >> 4), a[0], a[1], a[2], a[3]);
                // B = Wa^T: fragment rows are Wa rows j (n), columns k
                const int bn = (lane & 7) + 8 * (lane >> 4), bk = k0 + 8 * ((lane >> 3) & 1);
                uint32_t bh[4], bl[4];
                ldsm_x4(sb + S::WA_HI + bn * HP + bk, bh[0], bh[1], bh[2], bh[3]);
                ldsm_x4(sb + S::WA_LO + bn * HP + bk, bl[0], bl[1], bl[2], bl[3]);
                mma16816(acc[0], a, bh[0], bh[1]);
                mma16816(acc[0], a, bl[0], bl[1]);
                mma16816(acc[1], a, bh[2], bh[3]);
                mma16816(acc[1], a, bl[2], bl[3]);
            }
            if (do_c) {
                uint32_t c[4];
                ldsm_x4(hc + (r0 + (lane & 15)) * HP + k0 + 8 * (lane >> 4), c[0], c[1], c[2], c[3]);
                uint32_t ch0, ch1, cl0, cl1;
                const int cn = lane & 7, ck = k0 + 8 * ((lane >> 3) & 1);
                ldsm_x2(sb + S::WC_HI + cn * HP + ck, ch0, ch1);
                ldsm_x2(sb + S::WC_LO + cn * HP + ck, cl0, cl1);
                mma16816(accv, c, ch0, ch1);
                mma16816(accv, c, cl0, cl1);
            }
        }
        // fragments -> [row][16] fp32 (mu columns 0..15, V from column 0 of the critic tile)
        if (do_a) {
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int r = r0 + gq + 8 * h2;
                    mu_s[r * FP + 8 * nt + 2 * tq] = acc[nt][2 * h2];
                    mu_s[r * FP + 8 * nt + 2 * tq + 1] = acc[nt][2 * h2 + 1];
                }
        }
        // column 12 of the actor tile is zero (Wa rows >= A are zero): the critic writes it after
        __syncthreads();
        if (do_c && tq == 0) {
            mu_s[(r0 + gq) * FP + 12] = accv[0];
            mu_s[(r0 + gq + 8) * FP + 12] = accv[2];
        }
    }
    __syncthreads();

    // ---- per row: loss terms, d loss / d mu and d loss / d V; the row's TPR threads split the
    // dimensions and combine their sums by xor shuffles inside their group of lanes
    {
        const int r = rr_;
        float logp = 0.f, kl = 0.f, diff[DPT];
#pragma unroll
        for (int u = 0; u < DPT; ++u) {
            const int jj = qq + TPR * u;
            diff[u] = 0.f;
            if (jj < A && live) {
                const float mu = mu_s[r * FP + jj] + cst[48 + jj];
                const float ls = cst[jj], iv = cst[16 + jj];
                diff[u] = aold[u] - mu;
                logp += -0.5f * diff[u] * diff[u] * iv - ls - HALF_LOG_2PI;
                const float dm = muold[u] - mu;
                kl += cst[32 + jj] + 0.5f * dm * dm * iv;
            }
        }
#pragma unroll
        for (int o = 1; o < TPR; o <<= 1) {
            logp += __shfl_xor_sync(0xffffffffu, logp, o);
            kl += __shfl_xor_sync(0xffffffffu, kl, o);
        }
        const float v = mu_s[r * FP + 12] + cst[60];
        __syncwarp();                   // the row's mu / V are read before its record overwrites them
        const float inv_M = 1.0f / (float)p.M;
        const float ratio = expf(logp - lpo);
        const float s1 = ratio * adv;
        const float s2 = fminf(fmaxf(ratio, 1.f - p.clip), 1.f + p.clip) * adv;
        const float g_logp = -(s1 <= s2 ? adv : 0.f) * inv_M * ratio;
        const float dv = v - vo;
        const float vclip = vo + fminf(fmaxf(dv, -p.clip), p.clip);
        const float uu = (v - R) * (v - R), w = (vclip - R) * (vclip - R);
        float g_v = p.value_coef * inv_M * (uu >= w ? 2.f * (v - R) : ((dv > -p.clip && dv < p.clip) ? 2.f * (vclip - R) : 0.f));
        if (!live) g_v = 0.f;
        float* rc = recs + r * RP;
        if (qq == 0) {
            rc[0] = live ? fminf(s1, s2) : 0.f;
            rc[1] = live ? fmaxf(uu, w) : 0.f;
            rc[2] = live ? kl : 0.f;
            rc[3] = (live && fabsf(ratio - 1.f) > p.clip) ? 1.f : 0.f;
        }
        // G columns c = qq + TPR u: 0..11 d loss / d mu, 12 d loss / d V (the critic's weight
        // gradient comes out of the same transposed product as row 12 of G^T H_c; Wa has no row 12,
        // so the actor backward is unaffected), 13..15 zero
#pragma unroll
        for (int u = 0; u < 16 / TPR; ++u) {
            const int c = qq + TPR * u;
            float g = 0.f;
            if (u < DPT) {
                const bool on = live && c < A;
                const float iv = on ? cst[16 + c] : 0.f;
                g = on ? g_logp * diff[u] * iv : 0.f;
                rc[4 + c] = on ? g_logp * (diff[u] * diff[u] * iv - 1.f) : 0.f;
                g_s[r * FP + c] = g;
            }
            if (c == 12) {
                g = g_v;
                g_s[r * FP + 12] = g_v;
            }
            __nv_bfloat16 hi, lo;
            split_bf16(g, hi, lo);
            sb[S::G_HI + r * GP + c] = hi;
            sb[S::G_LO + r * GP + c] = lo;
        }
    }
    __syncthreads();

    // ---- head weight gradients: dWa = G^T H_a (MMA), dWc = g_v^T H_c, head bias gradients
    const HeadPart hp = head_part(A, H);
    const int PF = hp.PF, O_WA = hp.WA, O_BA = hp.BA, O_LS = hp.LS, O_WC = hp.WC, O_BC = hp.BC, O_DBA = hp.DBA,
              O_DBC = hp.DBC, O_ST = hp.ST;
    float* out = p.part + (size_t)blockIdx.x * PF;
    {
        // warp w: output columns [H/NW * w, H/NW * (w + 1)), two n-tiles of 8 per step
        static_assert((H / NW) % 16 == 0, "whole n-tile pairs per warp");
#pragma unroll
        for (int np = 0; np < H / NW / 16; ++np) {
            const int n0 = (H / NW) * warp + 16 * np;
            float acc[2][4] = {}, accc[2][4] = {};
#pragma unroll
            for (int ks = 0; ks < ROWS / 16; ++ks) {
                const int k0 = 16 * ks;                       // rows
                // A = G^T [j][row]: 8 x 8 blocks of G [row][j] loaded transposed; matrices
                // (j 0-7, rows 0-7), (j 8-15, rows 0-7), (j 0-7, rows 8-15), (j 8-15, rows 8-15)
                const int ar = k0 + (lane & 7) + 8 * (lane >> 4), aj = 8 * ((lane >> 3) & 1);
                uint32_t ah[4], al[4];
                ldsm_x4_t(sb + S::G_HI + ar * GP + aj, ah[0], ah[1], ah[2], ah[3]);
                ldsm_x4_t(sb + S::G_LO + ar * GP + aj, al[0], al[1], al[2], al[3]);
                // B = H_a [row][col], transposed 8 x 8 loads: (rows 0-7, cols 0-7), (rows 8-15,
                // cols 0-7), (rows 0-7, cols 8-15), (rows 8-15, cols 8-15)
                const int br = k0 + (lane & 7) + 8 * ((lane >> 3) & 1), bc = n0 + 8 * (lane >> 4);
                uint32_t b[4];
                ldsm_x4_t(ha + br * HP + bc, b[0], b[1], b[2], b[3]);
                mma16816(acc[0], ah, b[0], b[1]);
                mma16816(acc[0], al, b[0], b[1]);
                mma16816(acc[1], ah, b[2], b[3]);
                mma16816(acc[1], al, b[2], b[3]);
                // the same G^T against H_c: row 12 is the critic head's weight gradient
                ldsm_x4_t(hc + br * HP + bc, b[0], b[1], b[2], b[3]);
                mma16816(accc[0], ah, b[0], b[1]);
                mma16816(accc[0], al, b[0], b[1]);
                mma16816(accc[1], ah, b[2], b[3]);
                mma16816(accc[1], al, b[2], b[3]);
            }
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int j = gq + 8 * h2;
                    const int col = n0 + 8 * nt + 2 * tq;
                    if (j < A) {
                        out[O_WA + j * H + col] = acc[nt][2 * h2];
                        out[O_WA + j * H + col + 1] = acc[nt][2 * h2 + 1];
                    }
                    if (j == 12) {
                        out[O_WC + col] = accc[nt][2 * h2];
                        out[O_WC + col + 1] = accc[nt][2 * h2 + 1];
                    }
                }
        }
    }
    __syncthreads();

    // ---- backward into the last hidden layer, in place: dY_a = (G Wa) * ELU'(H_a); warp w: rows
    // 16 (w % 4) .. + 15, with eight warps one half of the columns each
    {
        const int r0 = 16 * (warp & 3);
        constexpr int NPW = NW == 8 ? H / 32 : H / 16;          // 16-column tiles per warp
        const int np0 = NW == 8 ? (warp >> 2) * NPW : 0;
        uint32_t gh[4], gl[4];
        ldsm_x4(sb + S::G_HI + (r0 + (lane & 15)) * GP + 8 * (lane >> 4), gh[0], gh[1], gh[2], gh[3]);
        ldsm_x4(sb + S::G_LO + (r0 + (lane & 15)) * GP + 8 * (lane >> 4), gl[0], gl[1], gl[2], gl[3]);
#pragma unroll 2
        for (int np = np0; np < np0 + NPW; ++np) {
            const int n0 = 16 * np;
            // B = Wa [j][col]: column-major fragments over j, i.e. rows of Wa^T [col][j]
            const int bn = n0 + (lane & 7) + 8 * (lane >> 4), bk = 8 * ((lane >> 3) & 1);
            uint32_t wh[4], wl[4];
            ldsm_x4(sb + S::WAT_HI + bn * GP + bk, wh[0], wh[1], wh[2], wh[3]);
            ldsm_x4(sb + S::WAT_LO + bn * GP + bk, wl[0], wl[1], wl[2], wl[3]);
            float acc[2][4] = {};
            mma16816(acc[0], gh, wh[0], wh[1]);
            mma16816(acc[0], gh, wl[0], wl[1]);
            mma16816(acc[0], gl, wh[0], wh[1]);
            mma16816(acc[1], gh, wh[2], wh[3]);
            mma16816(acc[1], gh, wl[2], wl[3]);
            mma16816(acc[1], gl, wh[2], wh[3]);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int r = r0 + gq + 8 * h2;
                    const int col = n0 + 8 * nt + 2 * tq;
                    __nv_bfloat162* e = reinterpret_cast<__nv_bfloat162*>(ha + r * HP + col);
                    const float2 hv = __bfloat1622float2(*e);
                    *e = __floats2bfloat162_rn(acc[nt][2 * h2] * elu_grad_y(hv.x), acc[nt][2 * h2 + 1] * elu_grad_y(hv.y));
                }
        }
    }
    // critic: dY_c = g_v Wc * ELU'(H_c), eight columns (one 16-byte vector) per thread step
    static_assert((HP * 2) % 16 == 0 && (S::WCF % 4) == 0, "16-byte rows and weights");
#pragma unroll 2
    for (int e8 = tid; e8 < ROWS * H / 8; e8 += THREADS) {
        const int r = e8 / (H / 8), k = (e8 % (H / 8)) * 8;
        const float gv = g_s[r * FP + 12];
        uint4* e = reinterpret_cast<uint4*>(hc + r * HP + k);
        const uint4 hv = *e;
        const float4 w0 = *reinterpret_cast<const float4*>(wcf + k), w1 = *reinterpret_cast<const float4*>(wcf + k + 4);
        const float wk[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
        const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
        uint32_t o[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float y0 = __uint_as_float(hw[i] << 16), y1 = __uint_as_float(hw[i] & 0xFFFF0000u);
            const __nv_bfloat162 d = __floats2bfloat162_rn(gv * wk[2 * i] * elu_grad_y(y0), gv * wk[2 * i + 1] * elu_grad_y(y1));
            o[i] = *reinterpret_cast<const uint32_t*>(&d);
        }
        *e = make_uint4(o[0], o[1], o[2], o[3]);
    }
    __syncthreads();

    // ---- hidden bias gradients: column sums of the bf16 dY rows as ones^T dY on the MMA (rows
    // past M are zero); warp w: columns [H/NW w, H/NW (w + 1)) of both networks
    {
        const uint32_t one2 = 0x3F803F80u;                  // two bf16 ones
        const uint32_t ones[4] = {one2, one2, one2, one2};
#pragma unroll
        for (int np = 0; np < H / NW / 16; ++np) {
            const int n0 = (H / NW) * warp + 16 * np;
            float sa[2][4] = {}, sc[2][4] = {};
#pragma unroll
            for (int ks = 0; ks < ROWS / 16; ++ks) {
                const int br = 16 * ks + (lane & 7) + 8 * ((lane >> 3) & 1), bc = n0 + 8 * (lane >> 4);
                uint32_t b[4];
                ldsm_x4_t(ha + br * HP + bc, b[0], b[1], b[2], b[3]);
                mma16816(sa[0], ones, b[0], b[1]);
                mma16816(sa[1], ones, b[2], b[3]);
                ldsm_x4_t(hc + br * HP + bc, b[0], b[1], b[2], b[3]);
                mma16816(sc[0], ones, b[0], b[1]);
                mma16816(sc[1], ones, b[2], b[3]);
            }
            if (gq == 0) {                                   // row 0 of the (identical) rows
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    const int col = n0 + 8 * nt + 2 * tq;
                    out[O_DBA + col] = sa[nt][0];
                    out[O_DBA + col + 1] = sa[nt][1];
                    out[O_DBC + col] = sc[nt][0];
                    out[O_DBC + col + 1] = sc[nt][1];
                }
            }
        }
    }
    // the block's statistics: record columns 0..3 loss terms, 4 g_v, 5..16 g_mu, 17..28 g_log_std
    for (int i = tid; i < 29; i += THREADS) {
        {
            const int c = i;
            const float* col = c < 4 ? recs + c : c == 4 ? g_s + 12 : c < 17 ? g_s + (c - 5) : recs + 4 + (c - 17);
            const int pitch = (c >= 4 && c < 17) ? FP : RP;
            float sum = 0.f;
            for (int r = 0; r < ROWS; ++r) sum += col[r * pitch];
            if (c < 4) out[O_ST + c] = sum;
            else if (c == 4) out[O_BC] = sum;
            else if (c < 17) { if (c - 5 < A) out[O_BA + c - 5] = sum; }
            else if (c - 17 < A) out[O_LS + c - 17] = sum - (blockIdx.x == 0 ? p.entropy_coef : 0.f);
        }
    }
    if (tid >= 4 && tid < 8) out[O_ST + tid] = 0.f;
    // ---- gradient rows out (16-byte vectors)
    {
        constexpr int VPR = H / 8;
        uint4* da = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(p.dya) + (size_t)m0 * H);
        uint4* dc = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(p.dyc) + (size_t)m0 * H);
        for (int v = tid; v < rows * VPR; v += THREADS) {
            const int r = v / VPR, c = (v % VPR) * 8;
            da[(size_t)r * VPR + c / 8] = *reinterpret_cast<const uint4*>(ha + r * HP + c);
            dc[(size_t)r * VPR + c / 8] = *reinterpret_cast<const uint4*>(hc + r * HP + c);
        }
    }

    // the minibatch statistics and Algorithm 1 follow in loss_stats_kernel
}

template <int H>
cudaError_t mma_dispatch(const HeadParams& p, cudaStream_t s) {
    cudaError_t e = launch_pdl(loss_mma_kernel<H>, dim3(p.nblocks), dim3(32 * warps_of<H>()), Smem<H>::BYTES, s, p);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace

int loss_mma_rows() { return ROWS; }

// Dynamic shared-memory limits, and the whole of the SM's unified L1 / shared memory offered as
// shared memory, so that three 74 KB blocks of the 128-wide form are resident per SM (one wave
// for a 24576-row minibatch instead of two).
template <int H>
cudaError_t mma_attrs() {
    cudaError_t e = cudaFuncSetAttribute(loss_mma_kernel<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<H>::BYTES);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(loss_mma_kernel<H>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}

cudaError_t loss_mma_prepare() {
    cudaError_t e = mma_attrs<64>();
    if (e == cudaSuccess) e = mma_attrs<128>();
    if (e == cudaSuccess) e = mma_attrs<256>();
    return e;
}

cudaError_t launch_loss_mma(const HeadParams& p, cudaStream_t s) {
    // 16-byte copies of the head weights and of the h rows
    if ((reinterpret_cast<uintptr_t>(p.Wa) | reinterpret_cast<uintptr_t>(p.Wc) | reinterpret_cast<uintptr_t>(p.ha) |
         reinterpret_cast<uintptr_t>(p.hc)) & 15u)
        return cudaErrorMisalignedAddress;
    if ((p.A * p.H) % 4) return cudaErrorInvalidValue;
    if (p.H == 64) return mma_dispatch<64>(p, s);
    if (p.H == 128) return mma_dispatch<128>(p, s);
    if (p.H == 256) return mma_dispatch<256>(p, s);
    return cudaErrorInvalidValue;
}

}  // namespace rl
