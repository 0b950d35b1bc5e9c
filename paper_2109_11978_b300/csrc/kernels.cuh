// Internal kernel interfaces of the library (parameter blocks and launchers).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rl {

// ------------------------------------------------------------------ GAE
cudaError_t launch_gae(int T, int N, float gamma, float lam, const float* rew, const float* val,
                       const float* last_val, const uint8_t* done, float* adv, float* ret,
                       int normalize, float* adv_stats, float* partials, int nparts, cudaStream_t s);
// partials: device scratch of gae_workspace_bytes (one 16-byte slot per 256 robots and a
// (mean, std) slot); nparts = gae_num_partials(T, N)
int gae_num_partials(int T, int N);
size_t gae_workspace_bytes(int T, int N);
int gae_noalloc_max_envs();
cudaError_t gae_noalloc_scratch(cudaStream_t s, void** out);

// ------------------------------------------------------------------ SIMT FP32 GEMM
// C[m][n] = sum_k A(m,k) B(n,k);  A(m,k) = a_t ? A[k*lda+m] : A[m*lda+k];
// B(n,k) = b_t ? B[k*ldb+n] : B[n*ldb+k].  Batched over blockIdx.z = batch * splits + split;
// split s covers k in [s*kchunk, min(K, (s+1)*kchunk)).
enum { EPI_STORE = 0, EPI_BIAS_ELU = 1, EPI_ELU_GRAD = 2 };
struct GemmBatch {
    const float* A[2];
    const float* B[2];
    float* C[2];
    const float* bias[2];    // EPI_BIAS_ELU
    const float* H[2];       // EPI_ELU_GRAD: activation whose ELU derivative scales the result
    float* colsum[2];        // EPI_ELU_GRAD: per-row-tile column sums [gridDim.x][N] (or null)
    long long split_stride;  // EPI_STORE with splits: C + split * split_stride
};
cudaError_t launch_gemm_f32(int epi, bool a_t, bool b_t, int M, int N, int K, int lda, int ldb, int ldc,
                            int ldh, int batch, int splits, int kchunk, const GemmBatch& g, cudaStream_t s);
constexpr int SIMT_BM = 128;

// ------------------------------------------------------------------ heads, loss, Adam
struct HeadParams {
    int M, H, A;                 // rows, last hidden width, action dims
    int bf16;                    // activations / gradients in bf16 (else fp32)
    const void* ha;              // actor last hidden [M][H]
    const void* hc;              // critic last hidden [M][H]
    const float* Wa;             // actor head [A][H]
    const float* ba;             // [A]
    const float* log_std;        // [A]
    const float* Wc;             // critic head [1][H]
    const float* bc;             // [1]
    // act mode
    uint64_t seed;
    const unsigned long long* iteration;
    int t;
    float* actions;
    float* mu;
    float* logp;
    float* values;
    // loss mode
    const int* idx;              // minibatch row -> sample index (null = identity)
    const float* rec;            // packed per-sample loss inputs (launch_pack_records layout, indexed like
                                 // the fields below), or null
    int rec_ld;
    const float* a_old;          // [B][A]
    const float* logp_old;       // [B]
    const float* mu_old;         // [B][A]
    const float* log_std_old;    // [A]
    const float* v_old;          // [B]
    const float* adv;            // [B] (normalised)
    const float* ret;            // [B]
    float clip, value_coef, entropy_coef;
    void* dya;                   // actor d loss / d h_L, row-major [M][H] (fp32 or bf16)
    void* dyc;                   // critic
    float* part;                 // per-block partials, layout HEAD_PART_* below
    int nblocks;
    float* scal;                 // device scalars (alpha, KL, ...)
    float* stats;                // [RL_NSTATS] accumulators (optional)
    float kl_target, lr_min, lr_max;
    float* trace;                // optional: [2] = this minibatch's KL and alpha after Algorithm 1
};
// Per-block partial layout of the loss head (floats): Wa grad [A*H], ba [A], log_std [A], Wc grad
// [H], bc [1], db_a [H], db_c [H], stats [8]; every field starts on a 16-byte boundary so Adam
// reads the partials as float4 (A * H and H are multiples of 4).
struct HeadPart {
    int WA, BA, LS, WC, BC, DBA, DBC, ST, PF;
};
__host__ __device__ inline int pad4(int n) { return (n + 3) & ~3; }
__host__ __device__ inline HeadPart head_part(int A, int H) {
    HeadPart o;
    o.WA = 0;
    o.BA = pad4(A * H);
    o.LS = o.BA + pad4(A);
    o.WC = o.LS + pad4(A);
    o.BC = o.WC + pad4(H);
    o.DBA = o.BC + 4;
    o.DBC = o.DBA + pad4(H);
    o.ST = o.DBC + pad4(H);
    o.PF = o.ST + 8;
    return o;
}
__host__ __device__ inline int head_part_floats(int A, int H) { return head_part(A, H).PF; }
// ------------------------------------------------------------------ env step
struct EnvParams {
    int N, O, Op, GX, GY, decimation, max_ep, L, C, cpt, nx, ny;
    int push_interval, noise_on, push_on, randomize_eplen, t;
    float kp, kd, ascale, dt, sim_dt, gamma, push_vel, grid_sp, inv_res, tile;
    float cmd_range[3];
    float q_def[12];
    uint32_t crash_thr;
    uint64_t seed;
    const float* hf;
    float* sf;
    int* si;
    const unsigned long long* iteration;
    const float* actions;
    const float* values;
    void* obs;
    int obs_bf16;
    float* rew;
    uint8_t* done;
    uint8_t* timeout;
    int* level_out;
    int* tidx_out;
    float* stats;   // optional: [0] += sum reward, [1] += resets, [2] += sum level
    // fused policy head (act.ha non-null): the step first evaluates the action head on the
    // rollout's last hidden rows (act.M = N), writes act.actions / mu / logp / values and steps
    // with those actions and values instead of reading actions / values
    HeadParams act;
};
cudaError_t launch_env_step(const EnvParams& p, int mode, cudaStream_t s);
cudaError_t env_prepare();


cudaError_t launch_act_head(const HeadParams& p, cudaStream_t s);
cudaError_t launch_loss_head(const HeadParams& p, cudaStream_t s);
// The minibatch statistics of a loss-head launch (its partials), Algorithm 1 and Adam's step size
// and bias corrections (loss_stats.cu); one block, run after the loss head.
cudaError_t launch_loss_stats(const HeadParams& p, cudaStream_t s);
int loss_head_blocks(int M, int H, int bf16);   // blocks (= partial slots) of one loss-head launch
// BF16 loss head on warp-level tensor-core MMAs (loss_mma.cu)
int loss_mma_rows();
cudaError_t loss_mma_prepare();
cudaError_t launch_loss_mma(const HeadParams& p, cudaStream_t s);
void heads_prepare();

// Device scalar block (floats): alpha, kl, adam step (as float bits of int), ...
enum { SC_ALPHA = 0, SC_KL = 1, SC_STEP = 2, SC_LOSS = 3, SC_SURR = 4, SC_VLOSS = 5, SC_ENT = 6,
       SC_CLIPFRAC = 7, SC_ADV_MEAN = 8, SC_ADV_STD = 9, SC_STEPSIZE = 10, SC_INVSQRT_BC2 = 11, SC_NSCAL = 16 };

struct AdamSeg {
    long long offset;      // into the flat internal parameter vector
    long long size;
    const float* partials; // partial q of element i at partials[q * stride + i]
    long long stride;
    int nsplit;
    int block_start;       // first block of this segment
    int vec;               // 1: offset, size, stride multiples of 4 and partials 16-byte aligned
};
constexpr int MAX_SEGS = 40;
struct AdamParams {
    float* p;
    float* m;
    float* v;
    float* scal;           // SC_ALPHA, SC_STEP
    int nsegs;
    int nblocks;
    AdamSeg seg[MAX_SEGS];
    // bf16 weight copies (optional): for segment s, wbf[s] has the segment's layout
    void* wbf[MAX_SEGS];
    float* grad_out;       // optional: reduced gradient (flat internal) instead of a step
    // without a device scalar block (scal null): the step size alpha / (1 - 0.9^t) and
    // 1 / sqrt(1 - 0.999^t) given by the host
    float step_size_host, inv_sqrt_bc2_host;
};
constexpr int ADAM_THREADS = 256;
constexpr int ADAM_WIDE = 64;      // segments with more partials than this: a warp per parameter group
// parameters per block: one (scalar) or four (vec) per thread, or per warp for wide segments
__host__ __device__ inline long long adam_per_block(int nsplit, int vec) {
    return (long long)(nsplit > ADAM_WIDE ? ADAM_THREADS / 32 : ADAM_THREADS) * (vec ? 4 : 1);
}
cudaError_t launch_adam(const AdamParams& p, cudaStream_t s);
// One warp waiting (bounded) on an mbarrier nothing arrives on: records RL_ERR_TIMEOUT in *status.
cudaError_t launch_forced_timeout(int* status, cudaStream_t s);

// Minibatch gather: rows idx[i] of obs [B][Op] -> X [M][Op].
// Batched LSTM actuator cell (actuator.cu): n joints, inputs [n][2], state h, c [n][32] updated in
// place, torques [n]; weights as rl_actuator_lstm_step documents.
constexpr int ACT_INPUTS = 2, ACT_HIDDEN = 32;
cudaError_t launch_actuator_lstm(int n, const float* w, const float* x, float* h, float* c, float* tau, cudaStream_t s);

// Procedural terrain family (terrain.cu): grid of levels (rows) x terrain kinds (columns) of c x c
// cells; P, W, B: the spawn platform's half width, the stair width and the obstacle block in cells.
struct TerrainParams {
    int levels, cols, c, P, W, B;
    float res;
    uint64_t seed;
};
cudaError_t launch_terrain(const TerrainParams& p, float* hf, cudaStream_t s);

cudaError_t launch_gather(const void* obs, int bf16, const int* idx, int M, int Op, void* X, cudaStream_t s);
// Per-sample loss inputs packed once per iteration into one 128-byte record per sample:
// [a_old A][mu_old A][logp_old][adv][v_old][ret][zeros], REC_LD floats per record (A <= 12).
constexpr int REC_LD = 32;
cudaError_t launch_pack_records(int B, int A, const float* a_old, const float* mu_old, const float* logp_old,
                                const float* adv, const float* v_old, const float* ret, float* rec, cudaStream_t s);
// Minibatch indices: permutation of [0, B) by a cycle-walking Feistel network keyed by
// (seed, iteration, epoch); idx [epochs][B]; a walk that runs out of its bound records
// RL_ERR_STATE in *status.
cudaError_t launch_permutation(int B, int epochs, uint64_t seed, const unsigned long long* iteration,
                               int* idx, int* status, cudaStream_t s);
cudaError_t launch_small(int op, float* scal, unsigned long long* iteration, const float* stats_src,
                         float* stats_dst, float nsamp, cudaStream_t s);
// Statistics accumulator layout (floats): [0] loss, [1] surrogate, [2] value loss, [3] entropy,
// [4] KL, [6] clip fraction (sums over minibatches), [12] minibatch count, [13] reward sum,
// [14] resets, [15] level sum (env step).
constexpr int ACC_ENV = 13;
enum { SMALL_ITER_INC = 0, SMALL_ZERO_STATS = 1, SMALL_FINAL_STATS = 2 };

// Convert fp32 [rows][cols] -> bf16 (row-major copy and transposed copy).
cudaError_t launch_to_bf16(const float* src, int rows, int cols, void* dst, cudaStream_t s);

// ------------------------------------------------------------------ tcgen05 BF16 GEMM
struct TcGemm;   // defined in gemm_tc.cu
}  // namespace rl
