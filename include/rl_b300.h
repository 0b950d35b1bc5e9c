/*
 * rl_b300.h -- C ABI of the B300 (sm_103a) hot path of massively parallel PPO for legged
 * locomotion (Rudin, Hoeller, Reist, Hutter, "Learning to Walk in Minutes Using Massively
 * Parallel Deep Reinforcement Learning", CoRL 2021).
 *
 * One training iteration (Sec. 2, Sec. 2.2) is: n_steps times { batched actor/critic
 * inference (rl_policy_act) -> env-side tensor math for every robot (rl_env_step) }, then the
 * critic's value of the last observation, GAE (rl_gae), and epochs x minibatches of the
 * clipped-surrogate PPO update with the adaptive learning rate of Algorithm 1 and Adam
 * (rl_ppo_update).  rl_train_iteration runs all of it on buffers the context owns, optionally
 * as one CUDA graph.
 *
 * Conventions (all entry points):
 *   - Status codes only; no exception crosses the ABI.  Arguments are validated on the host
 *     before anything is launched; an invalid argument returns RL_ERR_INVALID_ARG (or
 *     RL_ERR_ALIGNMENT) and launches nothing.
 *   - Unless stated otherwise a pointer argument is a CUDA device pointer owned by the caller
 *     and valid for the duration of the asynchronous work on `stream`.  Host pointers are
 *     marked "host".  The library keeps no pointer to caller memory after a call returns.
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t passed as void*; NULL = the
 *     legacy default stream).  No entry point other than rl_create / rl_destroy /
 *     rl_get_scalars / rl_train_iteration (when it copies stats to the host) synchronises.
 *   - Device-side failures that are not CUDA errors (a bounded wait that ran out, an index
 *     outside its buffer) are recorded in a device status word, read by
 *     rl_last_device_status.
 *   - Floating point: FP32 everywhere except the MLP GEMM operands in RL_BF16 precision
 *     (bfloat16 operands, FP32 accumulation).
 *   - Layouts: "[T][N]" means row-major, N contiguous; step t of a rollout is row t.
 */
#ifndef RL_B300_H
#define RL_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rl_ctx rl_ctx;
typedef int32_t rl_status;

#define RL_OK 0
#define RL_ERR_INVALID_ARG (-1)
#define RL_ERR_ALIGNMENT (-2)
#define RL_ERR_CUDA (-3)
#define RL_ERR_TIMEOUT (-4)
#define RL_ERR_STATE (-5)
#define RL_ERR_OOM (-6)
#define RL_ERR_UNSUPPORTED (-7)

#define RL_FP32 0
#define RL_BF16 1

/* Env state layout (structure of arrays).  float state: [RL_NF][num_envs]; int state:
 * [RL_NI][num_envs].  Rows: position relative to the spawn origin (x, y), base height z,
 * heading (cos, sin), base-frame linear velocity (3), angular velocity (3), projected gravity
 * (3), command (v*_x, v*_y, w*_z), feet air time (4), joint positions (12), joint velocities
 * (12), previous actions (12); int rows: episode length, curriculum level, foot-contact bits. */
#define RL_NF 57
#define RL_NI 3
#define RL_F_PX 0
#define RL_F_PY 1
#define RL_F_Z 2
#define RL_F_HC 3
#define RL_F_HS 4
#define RL_F_VX 5
#define RL_F_WX 8
#define RL_F_GX 11
#define RL_F_CMDX 14
#define RL_F_TAIR 17
#define RL_F_Q 21
#define RL_F_QD 33
#define RL_F_AP 45
#define RL_I_EPLEN 0
#define RL_I_LEVEL 1
#define RL_I_CONTACT 2

/* Number of floats of the device statistics vector written by rl_ppo_update / rl_train_iteration:
 * [0] mean loss, [1] mean surrogate loss, [2] mean value loss, [3] entropy, [4] mean KL,
 * [5] final learning rate alpha, [6] clip fraction, [7] mean reward of the rollout (train only),
 * [8] mean advantage before normalisation, [9] its standard deviation, [10] number of resets,
 * [11] mean curriculum level, [12..15] reserved. */
#define RL_NSTATS 16

/* Configuration.  Defaults (rl_config_default) follow Table 3 (PPO), Algorithm 1, Table 2,
 * Table 4, Sec. 3.1 (8 m tiles), App. A.1.1 (50 Hz policy, 4 x 0.005 s substeps) and the
 * rough-terrain workload (4096 robots x 24 steps, 235 observations, 512-256-128 ELU MLPs). */
typedef struct rl_config {
    int32_t num_envs;        /* robots N (Sec. 2.2.1) */
    int32_t num_steps;       /* steps per robot and iteration T (Sec. 2.2.1) */
    int32_t obs_dim;         /* 48 proprioceptive + grid_x * grid_y heights (Sec. 3.2) */
    int32_t obs_pad;         /* row stride of observation buffers; multiple of 64, >= obs_dim */
    int32_t act_dim;         /* 12 joint targets */
    int32_t num_hidden;      /* hidden layers (1..4) */
    int32_t hidden[4];       /* widths, each a multiple of 64, <= 1024 */
    float gamma, lam, clip, entropy_coef, value_coef, kl_target, lr_init, lr_min, lr_max;
    int32_t epochs, minibatches;
    int32_t precision;       /* RL_FP32 or RL_BF16 (MLP GEMM operands) */
    float kp, kd, action_scale, dt, sim_dt;
    int32_t decimation, max_episode_len;
    int32_t num_levels, num_cols;
    float tile_size, hf_res;
    int32_t grid_x, grid_y;
    float grid_spacing;
    int32_t noise_on, push_on, push_interval;
    float push_vel;
    float cmd_range[3];
    uint32_t crash_threshold; /* stand-in physics: crash when a 32-bit draw is below this */
    float q_def[12];          /* default joint positions */
    int32_t reserved[2];      /* zero; keeps seed 8-byte aligned without implicit padding */
    uint64_t seed;
} rl_config;

/* Fills *cfg with the defaults listed above.  Never fails. */
void rl_config_default(rl_config* cfg);

/* Number of parameters of the flat layout (actor then critic, see rl_get_params). */
int64_t rl_param_count(const rl_config* cfg);

/* Human-readable name of a status code (static string). */
const char* rl_status_string(rl_status s);

/* Creates a learner.  heightfield: host, fp32 [num_levels * c][num_cols * c] with
 * c = tile_size / hf_res (x rows, y columns; Sec. 2.1 tiles all terrain levels and types in
 * one mesh), may be NULL when grid_x * grid_y == 0.  init_params: host, flat fp32 parameters
 * (layout of rl_get_params), required.  Allocates every buffer it will ever use (weights,
 * Adam moments, rollout storage, workspaces); no later call allocates.  The env state is
 * initialised as rl_env_reset_all describes.  Returns RL_ERR_INVALID_ARG for an inconsistent
 * config, RL_ERR_OOM if device memory runs out, RL_ERR_CUDA on any other CUDA error. */
rl_status rl_create(const rl_config* cfg, const float* heightfield, const float* init_params,
                    rl_ctx** out);

/* Frees everything the context owns.  Synchronises the device.  NULL is a no-op. */
void rl_destroy(rl_ctx* ctx);

/* Flat parameters (fp32), actor [W1, b1, ..., W_head, b_head, log_std] then critic
 * [W1, b1, ..., W_head, b_head], W_l row-major [fan_out][fan_in], first fan_in = obs_dim. */
rl_status rl_get_params(rl_ctx* ctx, float* params_out, void* stream);
rl_status rl_set_params(rl_ctx* ctx, const float* params, void* stream);

/* Adam's first and second moments (Adam with bias correction; the paper only names the
 * optimiser's learning rate, Algorithm 1) in the flat layout of rl_get_params: m_out, v_out device
 * fp32, rl_param_count values each, written on stream. */
rl_status rl_get_adam_moments(rl_ctx* ctx, float* m_out, float* v_out, void* stream);

/* Host-visible learner scalars (synchronises): out[0] = alpha, out[1] = iteration counter,
 * out[2] = Adam step count, out[3] = last minibatch KL. */
rl_status rl_get_scalars(rl_ctx* ctx, double out[4]);
/* Sets alpha, the iteration counter and the Adam step count (enqueued on stream). */
rl_status rl_set_scalars(rl_ctx* ctx, double alpha, int64_t iteration, int64_t adam_step, void* stream);

/* Batched LSTM actuator network (Sec. 3.3): one cell step for n joints, run once per simulation
 * substep.  The paper feeds only the current measurements to an LSTM that outputs the joint
 * torque; read here as inputs x = (q* - q, qd) [n][RL_ACT_INPUTS], one layer of RL_ACT_HIDDEN
 * units, the standard cell with a forget gate (gate order input, forget, cell, output):
 *   a = W_ih x + W_hh h + b;  c' = sigmoid(a_f) c + sigmoid(a_i) tanh(a_g);
 *   h' = sigmoid(a_o) tanh(c');  tau = w_out . h' + b_out.
 * weights: device fp32 [W_ih (4H x 2) | W_hh (4H x H) | b (4H) | w_out (H) | b_out], row-major,
 * RL_ACT_WEIGHTS values (trained weights are not part of this library; any values run).
 * h, c: device fp32 [n][RL_ACT_HIDDEN], updated in place; tau: device fp32 [n].  All device
 * pointers 4-byte aligned (RL_ERR_ALIGNMENT); enqueued on stream; n = 0 is a no-op. */
#define RL_ACT_INPUTS 2
#define RL_ACT_HIDDEN 32
#define RL_ACT_WEIGHTS (4 * RL_ACT_HIDDEN * RL_ACT_INPUTS + 4 * RL_ACT_HIDDEN * RL_ACT_HIDDEN + 4 * RL_ACT_HIDDEN + RL_ACT_HIDDEN + 1)
rl_status rl_actuator_lstm_step(int32_t n, const float* weights, const float* x, float* h, float* c, float* tau,
                                void* stream);

/* Procedural terrain family of Sec. 3.1 (Fig. 2) as the heightfield rl_create takes: tile rows
 * are curriculum levels (difficulty d = level / (num_levels - 1)), tile column k is terrain kind
 * k % 7: flat, slope pyramid, slope pit, randomly rough, discrete obstacles, stairs pyramid,
 * stairs pit.  Slopes rise at 25 deg x d, stair and obstacle steps are 0.05 + 0.15 d m, stairs
 * 0.3 m wide, rough terrain varies by 0.1 m, obstacles stand on 1 m blocks; every tile keeps a
 * flat 2 m x 2 m platform at its centre.  hf: device, fp32 [num_levels c][num_cols c] with
 * c = tile_size / hf_res, written on stream.  Random heights come from the seed's counter-based
 * generator, so equal configs give equal fields.  RL_ERR_INVALID_ARG unless the tile, 1 m and
 * 0.3 m are whole numbers of cells (c even, a multiple of the 1 m block). */
rl_status rl_terrain_generate(const rl_config* cfg, float* hf, void* stream);

/* Checkpoint and resume of the whole learner (the paper has no counterpart; training of
 * Sec. 2.2 / Algorithm 1 carries alpha and the Adam moments from iteration to iteration).  The
 * image holds a header (magic "RLB300CK", version 1, the config, the segment sizes and the GEMM
 * tile shapes of every site) followed by the parameters, Adam m and v, the device scalar block
 * (alpha, Adam step, ...), the iteration counter, the env state (fp32 and int32 parts), the
 * curriculum levels and the first observation of the next rollout.  Everything else is derived
 * from these (bf16 weight copies) or drawn afresh from the seed and the iteration counter
 * (shuffles, noise, actions), so a run resumed from an image continues bit for bit as the saved
 * run would have.
 * rl_checkpoint_bytes: size of the image in bytes (-1 for a NULL context).
 * rl_checkpoint_save: writes the image to host memory dst (bytes >= rl_checkpoint_bytes); copies
 *   on stream and synchronises it before returning.
 * rl_checkpoint_load: restores an image into a context created with the same config and
 *   heightfield: RL_ERR_INVALID_ARG for a wrong magic, version, config or size (the context is
 *   then unchanged).  Re-applies the saved tile shapes, copies on stream, refreshes the bf16
 *   weights and synchronises the stream before returning (src may be freed afterwards). */
int64_t rl_checkpoint_bytes(rl_ctx* ctx);
rl_status rl_checkpoint_save(rl_ctx* ctx, void* dst, size_t bytes, void* stream);
rl_status rl_checkpoint_load(rl_ctx* ctx, const void* src, size_t bytes, void* stream);

/* Env state access (layout above).  state_f: [RL_NF][num_envs] fp32, state_i: [RL_NI][num_envs],
 * in device or host memory (the copy direction follows from the unified address space; a pinned
 * host buffer keeps the copy asynchronous on stream, a pageable one makes it synchronous).  Both
 * enqueue on stream and return without synchronising it: a host buffer may be read or reused only
 * after the stream has reached the copy.  A caller that keeps the simulator state in host memory
 * between iterations passes it in with rl_env_set_state before rl_train_iteration and takes it back
 * with rl_env_get_state after it. */
rl_status rl_env_get_state(rl_ctx* ctx, float* state_f, int32_t* state_i, void* stream);
rl_status rl_env_set_state(rl_ctx* ctx, const float* state_f, const int32_t* state_i, void* stream);

/* Spawns every robot on level 0 at the centre of its tile with a fresh command and a random
 * episode length (Sec. 3.1), and writes the first observation to obs_out [num_envs][obs_pad]
 * (fp32 for RL_FP32, bf16 for RL_BF16; may be NULL). */
rl_status rl_env_reset_all(rl_ctx* ctx, void* obs_out, void* stream);

/* One 50 Hz policy step of the env-side math for all robots (Sec. 3.2, App. A.1.1, Table 2,
 * Sec. 2.2.2, Sec. 3.1, Sec. 3.3): 4 substeps of PD control (tau = Kp (q* - q) - Kd qd,
 * q* = q_def + action_scale * a) each followed by the seeded physics stand-in, the nine
 * Table 2 reward terms, crash / time-out, reward + gamma V on time-out, curriculum update and
 * respawn of finished robots, then the observation with bilinear height samples and Table 4
 * noise.  t: step index within the iteration (part of the random key).
 *   actions [N][act_dim] fp32; values [N] fp32 = V(o_t) stored at act time;
 *   obs_out [N][obs_pad] (fp32 or bf16 by precision; padding columns written as 0);
 *   rew_out [N] fp32; done_out, timeout_out [N] uint8; level_out, terrain_idx_out [N] int32
 *   (any output may be NULL except obs_out and rew_out). */
rl_status rl_env_step(rl_ctx* ctx, int32_t t, const float* actions, const float* values,
                      void* obs_out, float* rew_out, uint8_t* done_out, uint8_t* timeout_out,
                      int32_t* level_out, int32_t* terrain_idx_out, void* stream);

/* Batched policy inference (Sec. 2): mu = actor(obs), V = critic(obs) (ELU hidden layers,
 * linear heads), a = mu + exp(log_std) * eps with eps ~ N(0, 1) drawn from the counter-based
 * generator keyed by (seed, iteration, t, env), log pi(a) of the diagonal Gaussian.
 *   obs [n][obs_pad] (fp32 or bf16 by precision), n <= num_envs;
 *   actions, mu [n][act_dim] fp32; logp, values [n] fp32.  actions, mu and logp may all be
 *   NULL, which runs the critic only (the last value of a rollout). */
rl_status rl_policy_act(rl_ctx* ctx, int32_t t, int32_t n, const void* obs, float* actions,
                        float* mu, float* logp, float* values, void* stream);

/* Generalized advantage estimation (Sec. 2.2.1, Table 3) over [T][N] samples:
 *   delta_t = r_t + gamma (1 - d_t) V_{t+1} - V_t,  A_t = delta_t + gamma lambda (1 - d_t) A_{t+1},
 *   V_T = last_val, R_t = A_t + V_t.  Stateless.
 * rew, val [T][N] fp32; last_val [N]; done [T][N] uint8; adv_out, ret_out [T][N] fp32.
 * normalize != 0 replaces A by (A - mean) / (std + 1e-8) over all T*N samples (population std;
 * R keeps the unnormalised A).  adv_stats_out (may be NULL): [2] = mean, std of A.
 * workspace: device scratch of rl_gae_workspace_bytes(T, N) bytes (16 bytes per block of 256
 * robots, plus 16), 16-byte aligned (may be NULL when normalize == 0 and adv_stats_out == NULL);
 * nothing in it has to start at zero. */
size_t rl_gae_workspace_bytes(int32_t T, int32_t N);
rl_status rl_gae(int32_t T, int32_t N, float gamma, float lam, const float* rew, const float* val,
                 const float* last_val, const uint8_t* done, float* adv_out, float* ret_out,
                 int32_t normalize, float* adv_stats_out, void* workspace, size_t workspace_bytes,
                 void* stream);

/* rl_gae without any allocation, for callers that cannot allocate device memory: a process
 * whose GPU memory is reserved up front by another framework's allocator or a fixed budget, a
 * plugin that is not allowed to call the CUDA allocator, or a latency-critical loop that must
 * not pay for cudaMalloc and its implicit synchronisation.  The paper has no counterpart; this is
 * a deployment convenience.  Same arguments, results and layouts as rl_gae, minus the workspace:
 * the normalisation partial sums live in a file-scope device array of the library (64 KiB:
 * 4096 slots of 16 bytes, one per block of 256 robots plus one for the mean and standard
 * deviation), held by every GPU that loads the library until the process exits.
 *   - N <= 1048320 (4095 blocks of 256 robots); larger N returns RL_ERR_INVALID_ARG and
 *     launches nothing.  T is unrestricted.
 *   - Each call made outside stream capture looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and remembers it; a call on a capturing
 *     stream uses the remembered address.  So make the first call on a device before any stream
 *     capture (a first call inside a capture returns RL_ERR_CUDA), and after a cudaDeviceReset
 *     make one call outside capture before capturing again.
 *   - Every call on a device shares the one array and leaves its partial sums there.  Each call
 *     overwrites every slot it reads before reading it, so nothing has to start at zero, but
 *     calls that overlap on the GPU (other streams, other host threads) race on the array and
 *     must be serialised by the caller.
 *   - Calls no cudaMalloc, cudaFree or allocating library routine. */
rl_status rl_gae_noalloc(int32_t T, int32_t N, float gamma, float lam, const float* rew, const float* val,
                         const float* last_val, const uint8_t* done, float* adv_out, float* ret_out,
                         int32_t normalize, float* adv_stats_out, void* stream);

/* PPO update (Sec. 2.2, Table 3, Algorithm 1) on B = num_envs * num_steps samples:
 * for each of `epochs` epochs a fresh permutation (keyed by seed, iteration, epoch) splits
 * the batch into `minibatches` minibatches; for each minibatch: forward, clipped surrogate,
 * clipped value loss, entropy bonus, KL(pi_old || pi_new), alpha updated by Algorithm 1,
 * hand-written backward, Adam step with the new alpha.  Increments the iteration counter.
 *   obs [B][obs_pad] (fp32 / bf16 by precision); actions, mu_old [B][act_dim] fp32;
 *   logp_old, val_old, adv (normalised), ret [B] fp32; clip: the clip range c of the surrogate
 *   ratio (clip(ratio, 1 - c, 1 + c), Table 3: 0.2) and of the value loss (V_old +
 *   clip(V - V_old, -c, c)), 0 < c < 1; stats_out: device [RL_NSTATS] or NULL.
 * minibatches must give the config's minibatch size (B / minibatches) and epochs <= the config's
 * epochs (RL_ERR_INVALID_ARG otherwise).  The permutations and, per minibatch, the KL and the
 * alpha Algorithm 1 chose are left in rl_get_storage slots 13 and 14. */
rl_status rl_ppo_update(rl_ctx* ctx, const void* obs, const float* actions, const float* logp_old,
                        const float* mu_old, const float* val_old, const float* adv,
                        const float* ret, int32_t epochs, int32_t minibatches, float clip,
                        float* stats_out, void* stream);

/* Loss and gradient of one minibatch without a parameter step (the hand-written backward of
 * rl_ppo_update, exposed for gradient checks).  Inputs are M contiguous rows (same layouts
 * as rl_ppo_update); log_std_old [act_dim]; grad_out: flat layout of rl_get_params;
 * stats_out [RL_NSTATS] (loss terms, KL).  M <= num_envs * num_steps / minibatches. */
rl_status rl_ppo_loss_grad(rl_ctx* ctx, int32_t M, const void* obs, const float* actions,
                           const float* logp_old, const float* mu_old, const float* log_std_old,
                           const float* val_old, const float* adv, const float* ret,
                           float* grad_out, float* stats_out, void* stream);

/* One full training iteration on context-owned storage (rollout, last value, GAE with
 * normalisation, update).  use_graph != 0 replays a CUDA graph of the whole iteration
 * (captured on first use).  stats_host (host, may be NULL): RL_NSTATS floats copied back,
 * which synchronises stream. */
rl_status rl_train_iteration(rl_ctx* ctx, int32_t use_graph, float* stats_host, void* stream);

/* Several independent learners (own configs, weights, Adam state, learning rate, curriculum and
 * env state; e.g. uneven robot counts) trained together: one rl_group_train_iteration replays
 * one CUDA graph whose parallel branches hold every learner's whole iteration, so the GPU
 * overlaps the learners' kernels.  cfgs, heightfields, init_params: host arrays of n entries
 * (each as for rl_create).  n in [1, 16]. */
typedef struct rl_group rl_group;
rl_status rl_group_create(int32_t n, const rl_config* cfgs, const float* const* heightfields,
                          const float* const* init_params, rl_group** out);
void rl_group_destroy(rl_group* g);
/* The i-th learner's context (owned by the group; valid until rl_group_destroy). */
rl_ctx* rl_group_learner(rl_group* g, int32_t i);
/* One training iteration of every learner.  use_graph != 0 replays the grouped graph (captured
 * on first use); 0 enqueues the learners one after the other on `stream`. */
rl_status rl_group_train_iteration(rl_group* g, int32_t use_graph, void* stream);

/* Context-owned rollout storage (device pointers, valid until rl_destroy):
 * 0 obs [T+1][N][obs_pad], 1 actions [T][N][A], 2 mu [T][N][A], 3 logp [T][N], 4 values [T][N],
 * 5 rewards [T][N], 6 dones [T][N] u8, 7 timeouts [T][N] u8, 8 last values [N],
 * 9 advantages [T][N], 10 returns [T][N], 11 levels [N] int32, 12 stats [RL_NSTATS],
 * 13 the last update's minibatch permutations [epochs][B] int32 (minibatch m of epoch e is
 * rows m B / minibatches ... (m + 1) B / minibatches - 1 of row e), 14 the last update's
 * per-minibatch trace [epochs * minibatches][2] fp32 = (KL(pi_old || pi_new), alpha after
 * Algorithm 1), in the order the minibatches ran. */
rl_status rl_get_storage(rl_ctx* ctx, int32_t which, void** ptr, size_t* bytes);

/* Device status word: RL_OK, or the first device-side failure recorded (RL_ERR_TIMEOUT for a
 * bounded wait that ran out, RL_ERR_STATE for an out-of-range index).  Synchronises. */
rl_status rl_last_device_status(rl_ctx* ctx);

/* Resets the device status word to RL_OK (enqueued on stream), e.g. after a failure has been
 * handled; the context's buffers and state are untouched. */
rl_status rl_clear_device_status(rl_ctx* ctx, void* stream);

/* Forced time-out of the bounded device wait (a test of the failure path; no counterpart in the
 * paper): one warp initialises an mbarrier that nothing arrives on and waits for it with the bounded
 * wait of the tensor-core kernels (2 s on the global timer), which records RL_ERR_TIMEOUT in the
 * context's status word (the first failure recorded wins) and returns, leaving the CUDA context
 * usable.  Enqueued on stream without synchronising; rl_last_device_status then reports
 * RL_ERR_TIMEOUT.  RL_ERR_INVALID_ARG for a null context. */
rl_status rl_diag_forced_timeout(rl_ctx* ctx, void* stream);

/* In-graph timing of the kernels of rl_train_iteration, by class: RL_PROF_GEMM (every MLP GEMM,
 * rollout and update), RL_PROF_LOSS (loss head), RL_PROF_ADAM, RL_PROF_ENV (env step),
 * RL_PROF_ACT (action head), RL_PROF_GATHER (minibatch gather), RL_PROF_OTHER (GAE,
 * permutation, bookkeeping); RL_PROF_ALL selects every class.  enable (on != 0) adds the class
 * to the recorded set, on == 0 removes it; CUDA events are then recorded around each launch of
 * a recorded class on the launching stream (captured into the graph, which is rebuilt on next
 * use).  Events perturb the timing they measure, so time throughput with profiling off.
 * rl_profile_read: summed event time (ms) and launch count over every recorded class, for the
 * last iteration; rl_profile_read_class: the same for one class.  Both synchronise. */
#define RL_PROF_GEMM 0
#define RL_PROF_LOSS 1
#define RL_PROF_ADAM 2
#define RL_PROF_ENV 3
#define RL_PROF_ACT 4
#define RL_PROF_GATHER 5
#define RL_PROF_OTHER 6
#define RL_PROF_ALL 7
rl_status rl_profile_enable(rl_ctx* ctx, int32_t kernel_class, int32_t on);
rl_status rl_profile_read(rl_ctx* ctx, float* total_ms, int32_t* launches);
rl_status rl_profile_read_class(rl_ctx* ctx, int32_t kernel_class, float* total_ms, int32_t* launches);

/* Tile autotuner: times each GEMM site (per hidden layer: the update's forward, input gradient
 * and weight gradient at minibatch rows, and the rollout's forward at num_envs rows; actor and
 * critic in one launch) over candidate tile widths
 * (64, 128, 256 output columns), tile modes (one CTA per tile, a CTA pair on the cta_group::2
 * MMA, or one CTA per tile with two K blocks per pipeline stage) and, for weight gradients, split-K counts (one and two waves of the width's tiles over the SMs, half and double the default;
 * timed together with the summation of their partials, which Adam performs) on the context's
 * own buffers, keeps the fastest, then times the fused forward of the three hidden layers
 * (rl_set_forward_fused) against the chosen per-layer launches at both forward sites and keeps
 * the faster, and drops a captured iteration graph so the next
 * rl_train_iteration re-captures with the new shapes.  Synchronises; the buffers it runs on are
 * scratch (parameters, Adam state and env state are untouched).  report (host, may be NULL): a
 * JSON summary of the chosen shapes and their times, truncated to report_bytes. */
rl_status rl_autotune(rl_ctx* ctx, char* report, size_t report_bytes, void* stream);

/* Pins the tile shape of one GEMM site of a BF16 context (no counterpart in the paper: a tuning
 * control of this implementation).  site: 0 forward, 1 input gradient (layer >= 1), 2 weight
 * gradient (the update's sites, minibatch rows), 3 the rollout's forward (num_envs rows);
 * layer: hidden layer index; bn: output tile width 64, 128 or 256 dividing the site's output
 * width; cluster: 1 (one CTA per 128-row tile), 3 (pairs of CTAs run one 256-row tile on the
 * cta_group::2 MMA, each loading half of B) or 4 (one CTA per tile, two K blocks per pipeline
 * stage fetched by one 3D TMA copy per operand) or 5 (weight-stationary, sites 0, 1 and 3: each
 * CTA keeps one column tile of the layer's weights in shared memory and streams the activations of
 * its row tiles, two K blocks per stage), or, at the weight gradient (site 2) only, 6 and 7
 * (modes 1 and 4 with the split-K partials reduced inside the GEMM: the partials of a tile are
 * computed by a cluster of c CTAs, c the largest divisor of the split count in 2 .. 8, which sum
 * them in rank order through distributed shared memory, so that Adam sums splits / c partials;
 * one CTA per tile and split, and no reduction for a learner whose GEMM CTAs are capped below that
 * count); 3 needs at least two 128-row tiles at the site and a
 * tile width of at least 128, 4 and 7 a tile width of at most 128, 5 a weight slice (tile width x the
 * layer's K x 2 bytes) that leaves room for a stage of the ring (2, a B tile shared by TMA
 * multicast, is not offered and returns RL_ERR_INVALID_ARG);
 * splits: weight-gradient split-K count (1 .. the larger of twice the default and two waves of
 * 64-wide tiles over 148 SMs, rounded so every slice is a multiple of 64 rows), ignored for the
 * other sites.  Drops a captured iteration graph.
 * RL_ERR_INVALID_ARG for any other value or an FP32 context; nothing is changed then. */
rl_status rl_set_gemm_tiles(rl_ctx* ctx, int32_t site, int32_t layer, int32_t bn, int32_t cluster, int32_t splits);

/* Runs the forward pass of the three hidden layers (Sec. 2.2's ELU MLPs, actor and critic) as one
 * fused launch instead of one GEMM launch per layer (no counterpart in the paper: a scheduling
 * control of this implementation, chosen by rl_autotune).  site: 0 the update's forward (every
 * layer's activations are written, for the backward), 3 the rollout's (only the last layer's);
 * on: 1 fused, 0 layer by layer (the default).  Each CTA carries one 128-row tile of one network
 * through all three layers on the tensor cores, the activations staying in shared memory; the
 * products are accumulated in the same order and finished by the same epilogue arithmetic as the
 * per-layer launches, so both forms give the same bits.  While the context's GEMM CTAs are capped
 * (rl_set_gemm_ctas, grouped learners) the forward runs layer by layer whatever the setting, since
 * the fused launch takes one CTA per row tile and network; rl_autotune then does not time it.
 * Drops a captured iteration graph.
 * RL_ERR_INVALID_ARG for another site or value, or (on = 1) an FP32 context or widths the fused
 * form does not take: three hidden layers, input width a multiple of 64 up to 256, first width a
 * multiple of 128 up to 512, second and third multiples of 128 up to 256. */
rl_status rl_set_forward_fused(rl_ctx* ctx, int32_t site, int32_t on);
/* 1 if the site's forward runs fused (set, and the GEMM CTAs uncapped), 0 if layer by layer, -1
 * for a null context or another site. */
int32_t rl_get_forward_fused(rl_ctx* ctx, int32_t site);

/* Caps the persistent CTAs of the context's tensor-core GEMM launches (no counterpart in the
 * paper: a scheduling control of this implementation).  max_ctas 0: one CTA per SM (the default
 * of a lone learner); n >= 1: at most n CTAs (a cluster mode of two CTAs per tile counts both;
 * a weight-stationary site runs at least one CTA per (network, column tile) group).
 * rl_group_create sets each learner's cap to twice its share of the SMs by robot count (at least
 * 16), so that the learners' launches run side by side.  The cap changes which CTA computes a
 * tile, never a result.  Drops a captured iteration graph.  RL_ERR_INVALID_ARG for a negative
 * value or a null context. */
rl_status rl_set_gemm_ctas(rl_ctx* ctx, int32_t max_ctas);

/* One Adam step (Sec. 2.2, Table 3; Kingma & Ba's bias-corrected update with beta1 0.9, beta2
 * 0.999, eps 1e-8) by the library's Adam kernel, on caller buffers: the optimizer step of the PPO
 * update exposed on its own for measurement and tests (no entry point of its own in the paper).
 * n parameters p (fp32, updated in place); the gradient as nsplit >= 1 partial sums, partial q of
 * element i at g[q n + i], summed in the kernel's fixed order; moments m, v (fp32, in place, zero
 * before the first step); learning rate lr >= 0; t >= 1 the step count of the bias corrections
 * 1 - 0.9^t and 1 - 0.999^t; bf16_out (may be NULL): receives the new p rounded to bf16.  All
 * device pointers; 16-byte aligned buffers and n a multiple of 4 take the 4-wide form.  Enqueues on
 * stream without synchronising.  RL_ERR_INVALID_ARG for n < 1, nsplit < 1, t < 1, a negative or
 * NaN lr or a null buffer. */
rl_status rl_adam_step(int64_t n, float* p, const float* g, int32_t nsplit, float* m, float* v, float lr, int32_t t,
                       void* bf16_out, void* stream);

/* Diagnostic: C = A B^T with the library's tcgen05 BF16 tensor-core GEMM kernel (FP32
 * accumulation), for checking the tensor-core path in isolation.  A [M][K] bf16, B [N][K] bf16
 * (row-major, K contiguous), C [M][N] fp32.  K % 8 == 0 (16-byte rows), N % 64 == 0, pointers
 * 16-byte aligned.  The paper has no counterpart; it is the GEMM behind rl_policy_act and
 * rl_ppo_update in RL_BF16 precision. */
rl_status rl_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A, const void* B, float* C, void* stream);

/* Diagnostic, the weight-gradient form: C = At^T Bt, i.e. C[m][n] = sum_k At[k][m] Bt[k][n],
 * with At [K][M] bf16 and Bt [K][N] bf16 row-major (the operands read MN-major, as the
 * weight-gradient GEMM reads the row-major activations and gradients), C [M][N] fp32.
 * M % 8 == 0, N % 64 == 0, K >= 1, pointers 16-byte aligned.  No counterpart in the paper. */
rl_status rl_gemm_bf16_tn(int32_t M, int32_t N, int32_t K, const void* At, const void* Bt, float* C, void* stream);

/* Diagnostic with an explicit tile shape: operands 0 computes C = A B^T (A [M][K], B [N][K]), 1
 * computes C = At^T Bt (At [K][M], Bt [K][N]); bn: output tile width 64, 128 or 256 dividing N;
 * cluster: 1 (one CTA per tile) or 3 (pairs of CTAs run one 256-row tile on the cta_group::2
 * tensor-core MMA, each CTA loading half of the B tile; bn 128 or 256).  Requirements as for
 * rl_gemm_bf16 (operands 0) or rl_gemm_bf16_tn (operands 1).
 * operands 2 / 3: the forms of 0 / 1 with two K blocks per pipeline stage (one 3D TMA copy per
 * operand and stage), cluster 1 and bn <= 128 only; operands 2 needs K % 64 == 0, operands 3
 * M % 64 == 0.  No counterpart in the paper. */
rl_status rl_gemm_bf16_shape(int32_t M, int32_t N, int32_t K, const void* A, const void* B, float* C, int32_t operands,
                             int32_t bn, int32_t cluster, void* stream);

/* Number of kernel launches one rl_train_iteration enqueues (host-side count). */
int32_t rl_launches_per_iteration(rl_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* RL_B300_H */
