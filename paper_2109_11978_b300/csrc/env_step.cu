// Env-side tensor math of one 50 Hz policy step for all robots, fused in one kernel:
// PD control over the simulation substeps with the seeded physics stand-in, the Table 2
// reward, termination / time-out / bootstrap, the curriculum update and respawn, and the
// observation with bilinear height samples and Table 4 noise.
//
// Layout: the env state is a structure of arrays in HBM ([57][N] fp32 + [3][N] int32).  A block
// of 512 threads owns 16 robots.  Phase 0 (policy heads fused in): one warp per robot.  Phase 1:
// the stand-in's independent recurrences of a robot (its 12 joints and three base chains) on
// separate threads of the first 256, the feet on a sixteenth, meeting in shared memory for the
// reward and the reset, leaving a 60-float record per robot in shared memory.  Phase 2: the 16
// warps assemble the observation rows (a pair of robots per two warps, which take alternate
// 64-column blocks, two adjacent columns per lane), so the row of obs_pad floats (or bf16) leaves
// as full 128-byte lines and the height samples of a robot are gathered by many lanes in
// parallel from the L2-resident heightfield; the rotated sample offsets of the grid come from a
// per-block table.  At a few thousand robots the kernel is one wave of latency-bound blocks, so
// the extra threads shorten each block's path rather than add throughput.
#include "act_row.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace rl {

namespace {

// Physics stand-in constants (dyadic, exact in fp32).  The stand-in is not the paper's
// method: it replaces PhysX with a linear stochastic transition that both the CUDA path and
// the oracle evaluate as the same fp32 recurrence, operation by operation.
constexpr float A_Q = 0.96875f, INV_I = 2.0f, S_Q = 0.0625f;
constexpr float RHO_V = 0.96875f, ONE_M_RHO_V = 0.03125f, S_V = 0.03125f;
constexpr float RHO_W = 0.96875f, ONE_M_RHO_W = 0.03125f, S_W = 0.0625f;
constexpr float RHO_G = 0.96875f, S_G = 0.0078125f;
constexpr float RHO_Z = 0.96875f, ONE_M_RHO_Z = 0.03125f, S_Z = 0.00390625f;
constexpr float Z_NOM0 = 0.5f, Z_NOM_PER_LEVEL = 0.0625f;

// Table 2 weights (times dt) and phi(x) = exp(-|x|^2 / 0.25).
constexpr float W_LIN = 1.0f, W_ANG = 0.5f, W_VZ = 4.0f, W_WXY = 0.05f, W_JOINT = 0.001f;
constexpr float W_TAU = 0.00002f, W_RATE = 0.25f, W_COLL = 0.001f, W_AIR = 2.0f;
constexpr float PHI_INV = 4.0f, AIR_TARGET = 0.5f;

// Random-key slots.
constexpr int SLOT_CRASH = 128, SLOT_COLL = 129, SLOT_LOOP = 130, SLOT_PUSH = 131;
constexpr int SLOT_CMD = 133, SLOT_HEADING = 136, SLOT_EPLEN = 138, SLOT_OBS = 256;

// Foot-contact schedule of the stand-in.
constexpr int CONTACT_PERIOD = 40, CONTACT_DUTY = 20, CONTACT_ENV_STRIDE = 7;

constexpr int REC = 64;         // floats per robot record in shared memory
constexpr int GTAB = 1024;      // height-grid offset table entries (larger grids compute in place)

// Record fields (after the 48 proprioceptive observations).
constexpr int R_PX = 48, R_PY = 49, R_HC = 50, R_HS = 51, R_Z = 52, R_BX = 53, R_BY = 54;
constexpr int R_KEYLO = 55, R_KEYHI = 56;

#define FADD __fadd_rn
#define FSUB __fsub_rn
#define FMUL __fmul_rn

__device__ __forceinline__ float znom(int level) {
    return FADD(FMUL(__int2float_rn(level), Z_NOM_PER_LEVEL), Z_NOM0);
}

// Table 4 half-widths by observation column.
__device__ __forceinline__ float noise_scale(int c) {
    if (c < 3) return 0.01f;       // base linear velocity
    if (c < 6) return 0.2f;        // base angular velocity
    if (c < 9) return 0.05f;       // projected gravity
    if (c < 12) return 0.0f;       // commands
    if (c < 24) return 0.01f;      // joint positions
    if (c < 36) return 1.5f;       // joint velocities
    if (c < 48) return 0.0f;       // previous actions (not listed)
    return 0.1f;                   // terrain heights
}

struct Respawn {
    float hc, hs, cx, cy, cw;
};

// Fresh heading and command of a respawned robot (Sec. 3.1: commands are drawn at reset and
// held for the episode).  The heading is a random direction normalised in fp32.
__device__ __forceinline__ Respawn respawn_draw(uint64_t key, const EnvParams& p) {
    Respawn r;
    float hx = uniform_pm1(hi32(rng_word(key, SLOT_HEADING)));
    float hy = uniform_pm1(hi32(rng_word(key, SLOT_HEADING + 1)));
    float n2 = FADD(FMUL(hx, hx), FMUL(hy, hy));
    bool ok = n2 > 9.5367431640625e-07f;   // 2^-20
    float nn = __fsqrt_rn(ok ? n2 : 1.0f);
    r.hc = ok ? __fdiv_rn(hx, nn) : 1.0f;
    r.hs = ok ? __fdiv_rn(hy, nn) : 0.0f;
    r.cx = FMUL(uniform_pm1(hi32(rng_word(key, SLOT_CMD))), p.cmd_range[0]);
    r.cy = FMUL(uniform_pm1(hi32(rng_word(key, SLOT_CMD + 1))), p.cmd_range[1]);
    r.cw = FMUL(uniform_pm1(hi32(rng_word(key, SLOT_CMD + 2))), p.cmd_range[2]);
    return r;
}

// Bilinear terrain height at cell coordinate (ib + f) along each axis, clamped to the map.
// ib is the integer cell of the tile centre, f the fp32 offset in cells (small magnitude,
// so the split keeps sub-micrometre resolution anywhere on the 80 m x 160 m map).
__device__ __forceinline__ float terrain_height(const float* __restrict__ hf, int nx, int ny, int ibx,
                                               float fx, int iby, float fy) {
    float flx = floorf(fx), fly = floorf(fy);
    int i0 = ibx + (int)flx, j0 = iby + (int)fly;
    float fu = fx - flx, fv = fy - fly;
    if (i0 < 0) { i0 = 0; fu = 0.f; }
    if (i0 >= nx - 1) { i0 = nx - 2; fu = 1.f; }
    if (j0 < 0) { j0 = 0; fv = 0.f; }
    if (j0 >= ny - 1) { j0 = ny - 2; fv = 1.f; }
    const float* h = hf + (size_t)i0 * ny + j0;
    float h00 = __ldg(h), h01 = __ldg(h + 1), h10 = __ldg(h + ny), h11 = __ldg(h + ny + 1);
    return (1.f - fu) * (1.f - fv) * h00 + fu * (1.f - fv) * h10 + (1.f - fu) * fv * h01 + fu * fv * h11;
}

// Phase-1 roles of the first 256 threads of a block (16 robots): threads 0..191 one (robot, joint) pair
// each; then 16 threads each for the three independent base chains of the stand-in (planar
// velocity / yaw / heading / position; vertical and roll / pitch rates; gravity direction and
// height) and 16 for the feet (from thread 192 on: 16 threads per role).  Each role is a whole
// number of warps or half-warps.
constexpr int T_PLANE = 192;
constexpr int T_ROLES = T_PLANE + 64;   // planar, rates, gravity, feet: 16 threads each

// FUSE: 0, or 16 * bf16 + H / 32 of a fused policy head (its per-row evaluation runs first).
template <int MODE, int FUSE>   // MODE 0 = policy step, 1 = spawn all robots (initial state)
__global__ void __launch_bounds__(512, 2) env_step_kernel(EnvParams p) {
    // The fused form follows the rollout's last forward layer, which writes only the hidden rows:
    // the robot state, the head weights and the iteration counter come from kernels that have
    // completed when this one starts, so they are read before the wait for that layer.  The plain
    // form may follow a kernel that writes the state (a reset) and waits first.
    if constexpr (FUSE == 0) {
        pdl_wait();
        pdl_trigger();
    }
    constexpr int ENVS = 16, THREADS = 512;
    extern __shared__ float rec_raw[];
    float (*rec)[REC] = reinterpret_cast<float (*)[REC]>(rec_raw);       // [ENVS][REC]
    // exchange of phase 1: the joints' reward terms, the rates, the feet, the reset decision
    __shared__ float xj[4][ENVS][12];
    __shared__ float xr[3][ENVS];
    __shared__ float xf[ENVS];
    __shared__ int xfi[ENVS], xd[ENVS], xl[ENVS];
    __shared__ float act_s[ENVS][12], val_s[ENVS];            // fused head: actions and values
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tid = threadIdx.x;
    const int env0 = blockIdx.x * ENVS;
    const int N = p.N;
    const unsigned long long it = p.iteration ? *p.iteration : 0ull;
    // grid sample offsets (before rotation) of the height columns, shared by the block's robots
    float* gtab = rec_raw + ENVS * REC;                                  // [2][GTAB]
    const int ng = p.GX * p.GY;
    for (int k = tid; k < ng && k < GTAB; k += THREADS) {
        const int ix = k % p.GX, iy = k / p.GX;
        gtab[k] = ((float)ix - 0.5f * (float)(p.GX - 1)) * p.grid_sp;
        gtab[GTAB + k] = ((float)iy - 0.5f * (float)(p.GY - 1)) * p.grid_sp;
    }
    // Phase 1's inputs: each thread's role and its part of the robot state
    const bool joint = tid < T_PLANE;
    const bool p1 = tid < T_ROLES;                                     // threads past the roles idle here
    const int lr = joint ? tid / 12 : (tid - T_PLANE) & 15;           // robot of the block
    const int jl = joint ? tid % 12 : 0;
    const int role = joint ? 0 : p1 ? 1 + (tid - T_PLANE) / 16 : 5;   // 1 planar, 2 rates, 3 grav, 4 feet, 5 idle
    const int e = env0 + lr;
    const bool valid = e < N;
    const int ec = valid ? e : N - 1;          // a readable robot for the threads of a missing one
    float* sf = p.sf;
    int* si = p.si;
    auto F = [&](int r) -> float& { return sf[(size_t)r * N + ec]; };
    float q = 0.f, qd = 0.f, ap = 0.f, a = 0.f;                          // joint
    float px = 0.f, py = 0.f, hc = 0.f, hs = 0.f, vx = 0.f, vy = 0.f, wz = 0.f, cx = 0.f, cy = 0.f, cw = 0.f;   // planar
    float vz = 0.f, wx = 0.f, wy = 0.f;                                  // rates
    float gx = 0.f, gy = 0.f, gz = 0.f, z = 0.f;                         // grav
    float tair[4] = {0.f, 0.f, 0.f, 0.f};                               // feet
    if (joint) {
        q = F(RL_F_Q + jl); qd = F(RL_F_QD + jl); ap = F(RL_F_AP + jl);
    } else if (role == 1) {
        px = F(RL_F_PX); py = F(RL_F_PY); hc = F(RL_F_HC); hs = F(RL_F_HS);
        vx = F(5); vy = F(6); wz = F(10); cx = F(14); cy = F(15); cw = F(16);
    } else if (role == 2) {
        vz = F(7); wx = F(8); wy = F(9);
    } else if (role == 3) {
        gx = F(11); gy = F(12); gz = F(13); z = F(RL_F_Z);
    } else if (role == 4) {
#pragma unroll
        for (int f = 0; f < 4; ++f) tair[f] = F(RL_F_TAIR + f);
    }
    int eplen = si[(size_t)RL_I_EPLEN * N + ec];
    int level = si[(size_t)RL_I_LEVEL * N + ec];
    int contact = si[(size_t)RL_I_CONTACT * N + ec];
    if constexpr (FUSE != 0) {
        // Phase 0 (fused policy head): the head weights into shared memory, then one warp per
        // robot evaluates mu, the sampled action, logp and V exactly as the action-head kernel
        // does, writing the rollout's records and the block's actions / values for phase 1.  The
        // head weights are staged before the wait for the forward layer, the warp's hidden rows
        // loaded after it.
        static_assert(ENVS == THREADS / 32, "one robot per warp");
        constexpr bool HB = (FUSE >> 4) != 0;
        constexpr int NK = FUSE & 15;
        const int mm[1] = {env0 + warp};
        const bool ok[1] = {env0 + warp < N};
        float* Wa = gtab + 2 * GTAB;
        float* Wc = Wa + p.act.A * p.act.H;
        // every load of the staging issued before its stores (16-byte pieces where the layout
        // allows), so that the block waits for one round trip to L2 instead of one per piece
        const int nwa = p.act.A * p.act.H, nwc = p.act.H;
        if (((reinterpret_cast<uintptr_t>(p.act.Wa) | reinterpret_cast<uintptr_t>(p.act.Wc)) & 15u) == 0 && nwa % 4 == 0 &&
            nwc % 4 == 0) {
            const float4* wa4 = reinterpret_cast<const float4*>(p.act.Wa);
            const float4* wc4 = reinterpret_cast<const float4*>(p.act.Wc);
            float4 ra[2], rc;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int i = tid + u * THREADS;
                if (i < nwa / 4) ra[u] = __ldg(wa4 + i);
            }
            if (tid < nwc / 4) rc = __ldg(wc4 + tid);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int i = tid + u * THREADS;
                if (i < nwa / 4) reinterpret_cast<float4*>(Wa)[i] = ra[u];
            }
            if (tid < nwc / 4) reinterpret_cast<float4*>(Wc)[tid] = rc;
        } else {
            for (int i = tid; i < nwa; i += THREADS) Wa[i] = p.act.Wa[i];
            for (int i = tid; i < nwc; i += THREADS) Wc[i] = p.act.Wc[i];
        }
        pdl_wait();
        pdl_trigger();
        float hrc[1][NK], hra[1][NK];
        if (ok[0]) act_rows_load<HB, NK, 1>(p.act, mm, ok, true, lane, hrc, hra);
        __syncthreads();
        {
            float* const as[1] = {act_s[warp]};
            float* const vs[1] = {&val_s[warp]};
            if (ok[0]) act_rows_loaded<HB, NK, 1>(p.act, Wa, Wc, mm, ok, it, true, lane, as, vs, hrc, hra);
        }
        __syncthreads();
    }
    // Phase 1: the stand-in's joints and base chains are independent recurrences, each on its own
    // thread with the same fp32 operations as one robot per thread would use; the reward sums
    // and the reset decision meet on the robot's planar thread through shared memory (the joint
    // terms summed in joint order).
    uint64_t key;
    float st_r = 0.f, st_d = 0.f, st_l = 0.f;   // per-robot statistics (planar threads)
    if (MODE == 0) {
        key = rng_key(p.seed, kStreamEnv, it, (uint64_t)p.t, (uint64_t)ec);
        const float qd_old = qd;
        if (joint) a = FUSE != 0 ? act_s[lr][jl] : __ldg(p.actions + (size_t)ec * 12 + jl);
        // Pushes (Sec. 3.3): every push_interval steps of the episode, +-push_vel in x, y.
        if (role == 1 && p.push_on && eplen > 0 && (eplen % p.push_interval) == 0) {
            vx = FADD(vx, FMUL(p.push_vel, uniform_pm1(hi32(rng_word(key, SLOT_PUSH)))));
            vy = FADD(vy, FMUL(p.push_vel, uniform_pm1(hi32(rng_word(key, SLOT_PUSH + 1)))));
        }
        const float zn = znom(level);
        float sq_tau = 0.f;     // tau^2 of the last substep (Table 2 torque term), joints
        for (int k = 0; k < p.decimation; ++k) {
            const uint32_t base = 32u * (uint32_t)k;
            if (joint) {
                // PD torque (Sec. 3.2) on the target q* = q_def + action_scale a, recomputed every
                // substep (App. A.1.1), consumed by the physics stand-in (exact fp32 recurrence).
                const float qs = FADD(p.q_def[jl], FMUL(p.ascale, a));
                const float tau = FSUB(FMUL(p.kp, FSUB(qs, q)), FMUL(p.kd, qd));
                if (k == p.decimation - 1) sq_tau = tau * tau;
                const float xi = irwin_hall(rng_word(key, base + jl));
                qd = FADD(FADD(FMUL(A_Q, qd), FMUL(p.sim_dt, FMUL(INV_I, tau))), FMUL(S_Q, xi));
                q = FADD(q, FMUL(p.sim_dt, qd));
            } else if (role == 1) {
                vx = FADD(FADD(FMUL(RHO_V, vx), FMUL(ONE_M_RHO_V, cx)), FMUL(S_V, irwin_hall(rng_word(key, base + 12))));
                vy = FADD(FADD(FMUL(RHO_V, vy), FMUL(ONE_M_RHO_V, cy)), FMUL(S_V, irwin_hall(rng_word(key, base + 13))));
                wz = FADD(FADD(FMUL(RHO_W, wz), FMUL(ONE_M_RHO_W, cw)), FMUL(S_W, irwin_hall(rng_word(key, base + 17))));
                const float w = FMUL(wz, p.sim_dt);
                const float c1 = FSUB(hc, FMUL(hs, w)), s1 = FADD(hs, FMUL(hc, w));
                const float nrm = __fsqrt_rn(FADD(FMUL(c1, c1), FMUL(s1, s1)));
                hc = __fdiv_rn(c1, nrm);
                hs = __fdiv_rn(s1, nrm);
                const float dx = FSUB(FMUL(hc, vx), FMUL(hs, vy)), dy = FADD(FMUL(hs, vx), FMUL(hc, vy));
                px = FADD(px, FMUL(p.sim_dt, dx));
                py = FADD(py, FMUL(p.sim_dt, dy));
            } else if (role == 2) {
                vz = FADD(FMUL(RHO_V, vz), FMUL(S_V, irwin_hall(rng_word(key, base + 14))));
                wx = FADD(FMUL(RHO_W, wx), FMUL(S_W, irwin_hall(rng_word(key, base + 15))));
                wy = FADD(FMUL(RHO_W, wy), FMUL(S_W, irwin_hall(rng_word(key, base + 16))));
            } else if (role == 3) {
                gx = FADD(FMUL(RHO_G, gx), FMUL(S_G, irwin_hall(rng_word(key, base + 18))));
                gy = FADD(FMUL(RHO_G, gy), FMUL(S_G, irwin_hall(rng_word(key, base + 19))));
                gz = -__fsqrt_rn(fmaxf(0.0f, FSUB(1.0f, FADD(FMUL(gx, gx), FMUL(gy, gy)))));
                z = FADD(FADD(FMUL(RHO_Z, z), FMUL(ONE_M_RHO_Z, zn)), FMUL(S_Z, irwin_hall(rng_word(key, base + 20))));
            }
        }
        const int eplen_new = eplen + 1;
        if (joint) {
            const float inv_dt = 1.0f / p.dt;
            const float qdd = (qd - qd_old) * inv_dt, da = a - ap;
            xj[0][lr][jl] = qdd * qdd;
            xj[1][lr][jl] = qd * qd;
            xj[2][lr][jl] = da * da;
            xj[3][lr][jl] = sq_tau;
        } else if (role == 2) {
            xr[0][lr] = vz; xr[1][lr] = wx; xr[2][lr] = wy;
        } else if (role == 4) {
            // Feet: contact schedule, air time (fp32, exact), first contacts.
            const int off = (int)(((long long)ec * CONTACT_ENV_STRIDE) % CONTACT_PERIOD);
            int cbits = 0;
            float r_air = 0.f;
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const int ph = (f == 1 || f == 2) ? 20 : 0;
                const bool on = ((eplen_new + off + ph) % CONTACT_PERIOD) < CONTACT_DUTY;
                cbits |= (int)on << f;
                tair[f] = FADD(tair[f], p.dt);
                const bool first = on && !((contact >> f) & 1);
                if (first) r_air += tair[f] - AIR_TARGET;
                if (on) tair[f] = 0.f;
            }
            xf[lr] = r_air;
            xfi[lr] = cbits;
        }
        __syncthreads();
        if (role == 1) {
            const bool crash = hi32(rng_word(key, SLOT_CRASH)) < p.crash_thr;
            const float n_coll = (float)mulhi_n(hi32(rng_word(key, SLOT_COLL)), 3u);
            float sq_qdd = 0.f, sq_qd = 0.f, sq_rate = 0.f, sq_t = 0.f;
#pragma unroll
            for (int j = 0; j < 12; ++j) {
                sq_qdd += xj[0][lr][j];
                sq_qd += xj[1][lr][j];
                sq_rate += xj[2][lr][j];
                sq_t += xj[3][lr][j];
            }
            const float vz_ = xr[0][lr], wx_ = xr[1][lr], wy_ = xr[2][lr], r_air = xf[lr];
            // Reward: the nine Table 2 terms, each weight times dt.
            float e2 = (cx - vx) * (cx - vx) + (cy - vy) * (cy - vy);
            float ew = (cw - wz) * (cw - wz);
            float r = W_LIN * expf(-e2 * PHI_INV) + W_ANG * expf(-ew * PHI_INV) - W_VZ * vz_ * vz_ -
                      W_WXY * (wx_ * wx_ + wy_ * wy_) - W_JOINT * (sq_qdd + sq_qd) - W_TAU * sq_t - W_RATE * sq_rate -
                      W_COLL * n_coll + W_AIR * r_air;
            r *= p.dt;
            // Termination (Sec. 3.2: base contact = crash; Sec. 2.2.1: 20 s time-out) and the
            // time-out bootstrap r += gamma V(o_t) (Sec. 2.2.2).
            const bool timeout = (eplen_new >= p.max_ep) && !crash;
            const bool done = crash || timeout;
            if (timeout) r += p.gamma * (FUSE != 0 ? val_s[lr] : __ldg(p.values + ec));
            int level_new = level;
            if (done) {
                // Curriculum (Sec. 3.1), decided in fp64 with one rounding per operation.
                const double dpx = px, dpy = py, dcx = cx, dcy = cy;
                const double d2 = __dadd_rn(__dmul_rn(dpx, dpx), __dmul_rn(dpy, dpy));
                const double half = __dmul_rn(0.5, (double)p.tile);
                const bool promote = d2 > __dmul_rn(half, half);
                const double vv = __dadd_rn(__dmul_rn(dcx, dcx), __dmul_rn(dcy, dcy));
                const double T = __dmul_rn((double)p.max_ep, (double)p.dt);
                const double thr = __dmul_rn(__dmul_rn(vv, __dmul_rn(T, T)), 0.25);
                const bool demote = d2 < thr;
                if (promote) {
                    level_new = level + 1 >= p.L ? (int)mulhi_n(hi32(rng_word(key, SLOT_LOOP)), (uint32_t)p.L) : level + 1;
                } else if (demote) {
                    level_new = level > 0 ? level - 1 : 0;
                }
            }
            if (valid) {
                if (p.rew) p.rew[e] = r;
                if (p.done) p.done[e] = (uint8_t)done;
                if (p.timeout) p.timeout[e] = (uint8_t)timeout;
                st_r = r;
                st_d = (float)done;
                st_l = (float)(done ? level_new : level);
            }
            xd[lr] = done;
            xl[lr] = level_new;
        }
        __syncthreads();
        const bool done = xd[lr] != 0;
        ap = a;
        eplen = eplen_new;
        contact = xfi[lr];
        if (done) {
            level = xl[lr];
            // respawn: every thread resets its share (the planar thread draws heading and command)
            if (joint) {
                q = p.q_def[jl]; qd = 0.f; ap = 0.f;
            } else if (role == 1) {
                Respawn rs = respawn_draw(key, p);
                px = 0.f; py = 0.f;
                hc = rs.hc; hs = rs.hs;
                vx = vy = wz = 0.f;
                cx = rs.cx; cy = rs.cy; cw = rs.cw;
            } else if (role == 2) {
                vz = wx = wy = 0.f;
            } else if (role == 3) {
                gx = gy = 0.f; gz = -1.f; z = znom(level);
            } else if (role == 4) {
#pragma unroll
                for (int f = 0; f < 4; ++f) tair[f] = 0.f;
            }
            eplen = 0;
            contact = 0;
        }
    } else {
        // Spawn (initial state): level 0, fresh heading and command, random episode length.
        key = rng_key(p.seed, kStreamInit, 0ull, 0ull, (uint64_t)ec);
        level = 0;
        if (joint) {
            q = p.q_def[jl]; qd = 0.f; ap = 0.f;
        } else if (role == 1) {
            Respawn rs = respawn_draw(key, p);
            px = 0.f; py = 0.f;
            hc = rs.hc; hs = rs.hs;
            vx = vy = wz = 0.f;
            cx = rs.cx; cy = rs.cy; cw = rs.cw;
        } else if (role == 2) {
            vz = wx = wy = 0.f;
        } else if (role == 3) {
            gx = gy = 0.f; gz = -1.f; z = znom(0);
        } else if (role == 4) {
#pragma unroll
            for (int f = 0; f < 4; ++f) tair[f] = 0.f;
        }
        eplen = p.randomize_eplen ? (int)mulhi_n(hi32(rng_word(key, SLOT_EPLEN)), (uint32_t)p.max_ep) : 0;
        contact = 0;
    }
    // Store the state (each thread its share) and the record of the observation phase: the 48
    // proprioceptive values (Sec. 3.2 order), then position / heading / height and the
    // tile-centre cell.
    float* R = rec[lr];
    if (valid) {
        if (joint) {
            F(RL_F_Q + jl) = q; F(RL_F_QD + jl) = qd; F(RL_F_AP + jl) = ap;
            R[12 + jl] = q - p.q_def[jl];
            R[24 + jl] = qd;
            R[36 + jl] = ap;
        } else if (role == 1) {
            F(RL_F_PX) = px; F(RL_F_PY) = py; F(RL_F_HC) = hc; F(RL_F_HS) = hs;
            F(5) = vx; F(6) = vy; F(10) = wz; F(14) = cx; F(15) = cy; F(16) = cw;
            si[(size_t)RL_I_EPLEN * N + e] = eplen;
            si[(size_t)RL_I_LEVEL * N + e] = level;
            si[(size_t)RL_I_CONTACT * N + e] = contact;
            if (p.level_out) p.level_out[e] = level;
            if (p.tidx_out) p.tidx_out[e] = level * p.C + (e % p.C);
            R[0] = vx; R[1] = vy; R[5] = wz; R[9] = cx; R[10] = cy; R[11] = cw;
            R[R_PX] = px; R[R_PY] = py; R[R_HC] = hc; R[R_HS] = hs;
            R[R_BX] = __int_as_float(level * p.cpt + p.cpt / 2);
            R[R_BY] = __int_as_float((e % p.C) * p.cpt + p.cpt / 2);
            R[R_KEYLO] = __uint_as_float(lo32(key));
            R[R_KEYHI] = __uint_as_float(hi32(key));
        } else if (role == 2) {
            F(7) = vz; F(8) = wx; F(9) = wy;
            R[2] = vz; R[3] = wx; R[4] = wy;
        } else if (role == 3) {
            F(11) = gx; F(12) = gy; F(13) = gz; F(RL_F_Z) = z;
            R[6] = gx; R[7] = gy; R[8] = gz;
            R[R_Z] = z;
        } else if (role == 4) {
#pragma unroll
            for (int f = 0; f < 4; ++f) F(RL_F_TAIR + f) = tair[f];
        }
    }
    // per-block statistics (the planar threads of warp 6 carry them; other lanes add zeros)
    if (MODE == 0 && p.stats && warp == T_PLANE / 32) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            st_r += __shfl_xor_sync(0xffffffffu, st_r, o);
            st_d += __shfl_xor_sync(0xffffffffu, st_d, o);
            st_l += __shfl_xor_sync(0xffffffffu, st_l, o);
        }
        if (lane == 0) { atomicAdd(p.stats + 0, st_r); atomicAdd(p.stats + 1, st_d); atomicAdd(p.stats + 2, st_l); }
    }
    __syncthreads();

    // Phase 2: observation rows, two columns per lane; a warp's two robots (w, w + 8 for
    // w = warp mod 8) go through the column loop together, so that the height samples' loads of
    // both rows (and of several column pairs, unrolled) are in flight at once, and the two warps
    // of a robot pair take alternate 64-column blocks of the row.
    static_assert(ENVS == THREADS / 32, "two warps per robot pair");
    constexpr int PW = ENVS / 2;                 // warps per column half
    {
        int ev[2];
        bool okr[2];
        const float* Rr[2];
        uint64_t keyr[2];
        float pxr[2], pyr[2], hcr[2], hsr[2], zr[2];
        int ibxr[2], ibyr[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int le = (warp % PW) + q * PW;
            ev[q] = env0 + le;
            okr[q] = ev[q] < N;
            const float* R = rec[le];
            Rr[q] = R;
            keyr[q] = ((uint64_t)__float_as_uint(R[R_KEYHI]) << 32) | __float_as_uint(R[R_KEYLO]);
            pxr[q] = R[R_PX]; pyr[q] = R[R_PY]; hcr[q] = R[R_HC]; hsr[q] = R[R_HS]; zr[q] = R[R_Z];
            ibxr[q] = __float_as_int(R[R_BX]); ibyr[q] = __float_as_int(R[R_BY]);
        }
#pragma unroll 2
        for (int c0 = 2 * lane + 64 * (warp / PW); c0 < p.Op; c0 += 128) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (!okr[q]) continue;
                const float* R = Rr[q];
                float v[2];
                uint64_t w = (p.noise_on && c0 < p.O) ? rng_word(keyr[q], SLOT_OBS + (c0 >> 1)) : 0ull;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = c0 + h;
                    float val = 0.f;
                    if (c < 48) {
                        val = R[c];
                    } else if (c < p.O) {
                        const int k = c - 48;
                        float gxo, gyo;
                        if (k < GTAB) {
                            gxo = gtab[k];
                            gyo = gtab[GTAB + k];
                        } else {
                            const int ix = k % p.GX, iy = k / p.GX;
                            gxo = ((float)ix - 0.5f * (float)(p.GX - 1)) * p.grid_sp;
                            gyo = ((float)iy - 0.5f * (float)(p.GY - 1)) * p.grid_sp;
                        }
                        const float fx = (pxr[q] + (hcr[q] * gxo - hsr[q] * gyo)) * p.inv_res;
                        const float fy = (pyr[q] + (hsr[q] * gxo + hcr[q] * gyo)) * p.inv_res;
                        val = zr[q] - terrain_height(p.hf, p.nx, p.ny, ibxr[q], fx, ibyr[q], fy);
                    }
                    if (p.noise_on && c < p.O) val += noise_scale(c) * uniform_pm1(h == 0 ? hi32(w) : lo32(w));
                    v[h] = val;
                }
                const int e = ev[q];
                if (p.obs_bf16) {
                    __nv_bfloat162 b2 = __floats2bfloat162_rn(v[0], v[1]);
                    *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(p.obs) + (size_t)e * p.Op + c0) = b2;
                } else {
                    *reinterpret_cast<float2*>(reinterpret_cast<float*>(p.obs) + (size_t)e * p.Op + c0) = make_float2(v[0], v[1]);
                }
            }
        }
    }
}

}  // namespace

template <int MODE, int FUSE>
static cudaError_t launch_cfg(const EnvParams& p, cudaStream_t s) {
    size_t smem = ((size_t)16 * REC + 2 * GTAB) * sizeof(float);
    if (FUSE != 0) smem += (size_t)(p.act.A * p.act.H + p.act.H) * sizeof(float);
    cudaError_t e = launch_pdl(env_step_kernel<MODE, FUSE>, dim3((p.N + 15) / 16), dim3(512), smem, s, p);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Shared memory: 12 KiB per block (16 robot records + the grid table), plus at most 13 KiB of
// head weights when the policy head is fused: within the default limit, nothing to set.  Blocks
// of 512 threads, 16 robots each.
cudaError_t env_prepare() { return cudaSuccess; }

cudaError_t launch_env_step(const EnvParams& p, int mode, cudaStream_t s) {
    if (p.N <= 0) return cudaSuccess;
    if (mode != 0) return launch_cfg<1, 0>(p, s);
    if (!p.act.ha) return launch_cfg<0, 0>(p, s);
    // fused policy head: 12 actions (the stand-in's joints), last hidden width 64, 128 or 256
    const HeadParams& h = p.act;
    if (h.A != 12 || !(h.H == 64 || h.H == 128 || h.H == 256) || !h.hc || !h.Wa || !h.Wc || !h.ba || !h.bc || !h.log_std ||
        !h.values || !h.actions || !h.mu || !h.logp)
        return cudaErrorInvalidValue;
    const int nk = h.H / 32;
    if (h.bf16) {
        if (nk == 2) return launch_cfg<0, 16 + 2>(p, s);
        if (nk == 4) return launch_cfg<0, 16 + 4>(p, s);
        return launch_cfg<0, 16 + 8>(p, s);
    }
    if (nk == 2) return launch_cfg<0, 2>(p, s);
    if (nk == 4) return launch_cfg<0, 4>(p, s);
    return launch_cfg<0, 8>(p, s);
}

}  // namespace rl
