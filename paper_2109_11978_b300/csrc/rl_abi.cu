// C ABI of the library: the learner context (every buffer allocated once, at creation), the
// orchestration of the rollout step, GAE and the PPO update over the kernels, and the CUDA
// graph of a whole training iteration.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "gemm_tc.cuh"
#include "mlp_fused.cuh"
#include "kernels.cuh"

using namespace rl;

namespace {

struct LayerInfo {
    int in_log, in, out;   // fan-in (logical / padded), fan-out
    long long w, b;        // offsets in the internal flat parameter vector
};

struct Seg {               // one tensor of the flat parameter layout
    long long ioff, loff;  // internal / logical offset
    int rows, cols_int, cols_log;
};

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

struct rl_ctx {
    rl_config cfg;
    int N, T, O, Op, A, NH, hid[4], B, Mb, HL, rows;
    bool bf16;
    int device;
    // parameters
    long long P = 0, P_log = 0;
    LayerInfo L[2][5];
    long long logstd = 0;
    std::vector<Seg> segs;
    std::vector<void*> allocs;
    float *params = nullptr, *am = nullptr, *av = nullptr, *grad_int = nullptr;
    float* scal = nullptr;
    unsigned long long* iter = nullptr;
    int* status = nullptr;
    float *acc = nullptr, *stats = nullptr;
    // env
    float* hf = nullptr;
    float* sf = nullptr;
    int* si = nullptr;
    int nx = 0, ny = 0, cpt = 0;
    // rollout storage
    void* obs = nullptr;
    float *actions = nullptr, *mu = nullptr, *logp = nullptr, *values = nullptr, *rew = nullptr, *last_val = nullptr;
    float *adv = nullptr, *ret = nullptr;
    uint8_t *done = nullptr, *timeout = nullptr;
    int* level = nullptr;
    float* gae_ws = nullptr;
    int gae_nparts = 0;
    // update workspaces
    int* perm = nullptr;
    float* trace = nullptr;                      // per minibatch of the last update: KL, alpha after Algorithm 1
    int* iota = nullptr;
    float* logstd_old = nullptr;
    void* X0 = nullptr;                          // the current minibatch's observations (= X0buf[xcur])
    void* X0buf[2] = {nullptr, nullptr};         // two buffers: the next minibatch is gathered into the other
    int xcur = 0;
    cudaStream_t side = nullptr;                 // the next minibatch's gather runs here, beside the current one
    cudaEvent_t ev_fork[2] = {nullptr, nullptr}, ev_join[2] = {nullptr, nullptr};
    cudaStream_t wside = nullptr;                // weight gradients, beside the next input gradient
    cudaEvent_t ev_dw[4] = {}, ev_dw_join = nullptr;
    cudaEvent_t ev_perm_fork = nullptr, ev_perm_join = nullptr;   // the shuffle, beside GAE
    cudaEvent_t ev_pack_fork = nullptr, ev_pack_join = nullptr;   // the records, beside minibatch 0
    void* H[2][4] = {};
    void* dY[2][4] = {};
    float* gw[2][4] = {};
    int S[4] = {}, kchunk[4] = {}, S_cap[4] = {};
    float* recs = nullptr;                       // packed per-sample loss inputs (BF16 update)
    float* gb[2][4] = {};
    int mtiles = 0;
    int gb_parts = 0;            // bias-gradient partials per row tile (4 TMEM lane quarters in bf16)
    float* head_part = nullptr;
    int head_blocks = 0;
    AdamParams adam;
    // the same step split in three, so that most of it leaves the update's critical path: early
    // (every parameter but W_0, b_0 and W_1: its gradients exist once dW_1 is in flight, and the
    // last input gradient no longer reads it), mid (W_1, once the last input gradient, which reads
    // W_1, has run) and late (W_0, b_0, after the last weight gradient dW_0)
    AdamParams adam_early, adam_mid, adam_late;
    cudaStream_t aside = nullptr;
    // persistent GEMM CTAs at most (0: one per SM); grouped learners share the SMs in proportion
    // to their robots
    int gemm_cap = 0;
    cudaEvent_t ev_early_fork = nullptr, ev_mid_fork = nullptr, ev_early_join = nullptr;
    // bf16 weights and tensor maps
    void* wbf[2][4] = {};
    int bn_fwd[4], bn_dx[4], bn_dw[4], bn_act[4];
    // cluster mode per site: 1 single CTA, 3 pairs of CTAs running one 256-row tile on the
    // cta_group::2 MMA (half of B each), 4 single CTA with two K blocks per pipeline stage
    int cm_fwd[4], cm_dx[4], cm_dw[4], cm_act[4];
    // the three hidden layers' forward as one fused launch (mlp_fused.cu): the update's (fwd) and
    // the rollout's (act); set by the autotuner or rl_set_forward_fused
    bool fuse_fwd = false, fuse_act = false;
    CUtensorMap tm_fwdB[2][4], tm_fwdA[2][4];   // A for l >= 1 (H of layer l-1), A for l == 0 unused
    CUtensorMap tm_actB[2][4];                   // forward B maps of the rollout's policy inference
    CUtensorMap tm_x0;                           // gathered minibatch observations
    CUtensorMap tm_dxA[2][4], tm_dxB[2][4];
    CUtensorMap tm_dwA[2][4], tm_dwB[2][4];
    // layer 0's weight-gradient B operand (the gathered observations) for each of the two
    // observation buffers, one- and two-block stage forms: [buffer][net]
    CUtensorMap tm_dwB_x0[2][2], tm_dwB2_x0[2][2];
    // the same operands for two-K-block stages (single-CTA tiles of width <= 128)
    CUtensorMap tm_fwdB2[2][4], tm_actB2[2][4], tm_fwdA2[2][4];
    CUtensorMap tm_dxA2[2][4], tm_dxB2[2][4], tm_dwA2[2][4], tm_dwB2[2][4];
    // graph / profiling
    cudaStream_t gstream = nullptr;              // capture / replay stream (never the legacy stream)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int launches = 0;
    unsigned prof_mask = 0;                      // recorded kernel classes (bit RL_PROF_*)
    std::vector<int> ev_cls;                     // class of each recorded event pair
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    float prof_ms = 0.f;
    int prof_n = 0;
};

namespace {

#define CK(x)                                     \
    do {                                          \
        cudaError_t e_ = (x);                     \
        if (e_ != cudaSuccess) return err_of(e_); \
    } while (0)

rl_status err_of(cudaError_t e) {
    if (e == cudaSuccess) return RL_OK;
    if (e == cudaErrorMemoryAllocation) return RL_ERR_OOM;
    if (e == cudaErrorInvalidValue) return RL_ERR_INVALID_ARG;
    return RL_ERR_CUDA;
}

template <class T>
cudaError_t dalloc(rl_ctx* c, T** p, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes < 16 ? 16 : bytes);
    if (e != cudaSuccess) return e;
    c->allocs.push_back(q);
    e = cudaMemset(q, 0, bytes < 16 ? 16 : bytes);
    *p = reinterpret_cast<T*>(q);
    return e;
}

size_t esize(const rl_ctx* c) { return c->bf16 ? 2 : 4; }

bool config_ok(const rl_config* g) {
    if (!g) return false;
    if (g->num_envs < 1 || g->num_steps < 1 || g->act_dim != 12) return false;
    if (g->grid_x < 0 || g->grid_y < 0 || g->obs_dim != 48 + g->grid_x * g->grid_y) return false;
    if (g->obs_pad < g->obs_dim || g->obs_pad % 64) return false;
    if (g->num_hidden < 1 || g->num_hidden > 4) return false;
    for (int i = 0; i < g->num_hidden; ++i)
        if (g->hidden[i] < 64 || g->hidden[i] % 64 || g->hidden[i] > 1024) return false;
    const int hl = g->hidden[g->num_hidden - 1];
    if (hl != 64 && hl != 128 && hl != 256) return false;
    if (g->epochs < 1 || g->minibatches < 1) return false;
    const long long B = (long long)g->num_envs * g->num_steps;
    if (B % g->minibatches || (B / g->minibatches) % 64) return false;
    if (B > (1ll << 30)) return false;
    if (g->precision != RL_FP32 && g->precision != RL_BF16) return false;
    if (g->decimation < 1 || g->max_episode_len < 1 || g->num_levels < 1 || g->num_cols < 1) return false;
    if (!(g->hf_res > 0.f) || !(g->tile_size > 0.f)) return false;
    const double cpt = (double)g->tile_size / (double)g->hf_res;
    const long long icpt = llround(cpt);
    if (std::fabs(cpt - (double)icpt) > 1e-4 || icpt < 2 || icpt % 2) return false;
    if (g->push_on && g->push_interval < 1) return false;
    return true;
}

// Host-side launch bookkeeping: the launch counter and, for the recorded kernel classes, CUDA
// events around each launch.
struct Enq {
    rl_ctx* c;
    cudaStream_t s;
    bool profile;
    template <class F>
    cudaError_t run(int cls, int nlaunch, F&& launch) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (profile && ((c->prof_mask >> cls) & 1u) && c->ev_used + 2 <= c->ev.size()) {
            e0 = c->ev[c->ev_used];
            e1 = c->ev[c->ev_used + 1];
            c->ev_cls[c->ev_used / 2] = cls;
            c->ev_used += 2;
            cudaError_t e = cudaEventRecordWithFlags(e0, s, cudaEventRecordExternal);
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = launch();
        c->launches += nlaunch;
        if (e == cudaSuccess && e1) e = cudaEventRecordWithFlags(e1, s, cudaEventRecordExternal);
        return e;
    }
    cudaError_t gemm(const TcParams* tp, int epi, bool a_t, bool b_t, int M, int N, int K, int lda, int ldb, int ldc,
                     int ldh, int batch, int splits, int kchunk, const GemmBatch* g) {
        return run(RL_PROF_GEMM, 1, [&] {
            return tp ? launch_tc_gemm(*tp, s)
                      : launch_gemm_f32(epi, a_t, b_t, M, N, K, lda, ldb, ldc, ldh, batch, splits, kchunk, *g, s);
        });
    }
};

// Tile modes of a GEMM site: 1 one CTA per tile, 3 pairs of CTAs on one 256-row tile
// (cta_group::2), 4 one CTA per tile with two K blocks per pipeline stage (bn <= 128), 5
// weight-stationary (forward and input-gradient sites: each CTA keeps one column tile of the
// weights in shared memory and streams its row tiles' activations, two K blocks per stage).
// (Mode 2, pairs of row tiles sharing the B tile by TMA multicast, is not offered.)
// B rows one CTA loads per K step for a K-major B (tile width bn, mode cm)
uint32_t b_rows(int bn, int cm) { return (uint32_t)(cm == 3 ? bn / 2 : bn); }
void set_cluster(TcParams& tp, int cm) {
    tp.cm = cm == 3 ? 2 : 1;
    tp.pair = cm == 3 ? 1 : 0;
    tp.ks = (cm == 4 || cm == 7) ? 2 : 1;
    tp.ws = cm == 5 ? 1 : 0;
}
// two-K-block stages of both operands (modes 4, 7); of the A operand (modes 4, 5, 7)
bool two_block(int cm) { return cm == 4 || cm == 7; }
bool a_two_block(int cm) { return cm == 4 || cm == 5 || cm == 7; }

// Cluster size of the in-GEMM split-K reduction of hidden layer l's weight gradient (modes 6, 7):
// the largest d in 2 .. 8 dividing the split count (one CTA per tile and split, so only when the
// learner's GEMMs are uncapped or the launch fits its cap); 0: every split's partial goes to Adam.
int split_cluster(const rl_ctx* c, int l) {
    if (!c->bf16 || (c->cm_dw[l] != 6 && c->cm_dw[l] != 7)) return 0;
    const LayerInfo& Li = c->L[0][l];
    const long long tiles = (long long)((Li.out + 127) / 128) * (Li.in / c->bn_dw[l]) * 2;
    if (c->gemm_cap > 0 && tiles * c->S[l] > c->gemm_cap) return 0;
    for (int d = 8; d >= 2; --d)
        if (c->S[l] % d == 0) return d;
    return 0;
}
// Partials of layer l's weight gradient that Adam sums.
int weight_partials(const rl_ctx* c, int l) {
    const int d = split_cluster(c, l);
    return d ? c->S[l] / d : c->S[l];
}
// Weight-gradient sites also take modes 6 and 7: modes 1 and 4 with the split-K partials reduced
// inside the GEMM by clusters of CTAs (see split_cluster).
// weight-stationary mode 5 fits a site: a ring stage beside the resident weight slice, and no
// more (network, column tile) groups than SMs
bool ws_fits(int bn, int epi, int kblocks, int width) {
    return tc_ws_stages(bn, epi, kblocks) >= 1 && 2 * (width / bn) <= 148;
}

int pick_bn(int n) {
    if (n % 128 == 0) return 128;
    return 64;
}

// TMA descriptors of layer l (both networks) for the current tile widths.
bool encode_layer_maps(rl_ctx* c, int l) {
    bool ok = true;
    for (int n = 0; n < 2; ++n) {
        const LayerInfo& Li = c->L[n][l];
        // two-K-block stage maps of the sites whose tile shape uses them
        if (two_block(c->cm_fwd[l]))
            ok = ok && make_tmap_bf16_k2(&c->tm_fwdB2[n][l], c->wbf[n][l], Li.out, Li.in, Li.in, (uint32_t)c->bn_fwd[l]);
        if (two_block(c->cm_act[l]))
            ok = ok && make_tmap_bf16_k2(&c->tm_actB2[n][l], c->wbf[n][l], Li.out, Li.in, Li.in, (uint32_t)c->bn_act[l]);
        if (l > 0) ok = ok && make_tmap_bf16_k2(&c->tm_fwdA2[n][l], c->H[n][l - 1], c->rows, Li.in, Li.in, 128);
        if (l > 0 && a_two_block(c->cm_dx[l]))
            ok = ok && make_tmap_bf16_k2(&c->tm_dxA2[n][l], c->dY[n][l], c->Mb, Li.out, Li.out, 128);
        if (l > 0 && two_block(c->cm_dx[l]))
            ok = ok && make_tmap_bf16_mn2(&c->tm_dxB2[n][l], c->wbf[n][l], Li.out, Li.in, Li.in, (uint32_t)c->bn_dx[l]);
        if (two_block(c->cm_dw[l])) {
            const void* xb2 = l == 0 ? c->X0 : c->H[n][l - 1];
            ok = ok && make_tmap_bf16_mn2(&c->tm_dwA2[n][l], c->dY[n][l], c->Mb, Li.out, Li.out, 128);
            ok = ok && make_tmap_bf16_mn2(&c->tm_dwB2[n][l], xb2, c->Mb, Li.in, Li.in, (uint32_t)c->bn_dw[l]);
            if (l == 0)
                for (int x = 0; x < 2; ++x)
                    ok = ok && make_tmap_bf16_mn2(&c->tm_dwB2_x0[x][n], c->X0buf[x], c->Mb, Li.in, Li.in, (uint32_t)c->bn_dw[l]);
        }
        ok = ok && make_tmap_bf16(&c->tm_fwdB[n][l], c->wbf[n][l], Li.out, Li.in, Li.in, b_rows(c->bn_fwd[l], c->cm_fwd[l]));
        ok = ok && make_tmap_bf16(&c->tm_actB[n][l], c->wbf[n][l], Li.out, Li.in, Li.in, b_rows(c->bn_act[l], c->cm_act[l]));
        if (l > 0) ok = ok && make_tmap_bf16(&c->tm_fwdA[n][l], c->H[n][l - 1], c->rows, Li.in, Li.in, 128);
        else c->tm_fwdA[n][l] = c->tm_x0;
        if (l > 0) {
            ok = ok && make_tmap_bf16(&c->tm_dxA[n][l], c->dY[n][l], c->Mb, Li.out, Li.out, 128);
            // input gradient, B read MN-major: W_l [out][in] as it is stored; one 3D copy per stage
            // in single-CTA mode, 64 x 64 boxes otherwise
            ok = ok && ((c->cm_dx[l] == 1 || c->cm_dx[l] == 5)
                            ? make_tmap_bf16_mn1(&c->tm_dxB[n][l], c->wbf[n][l], Li.out, Li.in, Li.in, (uint32_t)c->bn_dx[l])
                                         : make_tmap_bf16(&c->tm_dxB[n][l], c->wbf[n][l], Li.out, Li.in, Li.in, 64));
        }
        // weight gradient, MN-major operands: dY_l [rows][out] and H_{l-1} [rows][in]; one 3D copy per
        // operand and stage in single-CTA mode, 64 x 64 boxes otherwise
        const bool dw3 = c->cm_dw[l] == 1 || c->cm_dw[l] == 6;
        auto dw_map = [&](CUtensorMap* m, const void* base, int cols, int tile) {
            return dw3 ? make_tmap_bf16_mn1(m, base, c->Mb, cols, cols, (uint32_t)tile) : make_tmap_bf16(m, base, c->Mb, cols, cols, 64);
        };
        ok = ok && dw_map(&c->tm_dwA[n][l], c->dY[n][l], Li.out, 128);
        const void* xb = l == 0 ? c->X0 : c->H[n][l - 1];
        ok = ok && dw_map(&c->tm_dwB[n][l], xb, Li.in, c->bn_dw[l]);
        if (l == 0)
            for (int x = 0; x < 2; ++x) ok = ok && dw_map(&c->tm_dwB_x0[x][n], c->X0buf[x], Li.in, c->bn_dw[l]);
    }
    return ok;
}

// One hidden layer of the forward pass for `rows` rows (X = layer-0 input), batch = nnets
// networks starting at net0: 2 (actor + critic) or 1 with net0 = 1 (critic only).  act: the
// rollout's policy inference (its own tile shapes, tuned for num_envs rows), else the update.
// b_early: no kernel still running when this one starts writes the weights (the rollout's steps
// after the first, the last value), so a weight-stationary launch fetches its weight slice before
// it waits for the preceding kernel.
rl_status fwd_layer(rl_ctx* c, Enq& q, int l, const void* X, int rows, int net0, int nnets, bool act, bool b_early = false) {
    const LayerInfo& Li = c->L[0][l];
    if (c->bf16) {
        TcParams tp;
        std::memset(&tp, 0, sizeof(tp));
        const int bn = act ? c->bn_act[l] : c->bn_fwd[l], cm = act ? c->cm_act[l] : c->cm_fwd[l];
        const bool k2 = two_block(cm), ak2 = a_two_block(cm);
        for (int j = 0; j < nnets; ++j) {
            const int n = net0 + j;
            if (l == 0) {
                const bool mk = ak2 ? make_tmap_bf16_k2(&tp.tmA[j], X, (uint64_t)rows, (uint64_t)Li.in, (uint64_t)Li.in, 128)
                                   : make_tmap_bf16(&tp.tmA[j], X, (uint64_t)rows, (uint64_t)Li.in, (uint64_t)Li.in, 128);
                if (!mk) return RL_ERR_CUDA;
            } else {
                tp.tmA[j] = ak2 ? c->tm_fwdA2[n][l] : c->tm_fwdA[n][l];
            }
            if (k2) tp.tmB[j] = act ? c->tm_actB2[n][l] : c->tm_fwdB2[n][l];
            else tp.tmB[j] = act ? c->tm_actB[n][l] : c->tm_fwdB[n][l];
            if (!make_tmap_out(&tp.tmC[j], c->H[n][l], false, 1, (uint64_t)rows, (uint64_t)Li.out, (uint64_t)Li.out, 0))
                return RL_ERR_CUDA;
            tp.bias[j] = c->params + c->L[n][l].b;
        }
        tp.M = rows;
        tp.N = Li.out;
        tp.kblocks = Li.in / 64;
        tp.kb_per_split = tp.kblocks;
        tp.splits = 1;
        tp.batch = nnets;
        tp.bn = bn;
        set_cluster(tp, cm);
        tp.epi = EPI_BIAS_ELU;
        tp.b_early = (b_early && tp.ws) ? 1 : 0;
        tp.status = c->status;
        tp.max_ctas = c->gemm_cap;
        CK(q.gemm(&tp, 0, false, false, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, nullptr));
    } else {
        GemmBatch g;
        std::memset(&g, 0, sizeof(g));
        for (int j = 0; j < nnets; ++j) {
            const int n = net0 + j;
            g.A[j] = l == 0 ? reinterpret_cast<const float*>(X) : reinterpret_cast<const float*>(c->H[n][l - 1]);
            g.B[j] = c->params + c->L[n][l].w;
            g.C[j] = reinterpret_cast<float*>(c->H[n][l]);
            g.bias[j] = c->params + c->L[n][l].b;
        }
        CK(q.gemm(nullptr, EPI_BIAS_ELU, false, false, rows, Li.out, Li.in, Li.in, Li.in, Li.out, 0, nnets, 1, Li.in, &g));
    }
    return RL_OK;
}

// The fused forward fits the context: BF16, three hidden layers of the widths mlp_fwd_fits takes.
bool fused_fits(const rl_ctx* c) {
    return c->bf16 && c->NH == 3 && mlp_fwd_fits(c->L[0][0].in, c->L[0][0].out, c->L[0][1].out, c->L[0][2].out);
}
// The site's forward runs fused: chosen, fitting, and the context's GEMM CTAs uncapped (the fused
// launch takes one CTA per row tile and network, so it cannot keep to a learner's share of the SMs).
bool fused_on(const rl_ctx* c, bool act) { return (act ? c->fuse_act : c->fuse_fwd) && fused_fits(c) && c->gemm_cap == 0; }

// The three hidden layers in one launch (mlp_fused.cu): every layer's rows are kept for the
// update's backward, only the last layer's for the rollout.
rl_status forward_fused(rl_ctx* c, Enq& q, const void* X, int rows, int net0, int nnets, bool act, bool b_early) {
    MlpParams mp;
    std::memset(&mp, 0, sizeof(mp));
    const LayerInfo* L0 = c->L[0];
    if (!make_tmap_bf16(&mp.tmX, X, (uint64_t)rows, (uint64_t)L0[0].in, (uint64_t)L0[0].in, 128)) return RL_ERR_CUDA;
    for (int j = 0; j < nnets; ++j) {
        const int n = net0 + j;
        for (int l = 0; l < 3; ++l) {
            const LayerInfo& Li = c->L[n][l];
            if (!make_tmap_bf16(&mp.tmW[j][l], c->wbf[n][l], (uint64_t)Li.out, (uint64_t)Li.in, (uint64_t)Li.in, 128))
                return RL_ERR_CUDA;
            if ((!act || l == 2) &&
                !make_tmap_bf16(&mp.tmH[j][l], c->H[n][l], (uint64_t)rows, (uint64_t)Li.out, (uint64_t)Li.out, 128))
                return RL_ERR_CUDA;
            mp.bias[j][l] = c->params + Li.b;
        }
    }
    mp.M = rows;
    mp.K0 = L0[0].in;
    mp.N0 = L0[0].out;
    mp.N1 = L0[1].out;
    mp.N2 = L0[2].out;
    mp.nnets = nnets;
    mp.store_hidden = act ? 0 : 1;
    mp.b_early = b_early ? 1 : 0;
    mp.status = c->status;
    CK(q.run(RL_PROF_GEMM, 1, [&] { return launch_mlp_fwd(mp, q.s); }));
    return RL_OK;
}

// Forward through every hidden layer.
rl_status forward_hidden(rl_ctx* c, Enq& q, const void* X, int rows, int net0, int nnets, bool act, bool b_early = false) {
    if (fused_on(c, act)) return forward_fused(c, q, X, rows, net0, nnets, act, b_early);
    for (int l = 0; l < c->NH; ++l) {
        rl_status st = fwd_layer(c, q, l, X, rows, net0, nnets, act, b_early);
        if (st != RL_OK) return st;
    }
    return RL_OK;
}

// Input gradient of hidden layer k >= 1 for M minibatch rows (actor and critic in one launch).
rl_status dx_layer(rl_ctx* c, Enq& q, int k, int M) {
    const LayerInfo& Li = c->L[0][k];   // in = hid[k-1], out = hid[k]
    if (c->bf16) {
        TcParams tp;
        std::memset(&tp, 0, sizeof(tp));
        const bool k2 = two_block(c->cm_dx[k]);
        for (int n = 0; n < 2; ++n) {
            tp.tmA[n] = a_two_block(c->cm_dx[k]) ? c->tm_dxA2[n][k] : c->tm_dxA[n][k];
            tp.tmB[n] = k2 ? c->tm_dxB2[n][k] : c->tm_dxB[n][k];
            if (!make_tmap_out(&tp.tmC[n], c->dY[n][k - 1], false, 1, (uint64_t)M, (uint64_t)Li.in, (uint64_t)Li.in, 0))
                return RL_ERR_CUDA;
            tp.hsrc[n] = c->H[n][k - 1];
            tp.colsum[n] = c->gb[n][k - 1];
        }
        tp.M = M; tp.N = Li.in; tp.ldh = Li.in; tp.kblocks = Li.out / 64; tp.kb_per_split = tp.kblocks; tp.splits = 1;
        tp.batch = 2; tp.bn = c->bn_dx[k]; set_cluster(tp, c->cm_dx[k]); tp.mn = MAJ_B_MN; tp.epi = EPI_ELU_GRAD;
        tp.mn3 = (c->cm_dx[k] == 1 || c->cm_dx[k] == 5) ? 1 : 0;       // the maps of encode_layer_maps
        tp.status = c->status;
        tp.max_ctas = c->gemm_cap;
        CK(q.gemm(&tp, 0, false, false, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, nullptr));
    } else {
        GemmBatch g;
        std::memset(&g, 0, sizeof(g));
        for (int n = 0; n < 2; ++n) {
            g.A[n] = reinterpret_cast<const float*>(c->dY[n][k]);
            g.B[n] = c->params + c->L[n][k].w;
            g.C[n] = reinterpret_cast<float*>(c->dY[n][k - 1]);
            g.H[n] = reinterpret_cast<const float*>(c->H[n][k - 1]);
            g.colsum[n] = c->gb[n][k - 1];
        }
        CK(q.gemm(nullptr, EPI_ELU_GRAD, false, true, M, Li.in, Li.out, Li.out, Li.in, Li.in, Li.in, 2, 1, Li.out, &g));
    }
    return RL_OK;
}

// Weight gradient of hidden layer k, split over the minibatch rows.
rl_status dw_layer(rl_ctx* c, Enq& q, int k, int M) {
    const LayerInfo& Li = c->L[0][k];
    if (c->bf16) {
        TcParams tp;
        std::memset(&tp, 0, sizeof(tp));
        const bool k2 = two_block(c->cm_dw[k]);
        for (int n = 0; n < 2; ++n) {
            tp.tmA[n] = k2 ? c->tm_dwA2[n][k] : c->tm_dwA[n][k];
            if (k == 0) tp.tmB[n] = k2 ? c->tm_dwB2_x0[c->xcur][n] : c->tm_dwB_x0[c->xcur][n];
            else tp.tmB[n] = k2 ? c->tm_dwB2[n][k] : c->tm_dwB[n][k];
            if (!make_tmap_out(&tp.tmC[n], c->gw[n][k], true, (uint64_t)c->S[k], (uint64_t)Li.out, (uint64_t)Li.in, (uint64_t)Li.in,
                               (uint64_t)Li.out * Li.in))
                return RL_ERR_CUDA;
        }
        tp.M = Li.out; tp.N = Li.in; tp.kblocks = (M + 63) / 64; tp.kb_per_split = c->kchunk[k] / 64;
        tp.splits = c->S[k]; tp.batch = 2; tp.bn = c->bn_dw[k]; set_cluster(tp, c->cm_dw[k]); tp.mn = MAJ_MN; tp.epi = EPI_STORE;
        tp.mn3 = (c->cm_dw[k] == 1 || c->cm_dw[k] == 6) ? 1 : 0;       // the maps of encode_layer_maps
        tp.sred = split_cluster(c, k);
        for (int n = 0; n < 2; ++n) tp.sr_out[n] = c->gw[n][k];
        tp.sr_ld = Li.in;
        tp.sr_split_ld = (long long)Li.out * Li.in;
        tp.status = c->status;
        tp.max_ctas = c->gemm_cap;
        CK(q.gemm(&tp, 0, false, false, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, nullptr));
    } else {
        GemmBatch g;
        std::memset(&g, 0, sizeof(g));
        for (int n = 0; n < 2; ++n) {
            g.A[n] = reinterpret_cast<const float*>(c->dY[n][k]);
            g.B[n] = k == 0 ? reinterpret_cast<const float*>(c->X0) : reinterpret_cast<const float*>(c->H[n][k - 1]);
            g.C[n] = c->gw[n][k];
        }
        g.split_stride = (long long)Li.out * Li.in;
        CK(q.gemm(nullptr, EPI_STORE, true, true, Li.out, Li.in, M, Li.out, Li.in, Li.in, 0, 2, c->S[k], c->kchunk[k], &g));
    }
    return RL_OK;
}

HeadParams head_common(rl_ctx* c, int rows) {
    HeadParams h;
    std::memset(&h, 0, sizeof(h));
    const int l = c->NH - 1;
    h.M = rows;
    h.H = c->HL;
    h.A = c->A;
    h.bf16 = c->bf16 ? 1 : 0;
    h.ha = c->H[0][l];
    h.hc = c->H[1][l];
    h.Wa = c->params + c->L[0][c->NH].w;
    h.ba = c->params + c->L[0][c->NH].b;
    h.log_std = c->params + c->logstd;
    h.Wc = c->params + c->L[1][c->NH].w;
    h.bc = c->params + c->L[1][c->NH].b;
    h.seed = c->cfg.seed;
    h.iteration = c->iter;
    return h;
}

rl_status act_impl(rl_ctx* c, Enq& q, int t, int n, const void* obs, float* actions, float* mu, float* logp,
                   float* values, bool b_early = false) {
    const bool critic_only = !actions && !mu && !logp;
    rl_status st = forward_hidden(c, q, obs, n, critic_only ? 1 : 0, critic_only ? 1 : 2, true, b_early);
    if (st != RL_OK) return st;
    HeadParams h = head_common(c, n);
    h.t = t;
    h.actions = actions;
    h.mu = mu;
    h.logp = logp;
    h.values = values;
    CK(q.run(RL_PROF_ACT, 1, [&] { return launch_act_head(h, q.s); }));
    return RL_OK;
}

EnvParams env_params(rl_ctx* c) {
    EnvParams p;
    std::memset(&p, 0, sizeof(p));
    const rl_config& g = c->cfg;
    p.N = c->N; p.O = c->O; p.Op = c->Op; p.GX = g.grid_x; p.GY = g.grid_y; p.decimation = g.decimation;
    p.max_ep = g.max_episode_len; p.L = g.num_levels; p.C = g.num_cols; p.cpt = c->cpt; p.nx = c->nx; p.ny = c->ny;
    p.push_interval = g.push_interval > 0 ? g.push_interval : 1; p.noise_on = g.noise_on; p.push_on = g.push_on;
    p.randomize_eplen = 1;
    p.kp = g.kp; p.kd = g.kd; p.ascale = g.action_scale; p.dt = g.dt; p.sim_dt = g.sim_dt; p.gamma = g.gamma;
    p.push_vel = g.push_vel; p.grid_sp = g.grid_spacing; p.inv_res = 1.0f / g.hf_res; p.tile = g.tile_size;
    for (int i = 0; i < 3; ++i) p.cmd_range[i] = g.cmd_range[i];
    for (int i = 0; i < 12; ++i) p.q_def[i] = g.q_def[i];
    p.crash_thr = g.crash_threshold;
    p.seed = g.seed;
    p.hf = c->hf;
    p.sf = c->sf;
    p.si = c->si;
    p.iteration = c->iter;
    p.obs_bf16 = c->bf16 ? 1 : 0;
    return p;
}

// One minibatch: forward, loss head (+ Algorithm 1 when kl_target > 0), backward.
// X0 must already hold the minibatch observations.
rl_status minibatch_fwd_bwd(rl_ctx* c, Enq& q, int M, const int* idx, const float* a_old, const float* logp_old,
                            const float* mu_old, const float* log_std_old, const float* v_old, const float* adv,
                            const float* ret, float clip, bool step, const float* rec = nullptr, bool overlap_dw = false,
                            cudaEvent_t before_loss = nullptr, float* trace = nullptr) {
    rl_status st = forward_hidden(c, q, c->X0, M, 0, 2, false);
    if (st != RL_OK) return st;
    HeadParams h = head_common(c, M);
    const int l = c->NH - 1;
    h.idx = idx;
    h.rec = rec;
    h.rec_ld = REC_LD;
    h.a_old = a_old;
    h.logp_old = logp_old;
    h.mu_old = mu_old;
    h.log_std_old = log_std_old;
    h.v_old = v_old;
    h.adv = adv;
    h.ret = ret;
    h.clip = clip;
    h.trace = trace;
    h.value_coef = c->cfg.value_coef;
    h.entropy_coef = c->cfg.entropy_coef;
    h.dya = c->dY[0][l];
    h.dyc = c->dY[1][l];
    h.part = c->head_part;
    h.nblocks = c->head_blocks;
    h.scal = c->scal;
    h.stats = step ? c->acc : nullptr;
    h.kl_target = step ? c->cfg.kl_target : 0.f;
    h.lr_min = c->cfg.lr_min;
    h.lr_max = c->cfg.lr_max;
    if (before_loss) CK(cudaStreamWaitEvent(q.s, before_loss, 0));
    CK(q.run(RL_PROF_LOSS, 1, [&] { return launch_loss_head(h, q.s); }));
    // the minibatch statistics and Algorithm 1 (read only by Adam): on the weight-gradient stream
    // beside the first input gradient when the streams overlap, else right here
    if (!overlap_dw) CK(q.run(RL_PROF_LOSS, 1, [&] { return launch_loss_stats(h, q.s); }));
    // input gradients: dY_{l-1} = (dY_l W_l) * ELU'(H_{l-1}), plus the bias-gradient column sums;
    // weight gradients: dW_l = dY_l^T H_{l-1}, split over the minibatch rows.  dW_l needs only dY_l,
    // so with overlap_dw it runs on a second stream as soon as dY_l exists, beside the next input
    // gradient (the two persistent grids fill each other's ramp and tail), and the main stream
    // joins it before returning.  The results are the same either way.
    Enq qw{c, c->wside, q.profile};
    auto fork_dw = [&](int k) -> rl_status {
        CK(cudaEventRecord(c->ev_dw[k], q.s));
        CK(cudaStreamWaitEvent(c->wside, c->ev_dw[k], 0));
        if (k == c->NH - 1) {
            CK(launch_loss_stats(h, c->wside));
            ++c->launches;
        }
        rl_status r = dw_layer(c, qw, k, M);
        if (r != RL_OK || k != 1 || !step) return r;
        // every gradient but the first hidden layer's is now in flight or done: the early part of
        // Adam on its own stream, after this weight gradient and beside the last ones
        CK(cudaEventRecord(c->ev_early_fork, c->wside));
        CK(cudaStreamWaitEvent(c->aside, c->ev_early_fork, 0));
        c->adam_early.grad_out = nullptr;
        CK(launch_adam(c->adam_early, c->aside));
        ++c->launches;
        return RL_OK;
    };
    if (overlap_dw) {
        st = fork_dw(c->NH - 1);
        if (st != RL_OK) return st;
    }
    for (int k = c->NH - 1; k >= 1; --k) {
        st = dx_layer(c, q, k, M);
        if (st != RL_OK) return st;
        if (overlap_dw && step && k == 1) {
            // the last input gradient has read W_1: the mid part of Adam (W_1) after it, on the
            // early part's stream, beside dW_0
            CK(cudaEventRecord(c->ev_mid_fork, q.s));
            CK(cudaStreamWaitEvent(c->aside, c->ev_mid_fork, 0));
            c->adam_mid.grad_out = nullptr;
            CK(launch_adam(c->adam_mid, c->aside));
            ++c->launches;
            CK(cudaEventRecord(c->ev_early_join, c->aside));
        }
        if (overlap_dw) {
            st = fork_dw(k - 1);
            if (st != RL_OK) return st;
        }
    }
    if (overlap_dw) {
        CK(cudaEventRecord(c->ev_dw_join, c->wside));
        CK(cudaStreamWaitEvent(q.s, c->ev_dw_join, 0));
    } else {
        for (int k = 0; k < c->NH; ++k) {
            st = dw_layer(c, q, k, M);
            if (st != RL_OK) return st;
        }
    }
    return RL_OK;
}

// Builds the Adam segment table (gradient partial sources of every parameter tensor).
void build_adam(rl_ctx* c) {
    AdamParams& a = c->adam;
    std::memset(&a, 0, sizeof(a));
    a.p = c->params;
    a.m = c->am;
    a.v = c->av;
    a.scal = c->scal;
    const HeadPart hp = head_part(c->A, c->HL);
    const int PF = hp.PF, O_WA = hp.WA, O_BA = hp.BA, O_LS = hp.LS, O_WC = hp.WC, O_BC = hp.BC, O_DBA = hp.DBA,
              O_DBC = hp.DBC;
    int ns = 0, blocks = 0;
    // two passes: the segments with many partials (a warp per parameter group, the slowest blocks)
    // first, so that their blocks start in the first wave and the quick ones fill in behind them;
    // the order of the blocks changes no sum
    int pass = 0;
    auto add = [&](long long off, long long size, const float* part, long long stride, int nsplit, void* wbf, int rows,
                   int cols) {
        if ((nsplit > ADAM_WIDE) != (pass == 0)) return;
        AdamSeg& s = a.seg[ns];
        s.offset = off;
        s.size = size;
        s.partials = part;
        s.stride = stride;
        s.nsplit = nsplit;
        s.block_start = blocks;
        a.wbf[ns] = wbf;
        (void)rows;
        (void)cols;
        s.vec = (off % 4 == 0 && size % 4 == 0 && stride % 4 == 0 && (reinterpret_cast<uintptr_t>(part) & 15u) == 0 &&
                 (reinterpret_cast<uintptr_t>(wbf) & 7u) == 0)
                    ? 1
                    : 0;
        const long long per_block = adam_per_block(nsplit, s.vec);
        blocks += (int)((size + per_block - 1) / per_block);
        ++ns;
    };
    for (pass = 0; pass < 2; ++pass) {
        for (int n = 0; n < 2; ++n) {
            for (int l = 0; l < c->NH; ++l) {
                const LayerInfo& Li = c->L[n][l];
                add(Li.w, (long long)Li.out * Li.in, c->gw[n][l], (long long)Li.out * Li.in, weight_partials(c, l), c->wbf[n][l],
                    Li.out, Li.in);
                if (l < c->NH - 1)
                    add(Li.b, Li.out, c->gb[n][l], Li.out, c->gb_parts, nullptr, 0, 0);
                else
                    add(Li.b, Li.out, c->head_part + (n == 0 ? O_DBA : O_DBC), PF, c->head_blocks, nullptr, 0, 0);
            }
            const LayerInfo& Lh = c->L[n][c->NH];
            add(Lh.w, (long long)Lh.out * Lh.in, c->head_part + (n == 0 ? O_WA : O_WC), PF, c->head_blocks, nullptr, 0, 0);
            add(Lh.b, Lh.out, c->head_part + (n == 0 ? O_BA : O_BC), PF, c->head_blocks, nullptr, 0, 0);
            if (n == 0) add(c->logstd, c->A, c->head_part + O_LS, PF, c->head_blocks, nullptr, 0, 0);
        }
    }
    a.nsegs = ns;
    a.nblocks = blocks;
    // the early / mid / late parts: the segments keep their order and partial sources, with their
    // blocks renumbered per part
    AdamParams* part[3] = {&c->adam_early, &c->adam_mid, &c->adam_late};
    auto part_of = [&](long long off) {
        for (int n = 0; n < 2; ++n) {
            if (off == c->L[n][0].w || off == c->L[n][0].b) return 2;
            if (c->NH >= 2 && off == c->L[n][1].w) return 1;
        }
        return 0;
    };
    for (int h = 0; h < 3; ++h) {
        AdamParams& d = *part[h];
        d = a;
        d.nsegs = 0;
        d.nblocks = 0;
        for (int k = 0; k < a.nsegs; ++k) {
            if (part_of(a.seg[k].offset) != h) continue;
            AdamSeg sg = a.seg[k];
            sg.block_start = d.nblocks;
            d.nblocks += (int)((sg.size + adam_per_block(sg.nsplit, sg.vec) - 1) / adam_per_block(sg.nsplit, sg.vec));
            d.wbf[d.nsegs] = a.wbf[k];
            d.seg[d.nsegs++] = sg;
        }
    }
}

// Adam's partial-sum pass restricted to the weight matrices of hidden layer l (both networks),
// writing the summed gradient to the scratch gradient instead of stepping: the autotuner times
// it with the weight-gradient GEMM, since the split count trades GEMM parallelism for the
// partial-sum traffic.
AdamParams weight_reduce_params(rl_ctx* c, int l) {
    AdamParams a;
    std::memset(&a, 0, sizeof(a));
    a.p = c->params;
    a.m = c->am;
    a.v = c->av;
    a.grad_out = c->grad_int;
    int blocks = 0;
    for (int n = 0; n < 2; ++n) {
        const LayerInfo& Li = c->L[n][l];
        AdamSeg& sg = a.seg[a.nsegs];
        sg.offset = Li.w;
        sg.size = (long long)Li.out * Li.in;
        sg.partials = c->gw[n][l];
        sg.stride = sg.size;
        sg.nsplit = weight_partials(c, l);
        sg.block_start = blocks;
        sg.vec = (sg.offset % 4 == 0 && sg.size % 4 == 0) ? 1 : 0;
        const long long per_block = adam_per_block(sg.nsplit, sg.vec);
        blocks += (int)((sg.size + per_block - 1) / per_block);
        ++a.nsegs;
    }
    a.nblocks = blocks;
    return a;
}

rl_status refresh_bf16(rl_ctx* c, cudaStream_t s) {
    if (!c->bf16) return RL_OK;
    for (int n = 0; n < 2; ++n)
        for (int l = 0; l < c->NH; ++l) {
            const LayerInfo& Li = c->L[n][l];
            CK(launch_to_bf16(c->params + Li.w, Li.out, Li.in, c->wbf[n][l], s));
        }
    return RL_OK;
}

rl_status update_impl(rl_ctx* c, Enq& q, const void* obs, const float* actions, const float* logp_old, const float* mu_old,
                      const float* val_old, const float* adv, const float* ret, int epochs, int minibatches, float clip,
                      float* stats_out, bool perm_on_side) {
    const int B = c->B, Mb = B / minibatches;
    if (Mb != c->Mb || epochs > c->cfg.epochs) return RL_ERR_INVALID_ARG;
    cudaStream_t s = q.s;
    CK(cudaMemcpyAsync(c->logstd_old, c->params + c->logstd, sizeof(float) * c->A, cudaMemcpyDeviceToDevice, s));
    if (!perm_on_side)
        CK(q.run(RL_PROF_OTHER, 1, [&] { return launch_permutation(B, epochs, c->cfg.seed, c->iter, c->perm, c->status, s); }));
    // the BF16 loss head reads each row's loss inputs from one packed 128-byte record per sample
    // (one line per row of a shuffled minibatch instead of one per field); the records are packed
    // on the side stream, beside the first minibatch's gather and forward, when the shuffle ran there
    const bool pack_on_side = perm_on_side && c->bf16;
    if (pack_on_side) {
        CK(cudaEventRecord(c->ev_pack_fork, s));
        CK(cudaStreamWaitEvent(c->side, c->ev_pack_fork, 0));
        CK(launch_pack_records(B, c->A, actions, mu_old, logp_old, adv, val_old, ret, c->recs, c->side));
        ++c->launches;
        CK(cudaEventRecord(c->ev_pack_join, c->side));
    } else if (c->bf16) {
        CK(q.run(RL_PROF_OTHER, 1,
                 [&] { return launch_pack_records(B, c->A, actions, mu_old, logp_old, adv, val_old, ret, c->recs, s); }));
    }
    // The next minibatch's observations are gathered on a side stream into the other buffer
    // while the current minibatch trains (the gather is memory-bound, the GEMMs are not); the
    // forward of the next minibatch waits for it.  With per-class profiling every launch stays on
    // the main stream.
    const bool overlap = !q.profile;
    const int nmb = epochs * minibatches;
    auto mb_idx = [&](int k) { return c->perm + (size_t)(k / minibatches) * B + (size_t)(k % minibatches) * Mb; };
    c->xcur = 0;
    c->X0 = c->X0buf[0];
    if (perm_on_side) CK(cudaStreamWaitEvent(s, c->ev_perm_join, 0));
    CK(q.run(RL_PROF_GATHER, 1, [&] { return launch_gather(obs, c->bf16 ? 1 : 0, mb_idx(0), Mb, c->Op, c->X0buf[0], s); }));
    for (int k = 0; k < nmb; ++k) {
        const int cur = k & 1, nxt = cur ^ 1;
        c->xcur = cur;
        c->X0 = c->X0buf[cur];
        if (k > 0 && overlap) CK(cudaStreamWaitEvent(s, c->ev_join[cur], 0));   // this minibatch's gather
        if (k + 1 < nmb) {
            // the other buffer was last read by minibatch k - 1, already ordered before this point
            if (overlap) {
                CK(cudaEventRecord(c->ev_fork[nxt], s));
                CK(cudaStreamWaitEvent(c->side, c->ev_fork[nxt], 0));
                CK(launch_gather(obs, c->bf16 ? 1 : 0, mb_idx(k + 1), Mb, c->Op, c->X0buf[nxt], c->side));
                ++c->launches;
                CK(cudaEventRecord(c->ev_join[nxt], c->side));
            }
        }
        rl_status st = minibatch_fwd_bwd(c, q, Mb, mb_idx(k), actions, logp_old, mu_old, c->logstd_old, val_old, adv, ret, clip,
                                         true, c->bf16 ? c->recs : nullptr, overlap,
                                         k == 0 && pack_on_side ? c->ev_pack_join : nullptr, c->trace + 2 * k);
        if (st != RL_OK) return st;
        if (overlap && c->NH >= 2) {
            // the early and mid parts ran beside the last gradients (minibatch_fwd_bwd); the late
            // part here, and the next minibatch starts after all three
            c->adam_late.grad_out = nullptr;
            CK(q.run(RL_PROF_ADAM, 1, [&] { return launch_adam(c->adam_late, s); }));
            CK(cudaStreamWaitEvent(s, c->ev_early_join, 0));
        } else {
            c->adam.grad_out = nullptr;
            CK(q.run(RL_PROF_ADAM, 1, [&] { return launch_adam(c->adam, s); }));
        }
        if (k + 1 < nmb && !overlap)
            CK(q.run(RL_PROF_GATHER, 1,
                     [&] { return launch_gather(obs, c->bf16 ? 1 : 0, mb_idx(k + 1), Mb, c->Op, c->X0buf[nxt], s); }));
    }
    c->xcur = 0;
    c->X0 = c->X0buf[0];
    CK(q.run(RL_PROF_OTHER, 1, [&] { return launch_small(SMALL_ITER_INC, c->scal, c->iter, nullptr, nullptr, 0.f, s); }));
    if (stats_out)
        CK(q.run(RL_PROF_OTHER, 1,
                 [&] { return launch_small(SMALL_FINAL_STATS, c->scal, c->iter, c->acc, stats_out, (float)c->B, s); }));
    return RL_OK;
}

rl_status train_enqueue(rl_ctx* c, cudaStream_t s, bool profile) {
    Enq q{c, s, profile};
    c->launches = 0;
    c->ev_used = 0;
    const size_t obs_step = (size_t)c->N * c->Op * esize(c);
    uint8_t* obs = reinterpret_cast<uint8_t*>(c->obs);
    CK(q.run(RL_PROF_OTHER, 1, [&] { return launch_small(SMALL_ZERO_STATS, c->scal, c->iter, nullptr, c->acc, 0.f, s); }));
    EnvParams ep = env_params(c);
    ep.stats = c->acc + ACC_ENV;
    for (int t = 0; t < c->T; ++t) {
        const size_t o = (size_t)t * c->N;
        // policy inference: the hidden layers here, the output heads fused into the env step
        rl_status st = forward_hidden(c, q, obs + t * obs_step, c->N, 0, 2, true, t > 0);
        if (st != RL_OK) return st;
        ep.act = head_common(c, c->N);
        ep.act.t = t;
        ep.act.actions = c->actions + o * c->A;
        ep.act.mu = c->mu + o * c->A;
        ep.act.logp = c->logp + o;
        ep.act.values = c->values + o;
        ep.t = t;
        ep.actions = c->actions + o * c->A;
        ep.values = c->values + o;
        ep.obs = obs + (t + 1) * obs_step;
        ep.rew = c->rew + o;
        ep.done = c->done + o;
        ep.timeout = c->timeout + o;
        ep.level_out = c->level;
        ep.tidx_out = nullptr;
        CK(q.run(RL_PROF_ENV, 1, [&] { return launch_env_step(ep, 0, s); }));
    }
    // The shuffle depends only on the seed and the iteration counter (advanced at the end of the
    // update): it runs on the side stream beside the last value, GAE and the record packing, which
    // occupy few SMs.  With per-class profiling it stays on the main stream.
    const bool perm_on_side = !q.profile;
    if (perm_on_side) {
        CK(cudaEventRecord(c->ev_perm_fork, s));
        CK(cudaStreamWaitEvent(c->side, c->ev_perm_fork, 0));
        CK(launch_permutation(c->B, c->cfg.epochs, c->cfg.seed, c->iter, c->perm, c->status, c->side));
        ++c->launches;
        CK(cudaEventRecord(c->ev_perm_join, c->side));
    }
    rl_status st = act_impl(c, q, c->T, c->N, obs + c->T * obs_step, nullptr, nullptr, nullptr, c->last_val, true);
    if (st != RL_OK) return st;
    CK(q.run(RL_PROF_OTHER, 2, [&] {
        return launch_gae(c->T, c->N, c->cfg.gamma, c->cfg.lam, c->rew, c->values, c->last_val, c->done, c->adv, c->ret, 1,
                          c->scal + SC_ADV_MEAN, c->gae_ws, c->gae_nparts, s);
    }));
    st = update_impl(c, q, c->obs, c->actions, c->logp, c->mu, c->values, c->adv, c->ret, c->cfg.epochs, c->cfg.minibatches,
                     c->cfg.clip, c->stats, perm_on_side);
    if (st != RL_OK) return st;
    CK(cudaMemcpyAsync(obs, obs + c->T * obs_step, obs_step, cudaMemcpyDeviceToDevice, s));
    return RL_OK;
}

// ----------------------------------------------------------------------- tile autotuner
// Times every GEMM site of the update (forward, input gradient and weight gradient of each hidden
// layer, actor and critic together, minibatch rows) over candidate tile widths and split counts on
// the context's own buffers, and keeps the fastest.  CUDA events on the launching stream, one
// warm-up and `reps` timed launches per candidate.
// A captured iteration graph holds the tile shapes it was built with: rebuild it on next use.
void drop_graph(rl_ctx* c) {
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    if (c->graph) {
        cudaGraphDestroy(c->graph);
        c->graph = nullptr;
    }
}

rl_status autotune_impl(rl_ctx* c, cudaStream_t s, std::string& report) {
    Enq q{c, s, false};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int reps = 5;
    auto timed = [&](auto&& launch, float& ms) -> rl_status {
        rl_status st = launch();
        if (st != RL_OK) return st;
        CK(cudaEventRecord(e0, s));
        for (int r = 0; r < reps && st == RL_OK; ++r) st = launch();
        if (st != RL_OK) return st;
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(&ms, e0, e1));
        ms /= reps;
        return RL_OK;
    };
    char buf[256];
    rl_status st = RL_OK;
    report = "{\"sites\": [";
    bool first = true;
    std::string trials;
    auto note = [&](const char* site, int l, int bn, int cm, int S, float ms) {
        std::snprintf(buf, sizeof(buf),
                      "%s{\"site\": \"%s\", \"layer\": %d, \"bn\": %d, \"cluster\": %d, \"splits\": %d, \"us\": %.2f}",
                      first ? "" : ", ", site, l, bn, cm, S, ms * 1000.f);
        report += buf;
        first = false;
    };
    auto trial = [&](const char* site, int l, int bn, int cm, int S, float ms) {
        std::snprintf(buf, sizeof(buf), "%s[\"%s\", %d, %d, %d, %d, %.2f]", trials.empty() ? "" : ", ", site, l, bn, cm, S,
                      ms * 1000.f);
        trials += buf;
    };
    const int bns[3] = {64, 128, 256};
    const int cms[4] = {1, 3, 4, 5};
    const int dw_cms[5] = {1, 3, 4, 6, 7};      // weight gradients: no weight-stationary form
    for (int l = 0; l < c->NH && st == RL_OK; ++l) {
        const LayerInfo& Li = c->L[0][l];
        const int row_tiles = (c->Mb + 127) / 128;
        if (c->bf16) {
            // forward: tile width x cluster size
            int best_bn = c->bn_fwd[l], best_cm = c->cm_fwd[l];
            float best = 1e30f;
            for (int bn : bns)
                for (int cm : cms) {
                    if (Li.out % bn || (cm == 3 && row_tiles < 2) || (cm == 3 && bn < 128) || (cm == 4 && bn > 128) ||
                        (cm == 5 && !ws_fits(bn, EPI_BIAS_ELU, Li.in / 64, Li.out)) || st != RL_OK)
                        continue;
                    c->bn_fwd[l] = bn;
                    c->cm_fwd[l] = cm;
                    if (!encode_layer_maps(c, l)) return RL_ERR_CUDA;
                    float ms = 0.f;
                    st = timed([&] { return fwd_layer(c, q, l, c->X0, c->Mb, 0, 2, false); }, ms);
                    if (st == RL_OK) trial("forward", l, bn, cm, 1, ms);
                    if (st == RL_OK && ms < best) { best = ms; best_bn = bn; best_cm = cm; }
                }
            c->bn_fwd[l] = best_bn;
            c->cm_fwd[l] = best_cm;
            note("forward", l, best_bn, best_cm, 1, best);
            // the rollout's policy inference: num_envs rows, both networks
            {
                const int act_tiles = (c->N + 127) / 128;
                int abn = c->bn_act[l], acm = c->cm_act[l];
                float abest = 1e30f;
                for (int bn : bns)
                    for (int cm : cms) {
                        if (Li.out % bn || (cm == 3 && act_tiles < 2) || (cm == 3 && bn < 128) ||
                            (cm == 4 && bn > 128) || (cm == 5 && !ws_fits(bn, EPI_BIAS_ELU, Li.in / 64, Li.out)) ||
                            st != RL_OK)
                            continue;
                        c->bn_act[l] = bn;
                        c->cm_act[l] = cm;
                        if (!encode_layer_maps(c, l)) return RL_ERR_CUDA;
                        float ms = 0.f;
                        st = timed([&] { return fwd_layer(c, q, l, c->obs, c->N, 0, 2, true, true); }, ms);
                        if (st == RL_OK) trial("act_forward", l, bn, cm, 1, ms);
                        if (st == RL_OK && ms < abest) { abest = ms; abn = bn; acm = cm; }
                    }
                c->bn_act[l] = abn;
                c->cm_act[l] = acm;
                note("act_forward", l, abn, acm, 1, abest);
            }
            // input gradient
            if (l > 0 && st == RL_OK) {
                best_bn = c->bn_dx[l];
                best_cm = c->cm_dx[l];
                best = 1e30f;
                for (int bn : bns)
                    for (int cm : cms) {
                        if (Li.in % bn || (cm == 3 && (row_tiles < 2 || bn < 128)) || (cm == 4 && bn > 128) ||
                            (cm == 5 && !ws_fits(bn, EPI_ELU_GRAD, Li.out / 64, Li.in)) || st != RL_OK)
                            continue;
                        c->bn_dx[l] = bn;
                        c->cm_dx[l] = cm;
                        if (!encode_layer_maps(c, l)) return RL_ERR_CUDA;
                        float ms = 0.f;
                        st = timed([&] { return dx_layer(c, q, l, c->Mb); }, ms);
                        if (st == RL_OK) trial("input_grad", l, bn, cm, 1, ms);
                        if (st == RL_OK && ms < best) { best = ms; best_bn = bn; best_cm = cm; }
                    }
                c->bn_dx[l] = best_bn;
                c->cm_dx[l] = best_cm;
                note("input_grad", l, best_bn, best_cm, 1, best);
            }
        }
        // weight gradient: tile width and cluster size (bf16) and split count
        if (st == RL_OK) {
            const int S0 = c->S[l];
            int best_bn = c->bn_dw[l], best_cm = c->cm_dw[l], best_S = S0, best_kc = c->kchunk[l];
            float best = 1e30f;
            const int out_tiles = (Li.out + 127) / 128;
            for (int bi = 0; bi < (c->bf16 ? 3 : 1) && st == RL_OK; ++bi) {
                const int bn = c->bf16 ? bns[bi] : 64;
                if (Li.in % bn) continue;
                for (int cm : dw_cms) {
                    if (cm == 3 && (!c->bf16 || out_tiles < 2 || bn < 128)) continue;   // whole 64-wide B boxes per CTA
                    if ((cm == 4 || cm == 7) && (!c->bf16 || bn > 128)) continue;
                    if (cm == 6 && !c->bf16) continue;
                    // split counts: one or two waves of this width's tiles over the SMs, and the
                    // default's half and double
                    const long long tl = (long long)out_tiles * (Li.in / bn) * 2;
                    const int one_wave = (int)std::max(1ll, 148ll / tl), two_waves = (int)std::max(1ll, 296ll / tl);
                    int cand[4] = {one_wave, two_waves, S0 / 2, 2 * S0};
                    if (!c->bf16) { cand[0] = S0 / 4; cand[1] = S0; }
                    for (int ci = 0; ci < 4; ++ci) {
                        const int S = cand[ci];
                        bool seen = false;
                        for (int cj = 0; cj < ci; ++cj) seen = seen || cand[cj] == S;
                        if (seen || S < 1 || S > c->S_cap[l] || st != RL_OK) continue;
                        int kc = (c->Mb + S - 1) / S;
                        kc = (kc + 63) / 64 * 64;
                        const int Sr = (c->Mb + kc - 1) / kc;
                        if (Sr > c->S_cap[l] && Sr > S0) continue;
                        c->bn_dw[l] = bn;
                        c->cm_dw[l] = cm;
                        c->S[l] = Sr;
                        c->kchunk[l] = kc;
                        if (c->bf16 && !encode_layer_maps(c, l)) return RL_ERR_CUDA;
                        float ms = 0.f;
                        // the split-K partials are summed by Adam: time the GEMM together with that
                        // reduction (Adam's partial-sum pass over this layer's weights, gradient out)
                        st = timed(
                            [&] {
                                rl_status r = dw_layer(c, q, l, c->Mb);
                                if (r != RL_OK) return r;
                                AdamParams red = weight_reduce_params(c, l);
                                CK(launch_adam(red, s));
                                return RL_OK;
                            },
                            ms);
                        if (st == RL_OK) trial("weight_grad", l, bn, cm, Sr, ms);
                        if (st == RL_OK && ms < best) { best = ms; best_bn = bn; best_cm = cm; best_S = Sr; best_kc = kc; }
                    }
                }
            }
            c->bn_dw[l] = best_bn;
            c->cm_dw[l] = best_cm;
            c->S[l] = best_S;
            c->kchunk[l] = best_kc;
            note("weight_grad", l, best_bn, best_cm, best_S, best);
        }
        if (c->bf16 && !encode_layer_maps(c, l)) return RL_ERR_CUDA;
    }
    // the fused forward of the three hidden layers against the layer-by-layer form with the shapes
    // just chosen, at both sites (the update's minibatch rows, the rollout's num_envs rows); the
    // report's cluster field is 1 when the fused form is kept
    if (st == RL_OK && fused_fits(c) && c->gemm_cap == 0) {
        for (int site : {0, 3}) {
            bool& flag = site == 0 ? c->fuse_fwd : c->fuse_act;
            const char* name = site == 0 ? "forward_fused" : "act_forward_fused";
            float ms[2] = {0.f, 0.f};
            for (int f = 0; f < 2 && st == RL_OK; ++f) {
                flag = f == 1;
                st = timed(
                    [&] {
                        return site == 0 ? forward_hidden(c, q, c->X0, c->Mb, 0, 2, false)
                                         : forward_hidden(c, q, c->obs, c->N, 0, 2, true, true);
                    },
                    ms[f]);
                if (st == RL_OK) trial(name, 0, 128, f, 1, ms[f]);
            }
            flag = st == RL_OK && ms[1] < ms[0];
            note(name, 0, 128, flag ? 1 : 0, 1, flag ? ms[1] : ms[0]);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    report += "], \"trials_site_layer_bn_cluster_splits_us\": [" + trials + "]";
    if (c->bf16) {
        std::snprintf(buf, sizeof(buf), ", \"pairs_resident\": %d", tc_cluster_fit(256, EPI_BIAS_ELU, 3));
        report += buf;
    }
    report += "}";
    if (st != RL_OK) return st;
    build_adam(c);
    drop_graph(c);
    return RL_OK;
}

// Checks a tile shape for one GEMM site without applying it; on success *kc_out / *S_out hold the
// weight-gradient K chunk and split count it implies (the current ones for the other sites).
rl_status check_tiles(const rl_ctx* c, int site, int l, int bn, int cm, int splits, int* kc_out, int* S_out) {
    if (!c->bf16 || l < 0 || l >= c->NH || site < 0 || site > 3 || (site == 1 && l == 0)) return RL_ERR_INVALID_ARG;
    if ((bn != 64 && bn != 128 && bn != 256) || cm < 1 || cm > 7 || cm == 2) return RL_ERR_INVALID_ARG;
    if ((cm == 6 || cm == 7) && site != 2) return RL_ERR_INVALID_ARG;
    const LayerInfo& Li = c->L[0][l];
    const int width = (site == 0 || site == 3) ? Li.out : Li.in;
    if (cm == 5 && (site == 2 || width % bn ||
                    !ws_fits(bn, site == 1 ? EPI_ELU_GRAD : EPI_BIAS_ELU, (site == 1 ? Li.out : Li.in) / 64, width)))
        return RL_ERR_INVALID_ARG;
    const int row_tiles = site == 2 ? (Li.out + 127) / 128 : site == 3 ? (c->N + 127) / 128 : (c->Mb + 127) / 128;
    const bool paired = cm == 3;
    if (width % bn || (paired && row_tiles < 2) || (cm == 3 && bn < 128) || ((cm == 4 || cm == 7) && bn > 128))
        return RL_ERR_INVALID_ARG;
    if ((site == 1 || site == 2) && paired && bn < 128) return RL_ERR_INVALID_ARG;   // whole 64-wide B boxes per CTA
    int kc = c->kchunk[l], Sr = c->S[l];
    if (site == 2) {
        if (splits < 1 || splits > c->S_cap[l]) return RL_ERR_INVALID_ARG;
        kc = (c->Mb + splits - 1) / splits;
        kc = (kc + 63) / 64 * 64;
        Sr = (c->Mb + kc - 1) / kc;
    }
    *kc_out = kc;
    *S_out = Sr;
    return RL_OK;
}

rl_status set_tiles_impl(rl_ctx* c, int site, int l, int bn, int cm, int splits) {
    int kc = 0, Sr = 0;
    const rl_status chk = check_tiles(c, site, l, bn, cm, splits, &kc, &Sr);
    if (chk != RL_OK) return chk;
    int* const bnp[4] = {c->bn_fwd, c->bn_dx, c->bn_dw, c->bn_act};
    int* const cmp[4] = {c->cm_fwd, c->cm_dx, c->cm_dw, c->cm_act};
    const int old_bn = bnp[site][l], old_cm = cmp[site][l];
    auto assign = [&](int b, int m) {
        bnp[site][l] = b;
        cmp[site][l] = m;
    };
    assign(bn, cm);
    if (!encode_layer_maps(c, l)) {
        assign(old_bn, old_cm);
        encode_layer_maps(c, l);
        return RL_ERR_CUDA;
    }
    if (site == 2) {
        c->S[l] = Sr;
        c->kchunk[l] = kc;
        build_adam(c);
    }
    drop_graph(c);
    return RL_OK;
}

}  // namespace

// =====================================================================================
extern "C" {

void rl_config_default(rl_config* g) {
    if (!g) return;
    std::memset(g, 0, sizeof(*g));
    g->num_envs = 4096;
    g->num_steps = 24;
    g->grid_x = 17;
    g->grid_y = 11;
    g->obs_dim = 48 + 17 * 11;
    g->obs_pad = 256;
    g->act_dim = 12;
    g->num_hidden = 3;
    g->hidden[0] = 512;
    g->hidden[1] = 256;
    g->hidden[2] = 128;
    g->gamma = 0.99f;
    g->lam = 0.95f;
    g->clip = 0.2f;
    g->entropy_coef = 0.01f;
    g->value_coef = 1.0f;
    g->kl_target = 0.01f;
    g->lr_init = 1e-3f;
    g->lr_min = 1e-5f;
    g->lr_max = 1e-2f;
    g->epochs = 5;
    g->minibatches = 4;
    g->precision = RL_BF16;
    g->kp = 80.f;
    g->kd = 2.f;
    g->action_scale = 0.5f;
    g->dt = 0.02f;
    g->sim_dt = 0.005f;
    g->decimation = 4;
    g->max_episode_len = 1000;
    g->num_levels = 10;
    g->num_cols = 20;
    g->tile_size = 8.f;
    g->hf_res = 0.1f;
    g->grid_spacing = 0.1f;
    g->noise_on = 1;
    g->push_on = 1;
    g->push_interval = 500;
    g->push_vel = 1.f;
    g->cmd_range[0] = g->cmd_range[1] = g->cmd_range[2] = 1.f;
    g->crash_threshold = 9170000u;
    g->seed = 0;
}

int64_t rl_param_count(const rl_config* g) {
    if (!g || g->num_hidden < 1 || g->num_hidden > 4) return -1;
    int64_t total = 0;
    for (int net = 0; net < 2; ++net) {
        int in = g->obs_dim;
        for (int l = 0; l < g->num_hidden; ++l) {
            total += (int64_t)g->hidden[l] * in + g->hidden[l];
            in = g->hidden[l];
        }
        const int out = net == 0 ? g->act_dim : 1;
        total += (int64_t)out * in + out;
        if (net == 0) total += g->act_dim;
    }
    return total;
}

const char* rl_status_string(rl_status s) {
    switch (s) {
        case RL_OK: return "ok";
        case RL_ERR_INVALID_ARG: return "invalid argument";
        case RL_ERR_ALIGNMENT: return "misaligned pointer";
        case RL_ERR_CUDA: return "CUDA error";
        case RL_ERR_TIMEOUT: return "device wait timed out";
        case RL_ERR_STATE: return "invalid state";
        case RL_ERR_OOM: return "out of device memory";
        case RL_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

void rl_destroy(rl_ctx* c) {
    if (!c) return;
    cudaDeviceSynchronize();
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->wside) cudaStreamDestroy(c->wside);
    if (c->aside) cudaStreamDestroy(c->aside);
    if (c->ev_early_fork) cudaEventDestroy(c->ev_early_fork);
    if (c->ev_early_join) cudaEventDestroy(c->ev_early_join);
    if (c->ev_mid_fork) cudaEventDestroy(c->ev_mid_fork);
    for (cudaEvent_t e : c->ev_dw)
        if (e) cudaEventDestroy(e);
    if (c->ev_dw_join) cudaEventDestroy(c->ev_dw_join);
    if (c->ev_perm_fork) cudaEventDestroy(c->ev_perm_fork);
    if (c->ev_perm_join) cudaEventDestroy(c->ev_perm_join);
    if (c->ev_pack_fork) cudaEventDestroy(c->ev_pack_fork);
    if (c->ev_pack_join) cudaEventDestroy(c->ev_pack_join);
    for (int i = 0; i < 2; ++i) {
        if (c->ev_fork[i]) cudaEventDestroy(c->ev_fork[i]);
        if (c->ev_join[i]) cudaEventDestroy(c->ev_join[i]);
    }
    for (void* p : c->allocs) cudaFree(p);
    delete c;
}

static rl_status create_impl(rl_ctx* c, const float* heightfield, const float* init_params) {
    const rl_config& g = c->cfg;
    c->N = g.num_envs; c->T = g.num_steps; c->O = g.obs_dim; c->Op = g.obs_pad; c->A = g.act_dim; c->NH = g.num_hidden;
    for (int i = 0; i < 4; ++i) c->hid[i] = g.hidden[i];
    c->B = c->N * c->T;
    c->Mb = c->B / g.minibatches;
    c->HL = c->hid[c->NH - 1];
    c->rows = std::max(c->N, c->Mb);
    c->bf16 = g.precision == RL_BF16;
    c->cpt = (int)llround((double)g.tile_size / (double)g.hf_res);
    c->nx = g.num_levels * c->cpt;
    c->ny = g.num_cols * c->cpt;
    CK(cudaGetDevice(&c->device));
    CK(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
    CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&c->wside, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&c->aside, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->ev_early_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_early_join, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_mid_fork, cudaEventDisableTiming));
    for (cudaEvent_t& e : c->ev_dw) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_dw_join, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_perm_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_perm_join, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_pack_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_pack_join, cudaEventDisableTiming));
    for (int i = 0; i < 2; ++i) {
        CK(cudaEventCreateWithFlags(&c->ev_fork[i], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->ev_join[i], cudaEventDisableTiming));
    }
    CK(tc_prepare());
    CK(mlp_prepare());
    CK(env_prepare());
    heads_prepare();

    // parameter layout (internal: first-layer weights padded to obs_pad columns)
    long long off = 0, loff = 0;
    for (int n = 0; n < 2; ++n) {
        int in_log = c->O, in = c->Op;
        for (int l = 0; l <= c->NH; ++l) {
            const int out = l < c->NH ? c->hid[l] : (n == 0 ? c->A : 1);
            LayerInfo& Li = c->L[n][l];
            Li.in_log = in_log; Li.in = in; Li.out = out;
            Li.w = off; off += (long long)out * in;
            c->segs.push_back({Li.w, loff, out, in, in_log});
            loff += (long long)out * in_log;
            Li.b = off; off += out;
            c->segs.push_back({Li.b, loff, 1, out, out});
            loff += out;
            in_log = out; in = out;
        }
        if (n == 0) {
            c->logstd = off;
            c->segs.push_back({off, loff, 1, c->A, c->A});
            off += c->A;
            loff += c->A;
        }
    }
    c->P = off;
    c->P_log = loff;
    CK(dalloc(c, &c->params, sizeof(float) * c->P));
    CK(dalloc(c, &c->am, sizeof(float) * c->P));
    CK(dalloc(c, &c->av, sizeof(float) * c->P));
    CK(dalloc(c, &c->grad_int, sizeof(float) * c->P));
    CK(dalloc(c, &c->scal, sizeof(float) * SC_NSCAL));
    CK(dalloc(c, &c->iter, sizeof(unsigned long long)));
    CK(dalloc(c, &c->status, sizeof(int)));
    CK(dalloc(c, &c->acc, sizeof(float) * RL_NSTATS));
    CK(dalloc(c, &c->stats, sizeof(float) * RL_NSTATS));
    // env
    if (g.grid_x * g.grid_y > 0) {
        CK(dalloc(c, &c->hf, sizeof(float) * (size_t)c->nx * c->ny));
        CK(cudaMemcpy(c->hf, heightfield, sizeof(float) * (size_t)c->nx * c->ny, cudaMemcpyHostToDevice));
    }
    CK(dalloc(c, &c->sf, sizeof(float) * (size_t)RL_NF * c->N));
    CK(dalloc(c, &c->si, sizeof(int) * (size_t)RL_NI * c->N));
    // rollout storage
    const size_t NT = (size_t)c->N * c->T;
    CK(dalloc(c, &c->obs, (size_t)(c->T + 1) * c->N * c->Op * esize(c)));
    CK(dalloc(c, &c->actions, sizeof(float) * NT * c->A));
    CK(dalloc(c, &c->mu, sizeof(float) * NT * c->A));
    CK(dalloc(c, &c->logp, sizeof(float) * NT));
    CK(dalloc(c, &c->values, sizeof(float) * NT));
    CK(dalloc(c, &c->rew, sizeof(float) * NT));
    CK(dalloc(c, &c->done, NT));
    CK(dalloc(c, &c->timeout, NT));
    CK(dalloc(c, &c->last_val, sizeof(float) * c->N));
    CK(dalloc(c, &c->adv, sizeof(float) * NT));
    CK(dalloc(c, &c->ret, sizeof(float) * NT));
    CK(dalloc(c, &c->level, sizeof(int) * c->N));
    c->gae_nparts = gae_num_partials(c->T, c->N);
    CK(dalloc(c, &c->gae_ws, rl_gae_workspace_bytes(c->T, c->N)));
    // update workspaces
    CK(dalloc(c, &c->perm, sizeof(int) * (size_t)g.epochs * c->B));
    CK(dalloc(c, &c->trace, sizeof(float) * 2 * (size_t)g.epochs * g.minibatches));
    CK(dalloc(c, &c->iota, sizeof(int) * (size_t)c->Mb));
    {
        std::vector<int> io(c->Mb);
        for (int i = 0; i < c->Mb; ++i) io[i] = i;
        CK(cudaMemcpy(c->iota, io.data(), sizeof(int) * c->Mb, cudaMemcpyHostToDevice));
    }
    CK(dalloc(c, &c->logstd_old, sizeof(float) * c->A));
    for (int x = 0; x < 2; ++x) CK(dalloc(c, &c->X0buf[x], (size_t)c->rows * c->Op * esize(c)));
    c->X0 = c->X0buf[0];
    for (int n = 0; n < 2; ++n)
        for (int l = 0; l < c->NH; ++l) {
            CK(dalloc(c, &c->H[n][l], (size_t)c->rows * c->hid[l] * esize(c)));
            CK(dalloc(c, &c->dY[n][l], (size_t)c->rows * c->hid[l] * esize(c)));
        }
    // split-K of the weight-gradient GEMMs.  BF16: 256-wide tiles (each dY^T tile read once
    // per layer input width) and about one wave of 148 CTAs, each K range >= 384 rows.  FP32:
    // 128 x 64 tiles, about two CTAs per SM, at most 16 slices.
    c->mtiles = (c->Mb + 127) / 128;
    c->gb_parts = c->mtiles * (c->bf16 ? 4 : 1);
    for (int l = 0; l < c->NH; ++l) {
        const LayerInfo& Li = c->L[0][l];
        const int bn = c->bf16 ? (Li.in % 256 == 0 ? 256 : pick_bn(Li.in)) : 64;
        const long long tiles = (long long)((Li.out + 127) / 128) * (Li.in / bn) * 2;
        int S;
        if (c->bf16)
            S = (int)std::max(1ll, std::min((long long)std::max(1, c->Mb / 384), 148ll / tiles));
        else
            S = (int)std::max(1ll, std::min(16ll, (2ll * 148 + tiles / 2) / tiles));
        const int unit = 64;
        int kc = (c->Mb + S - 1) / S;
        kc = (kc + unit - 1) / unit * unit;
        S = (c->Mb + kc - 1) / kc;
        c->S[l] = S;
        c->kchunk[l] = kc;
        // room for the autotuner's larger splits: two waves of the narrowest (64-column) tiles
        const long long tiles64 = (long long)((Li.out + 127) / 128) * (Li.in / 64) * 2;
        c->S_cap[l] = (int)std::min((long long)std::max(1, c->Mb / 64), std::max(2ll * S, 296ll / tiles64 + 1));
        c->bn_fwd[l] = pick_bn(Li.out);
        c->bn_dx[l] = pick_bn(Li.in);
        c->bn_dw[l] = bn;
        // one CTA per tile until the autotuner or rl_set_gemm_tiles picks another mode
        c->cm_fwd[l] = 1;
        c->bn_act[l] = pick_bn(Li.out);
        c->cm_act[l] = 1;
        c->cm_dx[l] = 1;
        c->cm_dw[l] = 1;
        for (int n = 0; n < 2; ++n) {
            CK(dalloc(c, &c->gw[n][l], sizeof(float) * (size_t)std::max(S, c->S_cap[l]) * Li.out * Li.in));
            if (l < c->NH - 1) CK(dalloc(c, &c->gb[n][l], sizeof(float) * (size_t)c->gb_parts * Li.out));
        }
    }
    c->head_blocks = loss_head_blocks(c->Mb, c->HL, c->bf16 ? 1 : 0);
    CK(dalloc(c, &c->head_part, sizeof(float) * (size_t)c->head_blocks * head_part_floats(c->A, c->HL)));
    if (c->bf16) CK(dalloc(c, &c->recs, sizeof(float) * (size_t)c->B * REC_LD));
    if (c->bf16) {
        for (int n = 0; n < 2; ++n)
            for (int l = 0; l < c->NH; ++l) {
                const LayerInfo& Li = c->L[n][l];
                CK(dalloc(c, &c->wbf[n][l], (size_t)Li.out * Li.in * 2));
            }
        bool ok = make_tmap_bf16(&c->tm_x0, c->X0, c->rows, c->Op, c->Op, 128);
        for (int l = 0; l < c->NH; ++l) ok = ok && encode_layer_maps(c, l);
        if (!ok) return RL_ERR_CUDA;
    }
    for (int n = 0; n < 2; ++n)          // the GEMM epilogues read biases as float4
        for (int l = 0; l < c->NH; ++l)
            if (c->L[n][l].b % 4) return RL_ERR_UNSUPPORTED;
    build_adam(c);
    // parameters, learning rate, env state
    std::vector<float> pi(c->P, 0.f);
    for (const Seg& sg : c->segs)
        for (int r = 0; r < sg.rows; ++r)
            std::memcpy(&pi[sg.ioff + (long long)r * sg.cols_int], &init_params[sg.loff + (long long)r * sg.cols_log],
                        sizeof(float) * sg.cols_log);
    CK(cudaMemcpy(c->params, pi.data(), sizeof(float) * c->P, cudaMemcpyHostToDevice));
    float sc[SC_NSCAL] = {};
    sc[SC_ALPHA] = g.lr_init;
    CK(cudaMemcpy(c->scal, sc, sizeof(sc), cudaMemcpyHostToDevice));
    rl_status st = refresh_bf16(c, nullptr);
    if (st != RL_OK) return st;
    EnvParams ep = env_params(c);
    ep.obs = c->obs;
    ep.level_out = c->level;
    CK(launch_env_step(ep, 1, nullptr));
    CK(cudaDeviceSynchronize());
    return RL_OK;
}

rl_status rl_create(const rl_config* cfg, const float* heightfield, const float* init_params, rl_ctx** out) {
    if (!out) return RL_ERR_INVALID_ARG;
    *out = nullptr;
    if (!config_ok(cfg) || !init_params) return RL_ERR_INVALID_ARG;
    if (cfg->grid_x * cfg->grid_y > 0 && !heightfield) return RL_ERR_INVALID_ARG;
    rl_ctx* c = new rl_ctx();
    c->cfg = *cfg;
    rl_status st = create_impl(c, heightfield, init_params);
    if (st != RL_OK) {
        rl_destroy(c);
        cudaGetLastError();
        return st;
    }
    *out = c;
    return RL_OK;
}

static cudaStream_t S_(void* s) { return reinterpret_cast<cudaStream_t>(s); }

rl_status rl_get_params(rl_ctx* c, float* out, void* stream) {
    if (!c || !out) return RL_ERR_INVALID_ARG;
    for (const Seg& sg : c->segs)
        CK(cudaMemcpy2DAsync(out + sg.loff, sizeof(float) * sg.cols_log, c->params + sg.ioff, sizeof(float) * sg.cols_int,
                             sizeof(float) * sg.cols_log, sg.rows, cudaMemcpyDeviceToDevice, S_(stream)));
    return RL_OK;
}

rl_status rl_get_adam_moments(rl_ctx* c, float* m_out, float* v_out, void* stream) {
    if (!c || !m_out || !v_out) return RL_ERR_INVALID_ARG;
    for (const Seg& sg : c->segs) {
        CK(cudaMemcpy2DAsync(m_out + sg.loff, sizeof(float) * sg.cols_log, c->am + sg.ioff, sizeof(float) * sg.cols_int,
                             sizeof(float) * sg.cols_log, sg.rows, cudaMemcpyDeviceToDevice, S_(stream)));
        CK(cudaMemcpy2DAsync(v_out + sg.loff, sizeof(float) * sg.cols_log, c->av + sg.ioff, sizeof(float) * sg.cols_int,
                             sizeof(float) * sg.cols_log, sg.rows, cudaMemcpyDeviceToDevice, S_(stream)));
    }
    return RL_OK;
}

rl_status rl_set_params(rl_ctx* c, const float* in, void* stream) {
    if (!c || !in) return RL_ERR_INVALID_ARG;
    for (const Seg& sg : c->segs)
        CK(cudaMemcpy2DAsync(c->params + sg.ioff, sizeof(float) * sg.cols_int, in + sg.loff, sizeof(float) * sg.cols_log,
                             sizeof(float) * sg.cols_log, sg.rows, cudaMemcpyDeviceToDevice, S_(stream)));
    return refresh_bf16(c, S_(stream));
}

rl_status rl_actuator_lstm_step(int32_t n, const float* weights, const float* x, float* h, float* c, float* tau,
                                void* stream) {
    static_assert(ACT_INPUTS == RL_ACT_INPUTS && ACT_HIDDEN == RL_ACT_HIDDEN, "actuator cell sizes");
    if (n < 0 || (n > 0 && (!weights || !x || !h || !c || !tau))) return RL_ERR_INVALID_ARG;
    for (const void* p : {(const void*)weights, (const void*)x, (const void*)h, (const void*)c, (const void*)tau})
        if (reinterpret_cast<uintptr_t>(p) & 3u) return RL_ERR_ALIGNMENT;
    CK(launch_actuator_lstm(n, weights, x, h, c, tau, S_(stream)));
    return RL_OK;
}

rl_status rl_terrain_generate(const rl_config* cfg, float* hf, void* stream) {
    if (!cfg || !hf || cfg->num_levels < 1 || cfg->num_cols < 1 || !(cfg->hf_res > 0.f)) return RL_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(hf) & 3u) return RL_ERR_ALIGNMENT;
    // lengths in whole cells: the tile, the platform half width (1 m), the stair width (0.3 m) and
    // the obstacle block (1 m)
    auto cells = [&](double len, int& n) {
        const double r = (double)cfg->hf_res;
        n = (int)std::llround(len / r);
        return n > 0 && std::fabs(n * r - len) <= 1e-6 * std::max(1.0, len);
    };
    TerrainParams t;
    if (!cells((double)cfg->tile_size, t.c) || !cells(1.0, t.P) || !cells(0.3, t.W) || !cells(1.0, t.B)) return RL_ERR_INVALID_ARG;
    if (t.c % 2 || t.c % t.B || t.c / 2 < t.P) return RL_ERR_INVALID_ARG;
    if ((long long)cfg->num_levels * t.c * cfg->num_cols * t.c > (1ll << 31)) return RL_ERR_INVALID_ARG;
    t.levels = cfg->num_levels;
    t.cols = cfg->num_cols;
    t.res = cfg->hf_res;
    t.seed = cfg->seed;
    CK(launch_terrain(t, hf, S_(stream)));
    return RL_OK;
}

// ---- checkpoint image: header, then the state segments in a fixed order
namespace {
constexpr char CKPT_MAGIC[8] = {'R', 'L', 'B', '3', '0', '0', 'C', 'K'};
constexpr uint32_t CKPT_VERSION = 1;
constexpr int CKPT_SEGS = 9;
struct CkptHeader {
    char magic[8];
    uint32_t version, nseg;
    uint64_t seg_bytes[CKPT_SEGS];
    int32_t tiles[4][4][3];       // [hidden layer][site fwd / dx / dw / act][bn, cluster mode, splits]
    rl_config cfg;
};
struct CkptSeg {
    void* dev;
    size_t bytes;
};
// params, Adam m, Adam v, scalar block, iteration counter, env fp32 state, env int state, curriculum
// levels, the next rollout's first observation
void ckpt_segments(rl_ctx* c, CkptSeg (&sg)[CKPT_SEGS]) {
    sg[0] = {c->params, sizeof(float) * (size_t)c->P};
    sg[1] = {c->am, sizeof(float) * (size_t)c->P};
    sg[2] = {c->av, sizeof(float) * (size_t)c->P};
    sg[3] = {c->scal, sizeof(float) * (size_t)SC_NSCAL};
    sg[4] = {c->iter, sizeof(unsigned long long)};
    sg[5] = {c->sf, sizeof(float) * (size_t)RL_NF * c->N};
    sg[6] = {c->si, sizeof(int) * (size_t)RL_NI * c->N};
    sg[7] = {c->level, sizeof(int) * (size_t)c->N};
    sg[8] = {c->obs, (size_t)c->N * c->Op * esize(c)};
}
size_t ckpt_bytes(rl_ctx* c) {
    CkptSeg sg[CKPT_SEGS];
    ckpt_segments(c, sg);
    size_t n = sizeof(CkptHeader);
    for (const CkptSeg& x : sg) n += x.bytes;
    return n;
}
}  // namespace

int64_t rl_checkpoint_bytes(rl_ctx* c) { return c ? (int64_t)ckpt_bytes(c) : -1; }

rl_status rl_checkpoint_save(rl_ctx* c, void* dst, size_t bytes, void* stream) {
    if (!c || !dst || bytes < ckpt_bytes(c)) return RL_ERR_INVALID_ARG;
    CkptSeg sg[CKPT_SEGS];
    ckpt_segments(c, sg);
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, CKPT_MAGIC, sizeof(h.magic));
    h.version = CKPT_VERSION;
    h.nseg = CKPT_SEGS;
    for (int i = 0; i < CKPT_SEGS; ++i) h.seg_bytes[i] = sg[i].bytes;
    for (int l = 0; l < c->NH && l < 4; ++l) {
        const int bn[4] = {c->bn_fwd[l], c->bn_dx[l], c->bn_dw[l], c->bn_act[l]};
        const int cm[4] = {c->cm_fwd[l], c->cm_dx[l], c->cm_dw[l], c->cm_act[l]};
        for (int site = 0; site < 4; ++site) {
            h.tiles[l][site][0] = bn[site];
            h.tiles[l][site][1] = cm[site];
            h.tiles[l][site][2] = site == 2 ? c->S[l] : 1;
        }
    }
    h.cfg = c->cfg;
    std::memcpy(dst, &h, sizeof(h));
    uint8_t* out = reinterpret_cast<uint8_t*>(dst) + sizeof(h);
    for (const CkptSeg& x : sg) {
        CK(cudaMemcpyAsync(out, x.dev, x.bytes, cudaMemcpyDeviceToHost, S_(stream)));
        out += x.bytes;
    }
    CK(cudaStreamSynchronize(S_(stream)));
    return RL_OK;
}

rl_status rl_checkpoint_load(rl_ctx* c, const void* src, size_t bytes, void* stream) {
    if (!c || !src || bytes < sizeof(CkptHeader)) return RL_ERR_INVALID_ARG;
    CkptHeader h;
    std::memcpy(&h, src, sizeof(h));
    CkptSeg sg[CKPT_SEGS];
    ckpt_segments(c, sg);
    if (std::memcmp(h.magic, CKPT_MAGIC, sizeof(h.magic)) || h.version != CKPT_VERSION || h.nseg != CKPT_SEGS ||
        bytes < ckpt_bytes(c) || std::memcmp(&h.cfg, &c->cfg, sizeof(rl_config)))
        return RL_ERR_INVALID_ARG;
    for (int i = 0; i < CKPT_SEGS; ++i)
        if (h.seg_bytes[i] != sg[i].bytes) return RL_ERR_INVALID_ARG;
    // the GEMM shapes of the saved run: split counts fix the order of the weight-gradient sums,
    // so the resumed run repeats the saved one bit for bit.  Every record is checked before any
    // is applied, so a damaged image leaves the context as it was.
    if (c->bf16) {
        for (int pass = 0; pass < 2; ++pass)
            for (int l = 0; l < c->NH && l < 4; ++l)
                for (int site = 0; site < 4; ++site) {
                    if (site == 1 && l == 0) continue;
                    const int32_t* t = h.tiles[l][site];
                    int kc = 0, S = 0;
                    const rl_status st = pass == 0 ? check_tiles(c, site, l, t[0], t[1], t[2], &kc, &S)
                                                   : set_tiles_impl(c, site, l, t[0], t[1], t[2]);
                    if (st != RL_OK) return st;
                }
    }
    const uint8_t* in = reinterpret_cast<const uint8_t*>(src) + sizeof(h);
    for (const CkptSeg& x : sg) {
        CK(cudaMemcpyAsync(x.dev, in, x.bytes, cudaMemcpyHostToDevice, S_(stream)));
        in += x.bytes;
    }
    rl_status st = refresh_bf16(c, S_(stream));
    if (st != RL_OK) return st;
    CK(cudaStreamSynchronize(S_(stream)));
    return RL_OK;
}

rl_status rl_get_scalars(rl_ctx* c, double out[4]) {
    if (!c || !out) return RL_ERR_INVALID_ARG;
    float sc[SC_NSCAL];
    unsigned long long it = 0;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(sc, c->scal, sizeof(sc), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&it, c->iter, sizeof(it), cudaMemcpyDeviceToHost));
    out[0] = sc[SC_ALPHA];
    out[1] = (double)it;
    out[2] = sc[SC_STEP];
    out[3] = sc[SC_KL];
    return RL_OK;
}

rl_status rl_set_scalars(rl_ctx* c, double alpha, int64_t iteration, int64_t adam_step, void* stream) {
    if (!c || iteration < 0 || adam_step < 0 || !(alpha > 0)) return RL_ERR_INVALID_ARG;
    static thread_local float a;
    static thread_local float st;
    static thread_local unsigned long long it;
    a = (float)alpha;
    st = (float)adam_step;
    it = (unsigned long long)iteration;
    CK(cudaMemcpyAsync(c->scal + SC_ALPHA, &a, sizeof(float), cudaMemcpyHostToDevice, S_(stream)));
    CK(cudaMemcpyAsync(c->scal + SC_STEP, &st, sizeof(float), cudaMemcpyHostToDevice, S_(stream)));
    CK(cudaMemcpyAsync(c->iter, &it, sizeof(it), cudaMemcpyHostToDevice, S_(stream)));
    CK(cudaStreamSynchronize(S_(stream)));
    return RL_OK;
}

// host or device buffers: the copy direction follows from the unified address space
rl_status rl_env_get_state(rl_ctx* c, float* sf, int32_t* si, void* stream) {
    if (!c || !sf || !si) return RL_ERR_INVALID_ARG;
    CK(cudaMemcpyAsync(sf, c->sf, sizeof(float) * (size_t)RL_NF * c->N, cudaMemcpyDefault, S_(stream)));
    CK(cudaMemcpyAsync(si, c->si, sizeof(int) * (size_t)RL_NI * c->N, cudaMemcpyDefault, S_(stream)));
    return RL_OK;
}

rl_status rl_env_set_state(rl_ctx* c, const float* sf, const int32_t* si, void* stream) {
    if (!c || !sf || !si) return RL_ERR_INVALID_ARG;
    CK(cudaMemcpyAsync(c->sf, sf, sizeof(float) * (size_t)RL_NF * c->N, cudaMemcpyDefault, S_(stream)));
    CK(cudaMemcpyAsync(c->si, si, sizeof(int) * (size_t)RL_NI * c->N, cudaMemcpyDefault, S_(stream)));
    return RL_OK;
}

rl_status rl_env_reset_all(rl_ctx* c, void* obs_out, void* stream) {
    if (!c) return RL_ERR_INVALID_ARG;
    if (obs_out && !aligned16(obs_out)) return RL_ERR_ALIGNMENT;
    EnvParams ep = env_params(c);
    ep.obs = obs_out ? obs_out : c->obs;
    ep.level_out = c->level;
    CK(launch_env_step(ep, 1, S_(stream)));
    return RL_OK;
}

rl_status rl_env_step(rl_ctx* c, int32_t t, const float* actions, const float* values, void* obs_out, float* rew_out,
                      uint8_t* done_out, uint8_t* timeout_out, int32_t* level_out, int32_t* tidx_out, void* stream) {
    if (!c || !actions || !values || !obs_out || !rew_out || t < 0) return RL_ERR_INVALID_ARG;
    if (!aligned16(obs_out) || !aligned16(actions)) return RL_ERR_ALIGNMENT;
    EnvParams ep = env_params(c);
    ep.t = t;
    ep.actions = actions;
    ep.values = values;
    ep.obs = obs_out;
    ep.rew = rew_out;
    ep.done = done_out;
    ep.timeout = timeout_out;
    ep.level_out = level_out;
    ep.tidx_out = tidx_out;
    CK(launch_env_step(ep, 0, S_(stream)));
    return RL_OK;
}

rl_status rl_policy_act(rl_ctx* c, int32_t t, int32_t n, const void* obs, float* actions, float* mu, float* logp,
                        float* values, void* stream) {
    if (!c || !obs || !values || n < 1 || n > c->rows || t < 0) return RL_ERR_INVALID_ARG;
    if (!aligned16(obs)) return RL_ERR_ALIGNMENT;
    const bool any = actions || mu || logp;
    if (any && !(actions && mu && logp)) return RL_ERR_INVALID_ARG;
    Enq q{c, S_(stream), false};
    return act_impl(c, q, t, n, obs, actions, mu, logp, values);
}

size_t rl_gae_workspace_bytes(int32_t T, int32_t N) { return gae_workspace_bytes(T, N); }

rl_status rl_gae(int32_t T, int32_t N, float gamma, float lam, const float* rew, const float* val, const float* last_val,
                 const uint8_t* done, float* adv_out, float* ret_out, int32_t normalize, float* adv_stats_out,
                 void* workspace, size_t workspace_bytes, void* stream) {
    if (T <= 0 || N <= 0 || !rew || !val || !last_val || !done || !adv_out || !ret_out) return RL_ERR_INVALID_ARG;
    const bool need = normalize || adv_stats_out;
    if (need && (!workspace || workspace_bytes < rl_gae_workspace_bytes(T, N))) return RL_ERR_INVALID_ARG;
    if (!aligned16(adv_out) || (need && !aligned16(workspace))) return RL_ERR_ALIGNMENT;
    CK(launch_gae(T, N, gamma, lam, rew, val, last_val, done, adv_out, ret_out, normalize, adv_stats_out,
                  reinterpret_cast<float*>(workspace), gae_num_partials(T, N), S_(stream)));
    return RL_OK;
}

rl_status rl_gae_noalloc(int32_t T, int32_t N, float gamma, float lam, const float* rew, const float* val,
                         const float* last_val, const uint8_t* done, float* adv_out, float* ret_out, int32_t normalize,
                         float* adv_stats_out, void* stream) {
    if (T <= 0 || N <= 0 || !rew || !val || !last_val || !done || !adv_out || !ret_out) return RL_ERR_INVALID_ARG;
    if (N > gae_noalloc_max_envs()) return RL_ERR_INVALID_ARG;
    if (!aligned16(adv_out)) return RL_ERR_ALIGNMENT;
    void* scratch = nullptr;
    CK(gae_noalloc_scratch(S_(stream), &scratch));
    CK(launch_gae(T, N, gamma, lam, rew, val, last_val, done, adv_out, ret_out, normalize, adv_stats_out,
                  reinterpret_cast<float*>(scratch), gae_num_partials(T, N), S_(stream)));
    return RL_OK;
}

rl_status rl_ppo_update(rl_ctx* c, const void* obs, const float* actions, const float* logp_old, const float* mu_old,
                        const float* val_old, const float* adv, const float* ret, int32_t epochs, int32_t minibatches,
                        float clip, float* stats_out, void* stream) {
    if (!c || !obs || !actions || !logp_old || !mu_old || !val_old || !adv || !ret) return RL_ERR_INVALID_ARG;
    if (epochs < 1 || minibatches < 1 || c->B % minibatches || c->B / minibatches != c->Mb || epochs > c->cfg.epochs)
        return RL_ERR_INVALID_ARG;
    if (!(clip > 0.f && clip < 1.f)) return RL_ERR_INVALID_ARG;
    cudaStream_t s = S_(stream);
    CK(launch_small(SMALL_ZERO_STATS, c->scal, c->iter, nullptr, c->acc, 0.f, s));
    Enq q{c, s, false};
    return update_impl(c, q, obs, actions, logp_old, mu_old, val_old, adv, ret, epochs, minibatches, clip, stats_out, false);
}

rl_status rl_ppo_loss_grad(rl_ctx* c, int32_t M, const void* obs, const float* actions, const float* logp_old,
                           const float* mu_old, const float* log_std_old, const float* val_old, const float* adv,
                           const float* ret, float* grad_out, float* stats_out, void* stream) {
    if (!c || !obs || !actions || !logp_old || !mu_old || !log_std_old || !val_old || !adv || !ret || !grad_out)
        return RL_ERR_INVALID_ARG;
    if (M < 1 || M > c->Mb || M % 64) return RL_ERR_INVALID_ARG;
    cudaStream_t s = S_(stream);
    Enq q{c, s, false};
    CK(launch_gather(obs, c->bf16 ? 1 : 0, c->iota, M, c->Op, c->X0, s));
    for (int n = 0; n < 2; ++n)          // row tiles past M leave no bias-gradient partial
        for (int l = 0; l + 1 < c->NH; ++l)
            CK(cudaMemsetAsync(c->gb[n][l], 0, sizeof(float) * (size_t)c->gb_parts * c->hid[l], s));
    rl_status st = minibatch_fwd_bwd(c, q, M, nullptr, actions, logp_old, mu_old, log_std_old, val_old, adv, ret, c->cfg.clip,
                                     false);
    if (st != RL_OK) return st;
    AdamParams a = c->adam;
    a.grad_out = c->grad_int;
    CK(launch_adam(a, s));
    for (const Seg& sg : c->segs)
        CK(cudaMemcpy2DAsync(grad_out + sg.loff, sizeof(float) * sg.cols_log, c->grad_int + sg.ioff,
                             sizeof(float) * sg.cols_int, sizeof(float) * sg.cols_log, sg.rows, cudaMemcpyDeviceToDevice, s));
    if (stats_out) {
        // [0] loss, [1] surrogate, [2] value loss, [3] entropy, [4] KL, [6] clip fraction
        CK(cudaMemsetAsync(stats_out, 0, sizeof(float) * RL_NSTATS, s));
        CK(cudaMemcpyAsync(stats_out + 0, c->scal + SC_LOSS, sizeof(float) * 4, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(stats_out + 4, c->scal + SC_KL, sizeof(float), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(stats_out + 6, c->scal + SC_CLIPFRAC, sizeof(float), cudaMemcpyDeviceToDevice, s));
    }
    return RL_OK;
}

rl_status rl_train_iteration(rl_ctx* c, int32_t use_graph, float* stats_host, void* stream) {
    if (!c) return RL_ERR_INVALID_ARG;
    cudaStream_t s = S_(stream);
    if (use_graph) {
        // The graph is captured and replayed on the context's own stream (capture is not
        // allowed on the legacy default stream), ordered after and before the caller's stream.
        cudaStream_t g = c->gstream;
        CK(cudaEventRecord(c->ev_in, s));
        CK(cudaStreamWaitEvent(g, c->ev_in, 0));
        if (!c->gexec) {
            CK(cudaStreamBeginCapture(g, cudaStreamCaptureModeThreadLocal));
            rl_status st = train_enqueue(c, g, c->prof_mask != 0);
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamEndCapture(g, &graph);
            if (st != RL_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            CK(e);
            c->graph = graph;
            CK(cudaGraphInstantiate(&c->gexec, graph, 0));
        }
        CK(cudaGraphLaunch(c->gexec, g));
        CK(cudaEventRecord(c->ev_out, g));
        CK(cudaStreamWaitEvent(s, c->ev_out, 0));
    } else {
        rl_status st = train_enqueue(c, s, c->prof_mask != 0);
        if (st != RL_OK) return st;
    }
    if (stats_host) {
        CK(cudaMemcpyAsync(stats_host, c->stats, sizeof(float) * RL_NSTATS, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return RL_OK;
}

rl_status rl_get_storage(rl_ctx* c, int32_t which, void** ptr, size_t* bytes) {
    if (!c || !ptr) return RL_ERR_INVALID_ARG;
    const size_t NT = (size_t)c->N * c->T;
    void* p = nullptr;
    size_t b = 0;
    switch (which) {
        case 0: p = c->obs; b = (size_t)(c->T + 1) * c->N * c->Op * esize(c); break;
        case 1: p = c->actions; b = NT * c->A * 4; break;
        case 2: p = c->mu; b = NT * c->A * 4; break;
        case 3: p = c->logp; b = NT * 4; break;
        case 4: p = c->values; b = NT * 4; break;
        case 5: p = c->rew; b = NT * 4; break;
        case 6: p = c->done; b = NT; break;
        case 7: p = c->timeout; b = NT; break;
        case 8: p = c->last_val; b = (size_t)c->N * 4; break;
        case 9: p = c->adv; b = NT * 4; break;
        case 10: p = c->ret; b = NT * 4; break;
        case 11: p = c->level; b = (size_t)c->N * 4; break;
        case 12: p = c->stats; b = RL_NSTATS * 4; break;
        case 13: p = c->perm; b = sizeof(int) * (size_t)c->cfg.epochs * c->B; break;
        case 14: p = c->trace; b = sizeof(float) * 2 * (size_t)c->cfg.epochs * c->cfg.minibatches; break;
        default: return RL_ERR_INVALID_ARG;
    }
    *ptr = p;
    if (bytes) *bytes = b;
    return RL_OK;
}

rl_status rl_last_device_status(rl_ctx* c) {
    if (!c) return RL_ERR_INVALID_ARG;
    int st = 0;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost));
    return st;
}

rl_status rl_clear_device_status(rl_ctx* c, void* stream) {
    if (!c) return RL_ERR_INVALID_ARG;
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), S_(stream)));
    return RL_OK;
}

rl_status rl_diag_forced_timeout(rl_ctx* c, void* stream) {
    if (!c) return RL_ERR_INVALID_ARG;
    CK(launch_forced_timeout(c->status, S_(stream)));
    return RL_OK;
}

rl_status rl_profile_enable(rl_ctx* c, int32_t kernel_class, int32_t on) {
    if (!c || kernel_class < 0 || kernel_class > RL_PROF_ALL) return RL_ERR_INVALID_ARG;
    const unsigned bits = kernel_class == RL_PROF_ALL ? 0x7Fu : (1u << kernel_class);
    c->prof_mask = on ? (c->prof_mask | bits) : (c->prof_mask & ~bits);
    if (c->prof_mask && c->ev.empty()) {
        // one event pair per launch of an iteration, every class recorded
        const size_t launches = (size_t)(c->T + 1) * (c->NH + 2) + (size_t)c->cfg.epochs * c->cfg.minibatches * (3 * c->NH + 4) + 16;
        for (size_t i = 0; i < 2 * launches; ++i) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            c->ev.push_back(e);
        }
        c->ev_cls.assign(launches, -1);
    }
    // a graph built without (or with) the event nodes is rebuilt on next use
    drop_graph(c);
    return RL_OK;
}

static rl_status profile_sum(rl_ctx* c, int cls, float* total_ms, int32_t* launches) {
    if (!c || !total_ms || !launches) return RL_ERR_INVALID_ARG;
    float tot = 0.f;
    int n = 0;
    for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
        if (cls >= 0 && c->ev_cls[i / 2] != cls) continue;
        CK(cudaEventSynchronize(c->ev[i + 1]));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]));
        tot += ms;
        ++n;
    }
    *total_ms = tot;
    *launches = n;
    return RL_OK;
}

rl_status rl_profile_read(rl_ctx* c, float* total_ms, int32_t* launches) { return profile_sum(c, -1, total_ms, launches); }

rl_status rl_profile_read_class(rl_ctx* c, int32_t kernel_class, float* total_ms, int32_t* launches) {
    if (kernel_class < 0 || kernel_class >= RL_PROF_ALL) return RL_ERR_INVALID_ARG;
    return profile_sum(c, kernel_class, total_ms, launches);
}

rl_status rl_autotune(rl_ctx* c, char* report, size_t report_bytes, void* stream) {
    if (!c) return RL_ERR_INVALID_ARG;
    std::string rep;
    rl_status st = autotune_impl(c, S_(stream), rep);
    if (report && report_bytes) {
        std::snprintf(report, report_bytes, "%s", rep.c_str());
    }
    return st;
}

rl_status rl_set_gemm_ctas(rl_ctx* c, int32_t max_ctas) {
    if (!c || max_ctas < 0) return RL_ERR_INVALID_ARG;
    c->gemm_cap = max_ctas;
    build_adam(c);          // the cap decides which weight gradients reduce their splits in clusters
    drop_graph(c);
    return RL_OK;
}


rl_status rl_adam_step(int64_t n, float* p, const float* g, int32_t nsplit, float* m, float* v, float lr, int32_t t,
                       void* bf16_out, void* stream) {
    if (n < 1 || !p || !g || !m || !v || nsplit < 1 || t < 1 || !(lr >= 0.f)) return RL_ERR_INVALID_ARG;
    AdamParams a;
    std::memset(&a, 0, sizeof(a));
    a.p = p;
    a.m = m;
    a.v = v;
    const double t_d = (double)t;
    a.step_size_host = (float)((double)lr / (1.0 - std::pow(0.9, t_d)));
    a.inv_sqrt_bc2_host = (float)(1.0 / std::sqrt(1.0 - std::pow(0.999, t_d)));
    // one segment per 2^30 parameters (the segment's block count stays within an int)
    long long off = 0;
    int blocks = 0;
    while (off < n) {
        if (a.nsegs == MAX_SEGS) return RL_ERR_INVALID_ARG;
        const long long size = std::min<long long>(n - off, 1ll << 30);
        AdamSeg& sg = a.seg[a.nsegs];
        sg.offset = off;
        sg.size = size;
        sg.partials = g + off;
        sg.stride = n;
        sg.nsplit = nsplit;
        sg.block_start = blocks;
        a.wbf[a.nsegs] = bf16_out ? static_cast<void*>(static_cast<__nv_bfloat16*>(bf16_out) + off) : nullptr;
        sg.vec = (off % 4 == 0 && size % 4 == 0 && n % 4 == 0 && ((reinterpret_cast<uintptr_t>(g) | reinterpret_cast<uintptr_t>(p) |
                                                                   reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v)) & 15u) == 0 &&
                  (reinterpret_cast<uintptr_t>(bf16_out) & 7u) == 0)
                     ? 1
                     : 0;
        const long long per_block = adam_per_block(nsplit, sg.vec);
        const long long nb = (size + per_block - 1) / per_block;
        if (blocks + nb > (1ll << 31) - 1) return RL_ERR_INVALID_ARG;
        blocks += (int)nb;
        off += size;
        ++a.nsegs;
    }
    a.nblocks = blocks;
    CK(launch_adam(a, S_(stream)));
    return RL_OK;
}

rl_status rl_set_gemm_tiles(rl_ctx* c, int32_t site, int32_t layer, int32_t bn, int32_t cluster, int32_t splits) {
    if (!c) return RL_ERR_INVALID_ARG;
    return set_tiles_impl(c, site, layer, bn, cluster, splits);
}

rl_status rl_set_forward_fused(rl_ctx* c, int32_t site, int32_t on) {
    if (!c || (site != 0 && site != 3) || (on != 0 && on != 1) || (on && !fused_fits(c))) return RL_ERR_INVALID_ARG;
    (site == 0 ? c->fuse_fwd : c->fuse_act) = on != 0;
    drop_graph(c);
    return RL_OK;
}

int32_t rl_get_forward_fused(rl_ctx* c, int32_t site) {
    if (!c || (site != 0 && site != 3)) return -1;
    return fused_on(c, site == 3) ? 1 : 0;
}

rl_status rl_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A, const void* B, float* C, void* stream) {
    if (M < 1 || N < 64 || N % 64 || K < 8 || K % 8 || !A || !B || !C) return RL_ERR_INVALID_ARG;
    if (!aligned16(A) || !aligned16(B) || !aligned16(C)) return RL_ERR_ALIGNMENT;
    TcParams tp;
    std::memset(&tp, 0, sizeof(tp));
    const int bn = N % 256 == 0 ? 256 : (N % 128 == 0 ? 128 : 64);
    const int cm = 1;
    if (!make_tmap_bf16(&tp.tmA[0], A, (uint64_t)M, (uint64_t)K, (uint64_t)K, 128)) return RL_ERR_CUDA;
    if (!make_tmap_bf16(&tp.tmB[0], B, (uint64_t)N, (uint64_t)K, (uint64_t)K, (uint32_t)bn)) return RL_ERR_CUDA;
    CK(tc_prepare());
    tp.M = M; tp.N = N; tp.kblocks = (K + 63) / 64; tp.kb_per_split = tp.kblocks; tp.splits = 1; tp.batch = 1;
    tp.bn = bn; tp.cm = cm; tp.epi = EPI_STORE;
    if (!make_tmap_out(&tp.tmC[0], C, true, 1, (uint64_t)M, (uint64_t)N, (uint64_t)N, 0)) return RL_ERR_CUDA;
    CK(launch_tc_gemm(tp, S_(stream)));
    return RL_OK;
}

rl_status rl_gemm_bf16_tn(int32_t M, int32_t N, int32_t K, const void* At, const void* Bt, float* C, void* stream) {
    if (M < 8 || M % 8 || N < 64 || N % 64 || K < 1 || !At || !Bt || !C) return RL_ERR_INVALID_ARG;
    if (!aligned16(At) || !aligned16(Bt) || !aligned16(C)) return RL_ERR_ALIGNMENT;
    TcParams tp;
    std::memset(&tp, 0, sizeof(tp));
    const int bn = N % 256 == 0 ? 256 : (N % 128 == 0 ? 128 : 64);
    const int cm = 1;
    // M a multiple of 64: one 3D copy per operand and stage
    tp.mn3 = (cm == 1 && M % 64 == 0) ? 1 : 0;
    if (!(tp.mn3 ? make_tmap_bf16_mn1(&tp.tmA[0], At, (uint64_t)K, (uint64_t)M, (uint64_t)M, 128)
                 : make_tmap_bf16(&tp.tmA[0], At, (uint64_t)K, (uint64_t)M, (uint64_t)M, 64)))
        return RL_ERR_CUDA;
    if (!(tp.mn3 ? make_tmap_bf16_mn1(&tp.tmB[0], Bt, (uint64_t)K, (uint64_t)N, (uint64_t)N, (uint32_t)bn)
                 : make_tmap_bf16(&tp.tmB[0], Bt, (uint64_t)K, (uint64_t)N, (uint64_t)N, 64)))
        return RL_ERR_CUDA;
    CK(tc_prepare());
    tp.M = M; tp.N = N; tp.kblocks = (K + 63) / 64; tp.kb_per_split = tp.kblocks; tp.splits = 1; tp.batch = 1;
    tp.bn = bn; tp.cm = cm; tp.mn = MAJ_MN; tp.epi = EPI_STORE;
    if (!make_tmap_out(&tp.tmC[0], C, true, 1, (uint64_t)M, (uint64_t)N, (uint64_t)N, 0)) return RL_ERR_CUDA;
    CK(launch_tc_gemm(tp, S_(stream)));
    return RL_OK;
}

rl_status rl_gemm_bf16_shape(int32_t M, int32_t N, int32_t K, const void* A, const void* B, float* C, int32_t operands,
                             int32_t bn, int32_t cluster, void* stream) {
    if (M < 1 || N < 64 || N % 64 || K < 1 || !A || !B || !C) return RL_ERR_INVALID_ARG;
    if (operands < 0 || operands > 3) return RL_ERR_INVALID_ARG;
    const bool k2 = operands >= 2;             // two K blocks per stage
    const bool mn = operands == 1 || operands == 3;
    if ((bn != 64 && bn != 128 && bn != 256) || N % bn || (cluster != 1 && cluster != 3)) return RL_ERR_INVALID_ARG;
    if (!mn && K % 8) return RL_ERR_INVALID_ARG;
    if (mn && M % 8) return RL_ERR_INVALID_ARG;
    if (cluster == 3 && bn < 128) return RL_ERR_INVALID_ARG;
    if (k2 && (cluster != 1 || bn > 128 || (!mn && K % 64) || (mn && M % 64))) return RL_ERR_INVALID_ARG;
    if (!aligned16(A) || !aligned16(B) || !aligned16(C)) return RL_ERR_ALIGNMENT;
    TcParams tp;
    std::memset(&tp, 0, sizeof(tp));
    const int cm = cluster == 1 ? 1 : 2;
    const int pair = cluster == 3 ? 1 : 0;
    const uint32_t brows = pair ? bn / 2 : bn;
    if (!mn) {
        const bool ok = k2 ? make_tmap_bf16_k2(&tp.tmA[0], A, (uint64_t)M, (uint64_t)K, (uint64_t)K, 128) &&
                                 make_tmap_bf16_k2(&tp.tmB[0], B, (uint64_t)N, (uint64_t)K, (uint64_t)K, (uint32_t)bn)
                           : make_tmap_bf16(&tp.tmA[0], A, (uint64_t)M, (uint64_t)K, (uint64_t)K, 128) &&
                                 make_tmap_bf16(&tp.tmB[0], B, (uint64_t)N, (uint64_t)K, (uint64_t)K, brows);
        if (!ok) return RL_ERR_CUDA;
        tp.mn = MAJ_K;
    } else {
        // single CTA, one K block per stage, M a multiple of 64: 3D maps, one copy per operand
        tp.mn3 = (!k2 && cluster == 1 && M % 64 == 0) ? 1 : 0;
        const bool ok = k2 ? make_tmap_bf16_mn2(&tp.tmA[0], A, (uint64_t)K, (uint64_t)M, (uint64_t)M, 128) &&
                                 make_tmap_bf16_mn2(&tp.tmB[0], B, (uint64_t)K, (uint64_t)N, (uint64_t)N, (uint32_t)bn)
                           : tp.mn3 ? make_tmap_bf16_mn1(&tp.tmA[0], A, (uint64_t)K, (uint64_t)M, (uint64_t)M, 128) &&
                                          make_tmap_bf16_mn1(&tp.tmB[0], B, (uint64_t)K, (uint64_t)N, (uint64_t)N, (uint32_t)bn)
                                    : make_tmap_bf16(&tp.tmA[0], A, (uint64_t)K, (uint64_t)M, (uint64_t)M, 64) &&
                                          make_tmap_bf16(&tp.tmB[0], B, (uint64_t)K, (uint64_t)N, (uint64_t)N, 64);
        if (!ok) return RL_ERR_CUDA;
        tp.mn = MAJ_MN;
    }
    CK(tc_prepare());
    tp.M = M; tp.N = N; tp.kblocks = (K + 63) / 64; tp.kb_per_split = tp.kblocks; tp.splits = 1; tp.batch = 1;
    tp.bn = bn; tp.cm = cm; tp.pair = pair; tp.epi = EPI_STORE; tp.ks = k2 ? 2 : 1;
    if (!make_tmap_out(&tp.tmC[0], C, true, 1, (uint64_t)M, (uint64_t)N, (uint64_t)N, 0)) return RL_ERR_CUDA;
    CK(launch_tc_gemm(tp, S_(stream)));
    return RL_OK;
}

int32_t rl_launches_per_iteration(rl_ctx* c) { return c ? c->launches : -1; }

}  // extern "C"

// ------------------------------------------------------------------------ grouped learners
struct rl_group {
    std::vector<rl_ctx*> ctx;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaStream_t s0 = nullptr;
    cudaEvent_t fork = nullptr, ev_in = nullptr, ev_out = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
};

extern "C" {

void rl_group_destroy(rl_group* g) {
    if (!g) return;
    cudaDeviceSynchronize();
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    if (g->graph) cudaGraphDestroy(g->graph);
    for (cudaStream_t s : g->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : g->joins) cudaEventDestroy(e);
    if (g->fork) cudaEventDestroy(g->fork);
    if (g->ev_in) cudaEventDestroy(g->ev_in);
    if (g->ev_out) cudaEventDestroy(g->ev_out);
    if (g->s0) cudaStreamDestroy(g->s0);
    for (rl_ctx* c : g->ctx) rl_destroy(c);
    delete g;
}

static rl_status group_setup(rl_group* g, int n) {
    CK(cudaStreamCreateWithFlags(&g->s0, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&g->ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&g->ev_out, cudaEventDisableTiming));
    for (int i = 0; i < n; ++i) {
        cudaStream_t s;
        cudaEvent_t e;
        CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        g->streams.push_back(s);
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        g->joins.push_back(e);
    }
    return RL_OK;
}

rl_status rl_group_create(int32_t n, const rl_config* cfgs, const float* const* heightfields,
                          const float* const* init_params, rl_group** out) {
    if (!out) return RL_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || n > 16 || !cfgs || !init_params) return RL_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (!config_ok(&cfgs[i]) || !init_params[i] ||
            (cfgs[i].grid_x * cfgs[i].grid_y > 0 && (!heightfields || !heightfields[i])))
            return RL_ERR_INVALID_ARG;
    rl_group* g = new rl_group();
    rl_status st = group_setup(g, n);
    for (int i = 0; i < n && st == RL_OK; ++i) {
        rl_ctx* c = nullptr;
        st = rl_create(&cfgs[i], heightfields ? heightfields[i] : nullptr, init_params[i], &c);
        if (st == RL_OK) g->ctx.push_back(c);
    }
    if (st != RL_OK) {
        rl_group_destroy(g);
        return st;
    }
    if (n > 1) {
        // the learners' branches run side by side: each learner's persistent GEMMs take at most
        // twice its share of the SMs (by robots), so that no learner's launch occupies every SM
        // while the others wait (measured on 8 learners of 512 ... 8192 robots: 23.9 -> 30.0 M
        // env-steps/s; one and three times the share were within 2 % of it)
        int sms = 148;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
        long long total = 0;
        for (rl_ctx* c : g->ctx) total += c->N;
        for (rl_ctx* c : g->ctx) {
            c->gemm_cap = (int)std::max(16ll, (2ll * sms * c->N + total - 1) / total);
            build_adam(c);
        }
    }
    *out = g;
    return RL_OK;
}

rl_ctx* rl_group_learner(rl_group* g, int32_t i) {
    if (!g || i < 0 || i >= (int)g->ctx.size()) return nullptr;
    return g->ctx[i];
}

rl_status rl_group_train_iteration(rl_group* g, int32_t use_graph, void* stream) {
    if (!g) return RL_ERR_INVALID_ARG;
    cudaStream_t s = S_(stream);
    if (!use_graph) {
        for (rl_ctx* c : g->ctx) {
            rl_status st = train_enqueue(c, s, false);
            if (st != RL_OK) return st;
        }
        return RL_OK;
    }
    CK(cudaEventRecord(g->ev_in, s));
    CK(cudaStreamWaitEvent(g->s0, g->ev_in, 0));
    if (!g->gexec) {
        // fork: every learner's iteration on its own stream, joined back into s0
        CK(cudaStreamBeginCapture(g->s0, cudaStreamCaptureModeThreadLocal));
        rl_status st = RL_OK;
        cudaError_t e = cudaEventRecord(g->fork, g->s0);
        for (size_t i = 0; i < g->ctx.size() && e == cudaSuccess && st == RL_OK; ++i) {
            e = cudaStreamWaitEvent(g->streams[i], g->fork, 0);
            if (e == cudaSuccess) st = train_enqueue(g->ctx[i], g->streams[i], false);
            if (e == cudaSuccess && st == RL_OK) e = cudaEventRecord(g->joins[i], g->streams[i]);
            if (e == cudaSuccess && st == RL_OK) e = cudaStreamWaitEvent(g->s0, g->joins[i], 0);
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(g->s0, &graph);
        if (st != RL_OK || e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return st != RL_OK ? st : err_of(e != cudaSuccess ? e : e2);
        }
        g->graph = graph;
        CK(cudaGraphInstantiate(&g->gexec, graph, 0));
    }
    CK(cudaGraphLaunch(g->gexec, g->s0));
    CK(cudaEventRecord(g->ev_out, g->s0));
    CK(cudaStreamWaitEvent(s, g->ev_out, 0));
    return RL_OK;
}

}  // extern "C"
