"""Python binding of the C ABI with the same names, taking torch CUDA tensors.

Argument marshalling only: every function checks shapes/dtypes, passes data pointers and the
current CUDA stream to the library entry point of the same name, and raises RLError on a
non-OK status.  PyTorch provides device memory and streams; all arithmetic runs in the
library's kernels.
"""
import ctypes

import torch

from . import _native as N
from ._native import RLError, check, default_config, lib  # noqa: F401
from ._native import (RL_PROF_ACT, RL_PROF_ADAM, RL_PROF_ALL, RL_PROF_ENV, RL_PROF_GATHER, RL_PROF_GEMM,  # noqa: F401
                      RL_PROF_LOSS, RL_PROF_NAMES, RL_PROF_OTHER)

RL_FP32, RL_BF16, RL_NF, RL_NI, RL_NSTATS = N.RL_FP32, N.RL_BF16, N.RL_NF, N.RL_NI, N.RL_NSTATS


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise RLError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise RLError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _ptr_any(t):
    """A contiguous CUDA or host tensor (the env-state calls take either)."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise RLError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def rl_param_count(cfg):
    return int(lib().rl_param_count(ctypes.byref(cfg)))


def rl_create(cfg, heightfield, init_params):
    """heightfield: host float32 array/tensor or None; init_params: host float32 (flat layout)."""
    import numpy as np
    hf = None if heightfield is None else np.ascontiguousarray(heightfield, dtype=np.float32)
    ip = np.ascontiguousarray(init_params, dtype=np.float32)
    if ip.size != rl_param_count(cfg):
        raise RLError(f"init_params has {ip.size} values, layout needs {rl_param_count(cfg)}")
    out = ctypes.c_void_p()
    check(lib().rl_create(ctypes.byref(cfg), None if hf is None else hf.ctypes.data_as(ctypes.c_void_p),
                          ip.ctypes.data_as(ctypes.c_void_p), ctypes.byref(out)), "rl_create")
    return out


def rl_destroy(ctx):
    lib().rl_destroy(ctx)


def rl_get_params(ctx, out):
    check(lib().rl_get_params(ctx, _ptr(out), _stream()), "rl_get_params")


def rl_set_params(ctx, params):
    check(lib().rl_set_params(ctx, _ptr(params), _stream()), "rl_set_params")


def rl_get_adam_moments(ctx, m_out, v_out):
    check(lib().rl_get_adam_moments(ctx, _ptr(m_out), _ptr(v_out), _stream()), "rl_get_adam_moments")


def rl_get_scalars(ctx):
    arr = (ctypes.c_double * 4)()
    check(lib().rl_get_scalars(ctx, arr), "rl_get_scalars")
    return {"alpha": arr[0], "iteration": int(arr[1]), "adam_step": int(arr[2]), "kl": arr[3]}


def rl_set_scalars(ctx, alpha, iteration, adam_step):
    check(lib().rl_set_scalars(ctx, float(alpha), int(iteration), int(adam_step), _stream()), "rl_set_scalars")


def rl_actuator_lstm_step(weights, x, h, c, tau):
    """One LSTM actuator step for x.shape[0] joints (CUDA fp32 tensors; h, c updated in place)."""
    n = x.shape[0]
    if weights.numel() != N.RL_ACT_WEIGHTS or tuple(x.shape) != (n, N.RL_ACT_INPUTS) or \
            tuple(h.shape) != (n, N.RL_ACT_HIDDEN) or tuple(c.shape) != (n, N.RL_ACT_HIDDEN) or tau.numel() != n:
        raise RLError("rl_actuator_lstm_step: shapes")
    for t in (weights, x, h, c, tau):
        if t.dtype != torch.float32:
            raise RLError("rl_actuator_lstm_step: float32 tensors")
    check(lib().rl_actuator_lstm_step(int(n), _ptr(weights), _ptr(x), _ptr(h), _ptr(c), _ptr(tau), _stream()),
          "rl_actuator_lstm_step")


def rl_terrain_generate(cfg):
    """The procedural terrain family for cfg as a CUDA fp32 tensor [num_levels c][num_cols c]."""
    c = int(round(cfg.tile_size / cfg.hf_res))
    out = torch.empty((cfg.num_levels * c, cfg.num_cols * c), dtype=torch.float32, device="cuda")
    check(lib().rl_terrain_generate(ctypes.byref(cfg), _ptr(out), _stream()), "rl_terrain_generate")
    return out


def rl_checkpoint_bytes(ctx):
    return int(lib().rl_checkpoint_bytes(ctx))


def rl_checkpoint_save(ctx):
    """The learner's checkpoint image as a host uint8 tensor."""
    buf = torch.empty(rl_checkpoint_bytes(ctx), dtype=torch.uint8)
    check(lib().rl_checkpoint_save(ctx, buf.data_ptr(), buf.numel(), _stream()), "rl_checkpoint_save")
    return buf


def rl_checkpoint_load(ctx, image):
    buf = image.contiguous()
    if buf.dtype != torch.uint8 or buf.is_cuda:
        raise RLError("rl_checkpoint_load: the image is a host uint8 tensor")
    check(lib().rl_checkpoint_load(ctx, buf.data_ptr(), buf.numel(), _stream()), "rl_checkpoint_load")


def rl_env_get_state(ctx, sf, si):
    check(lib().rl_env_get_state(ctx, _ptr_any(sf), _ptr_any(si), _stream()), "rl_env_get_state")


def rl_env_set_state(ctx, sf, si):
    check(lib().rl_env_set_state(ctx, _ptr_any(sf), _ptr_any(si), _stream()), "rl_env_set_state")


def rl_env_reset_all(ctx, obs_out=None):
    check(lib().rl_env_reset_all(ctx, _ptr(obs_out), _stream()), "rl_env_reset_all")


def rl_env_step(ctx, t, actions, values, obs_out, rew_out, done_out=None, timeout_out=None, level_out=None,
                terrain_idx_out=None):
    check(lib().rl_env_step(ctx, int(t), _ptr(actions), _ptr(values), _ptr(obs_out), _ptr(rew_out), _ptr(done_out),
                            _ptr(timeout_out), _ptr(level_out), _ptr(terrain_idx_out), _stream()), "rl_env_step")


def rl_policy_act(ctx, t, obs, actions, mu, logp, values):
    n = obs.shape[0]
    check(lib().rl_policy_act(ctx, int(t), int(n), _ptr(obs), _ptr(actions), _ptr(mu), _ptr(logp), _ptr(values),
                              _stream()), "rl_policy_act")


def rl_gae_workspace_bytes(T, N):
    return int(lib().rl_gae_workspace_bytes(int(T), int(N)))


def rl_gae(gamma, lam, rew, val, last_val, done, adv_out, ret_out, normalize=False, adv_stats_out=None,
           workspace=None):
    T, Nn = rew.shape
    wb = 0 if workspace is None else workspace.numel() * workspace.element_size()
    check(lib().rl_gae(T, Nn, float(gamma), float(lam), _ptr(rew), _ptr(val), _ptr(last_val), _ptr(done),
                       _ptr(adv_out), _ptr(ret_out), int(bool(normalize)), _ptr(adv_stats_out), _ptr(workspace), wb,
                       _stream()), "rl_gae")


def rl_gae_noalloc(gamma, lam, rew, val, last_val, done, adv_out, ret_out, normalize=False, adv_stats_out=None):
    """rl_gae with its scratch in the library's static device array: no allocation anywhere
    (for callers that cannot allocate device memory); N <= 262144, overlapping calls race."""
    T, Nn = rew.shape
    check(lib().rl_gae_noalloc(T, Nn, float(gamma), float(lam), _ptr(rew), _ptr(val), _ptr(last_val), _ptr(done),
                               _ptr(adv_out), _ptr(ret_out), int(bool(normalize)), _ptr(adv_stats_out), _stream()),
          "rl_gae_noalloc")


def rl_ppo_update(ctx, obs, actions, logp_old, mu_old, val_old, adv, ret, epochs, minibatches, clip, stats_out=None):
    check(lib().rl_ppo_update(ctx, _ptr(obs), _ptr(actions), _ptr(logp_old), _ptr(mu_old), _ptr(val_old), _ptr(adv),
                              _ptr(ret), int(epochs), int(minibatches), float(clip), _ptr(stats_out), _stream()),
          "rl_ppo_update")


def rl_ppo_loss_grad(ctx, obs, actions, logp_old, mu_old, log_std_old, val_old, adv, ret, grad_out, stats_out=None):
    M = obs.shape[0]
    check(lib().rl_ppo_loss_grad(ctx, int(M), _ptr(obs), _ptr(actions), _ptr(logp_old), _ptr(mu_old), _ptr(log_std_old),
                                 _ptr(val_old), _ptr(adv), _ptr(ret), _ptr(grad_out), _ptr(stats_out), _stream()),
          "rl_ppo_loss_grad")


def rl_train_iteration(ctx, use_graph=True, stats_host=None):
    """stats_host: optional pinned CPU float32 tensor of RL_NSTATS values (filled, synchronising)."""
    p = None
    if stats_host is not None:
        if stats_host.is_cuda or stats_host.dtype != torch.float32 or stats_host.numel() < RL_NSTATS:
            raise RLError("stats_host must be a CPU float32 tensor of RL_NSTATS values")
        p = ctypes.c_void_p(stats_host.data_ptr())
    check(lib().rl_train_iteration(ctx, int(bool(use_graph)), p, _stream()), "rl_train_iteration")


def rl_get_storage(ctx, which):
    ptr, nbytes = ctypes.c_void_p(), ctypes.c_size_t()
    check(lib().rl_get_storage(ctx, int(which), ctypes.byref(ptr), ctypes.byref(nbytes)), "rl_get_storage")
    return ptr.value, nbytes.value


def rl_last_device_status(ctx):
    return int(lib().rl_last_device_status(ctx))


def rl_clear_device_status(ctx):
    """Resets the device status word to RL_OK (on the current stream)."""
    check(lib().rl_clear_device_status(ctx, _stream()), "rl_clear_device_status")


def rl_diag_forced_timeout(ctx):
    """Launches one warp whose bounded wait runs out (2 s), recording RL_ERR_TIMEOUT."""
    check(lib().rl_diag_forced_timeout(ctx, _stream()), "rl_diag_forced_timeout")


def rl_profile_enable(ctx, kernel_class=0, on=True):
    check(lib().rl_profile_enable(ctx, int(kernel_class), int(bool(on))), "rl_profile_enable")


def rl_profile_read_class(ctx, kernel_class):
    ms, n = ctypes.c_float(), ctypes.c_int32()
    check(lib().rl_profile_read_class(ctx, int(kernel_class), ctypes.byref(ms), ctypes.byref(n)), "rl_profile_read_class")
    return ms.value, n.value


def rl_profile_read(ctx):
    ms, n = ctypes.c_float(), ctypes.c_int32()
    check(lib().rl_profile_read(ctx, ctypes.byref(ms), ctypes.byref(n)), "rl_profile_read")
    return ms.value, n.value


def rl_autotune(ctx):
    """Times the update's GEMM sites over candidate tile shapes and keeps the fastest; returns the
    report (dict)."""
    import json
    buf = ctypes.create_string_buffer(65536)
    check(lib().rl_autotune(ctx, buf, len(buf), _stream()), "rl_autotune")
    return json.loads(buf.value.decode() or "{}")


def rl_adam_step(p, g, m, v, lr, t, nsplit=1, bf16_out=None):
    """One Adam step on device tensors (g holds nsplit partial sums of len(p) each)."""
    n = p.numel()
    check(lib().rl_adam_step(ctypes.c_int64(n), _ptr(p), _ptr(g), int(nsplit), _ptr(m), _ptr(v), float(lr), int(t),
                             _ptr(bf16_out), _stream()), "rl_adam_step")


def rl_set_gemm_ctas(ctx, max_ctas):
    """Caps the persistent CTAs of the context's GEMM launches (0: one per SM)."""
    check(lib().rl_set_gemm_ctas(ctx, int(max_ctas)), "rl_set_gemm_ctas")


def rl_set_gemm_tiles(ctx, site, layer, bn, cluster=1, splits=1):
    """Pins one GEMM site's tile shape (site 0 forward, 1 input gradient, 2 weight gradient)."""
    check(lib().rl_set_gemm_tiles(ctx, int(site), int(layer), int(bn), int(cluster), int(splits)), "rl_set_gemm_tiles")


def rl_set_forward_fused(ctx, site, on):
    """The three hidden layers' forward as one fused launch (site 0 the update's, 3 the rollout's)."""
    check(lib().rl_set_forward_fused(ctx, int(site), int(bool(on))), "rl_set_forward_fused")


def rl_get_forward_fused(ctx, site):
    """1 if the site's forward runs fused, 0 if layer by layer."""
    r = int(lib().rl_get_forward_fused(ctx, int(site)))
    if r < 0:
        raise RLError("rl_get_forward_fused: invalid context or site")
    return r


def rl_gemm_bf16(A, B, C):
    """C[M][N] (fp32) = A[M][K] (bf16) @ B[N][K]^T (bf16) on the tcgen05 tensor-core kernel."""
    M, K = A.shape
    Nn = B.shape[0]
    check(lib().rl_gemm_bf16(int(M), int(Nn), int(K), _ptr(A), _ptr(B), _ptr(C), _stream()), "rl_gemm_bf16")


def rl_gemm_bf16_tn(At, Bt, C):
    """C[M][N] (fp32) = At[K][M]^T (bf16) @ Bt[K][N] (bf16), operands read MN-major."""
    K, M = At.shape
    Nn = Bt.shape[1]
    check(lib().rl_gemm_bf16_tn(int(M), int(Nn), int(K), _ptr(At), _ptr(Bt), _ptr(C), _stream()), "rl_gemm_bf16_tn")


def rl_gemm_bf16_shape(A, B, C, operands=0, bn=128, cluster=1):
    """C = A B^T (operands 0: A [M][K], B [N][K]) or At^T Bt (operands 1: At [K][M], Bt [K][N]) with an
    explicit tile width and cluster mode (1 single CTA, 3 cta_group::2 pair);
    operands 2 / 3: the same forms with two K blocks per pipeline stage (cluster 1, bn <= 128)."""
    if operands in (0, 2):
        M, K = A.shape
        Nn = B.shape[0]
    else:
        K, M = A.shape
        Nn = B.shape[1]
    check(lib().rl_gemm_bf16_shape(int(M), int(Nn), int(K), _ptr(A), _ptr(B), _ptr(C), int(operands), int(bn), int(cluster),
                                   _stream()), "rl_gemm_bf16_shape")


def rl_launches_per_iteration(ctx):
    return int(lib().rl_launches_per_iteration(ctx))


def rl_group_create(cfgs, heightfields, init_params):
    """cfgs: list of rl_config; heightfields / init_params: lists of host float32 arrays."""
    import numpy as np
    n = len(cfgs)
    arr = (N.rl_config * n)(*cfgs)
    hfs = [None if h is None else np.ascontiguousarray(h, dtype=np.float32) for h in heightfields]
    ips = [np.ascontiguousarray(x, dtype=np.float32) for x in init_params]
    for c, x in zip(cfgs, ips):
        if x.size != rl_param_count(c):
            raise RLError("init_params size does not match its config")
    hp = (ctypes.c_void_p * n)(*[None if h is None else h.ctypes.data for h in hfs])
    ip = (ctypes.c_void_p * n)(*[x.ctypes.data for x in ips])
    out = ctypes.c_void_p()
    check(lib().rl_group_create(n, arr, hp, ip, ctypes.byref(out)), "rl_group_create")
    return out


def rl_group_destroy(group):
    lib().rl_group_destroy(group)


def rl_group_learner(group, i):
    return ctypes.c_void_p(lib().rl_group_learner(group, int(i)))


def rl_group_train_iteration(group, use_graph=True):
    check(lib().rl_group_train_iteration(group, int(bool(use_graph)), _stream()), "rl_group_train_iteration")


# ------------------------------------------------------------------------------------------
class Learner:
    """One learner (context) with torch views of its rollout storage.  Marshalling only."""

    STORAGE = {0: "obs", 1: "actions", 2: "mu", 3: "logp", 4: "values", 5: "rewards", 6: "dones", 7: "timeouts",
               8: "last_values", 9: "advantages", 10: "returns", 11: "levels", 12: "stats", 13: "permutations",
               14: "update_trace"}

    def __init__(self, cfg, heightfield, init_params):
        if not torch.cuda.is_available():
            raise RLError("a CUDA device is required")
        self.cfg = cfg
        self.ctx = rl_create(cfg, heightfield, init_params)
        self.n_params = rl_param_count(cfg)

    def close(self):
        if self.ctx is not None:
            rl_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def storage(self, which):
        """Torch tensor aliasing context-owned storage `which` (see rl_get_storage)."""
        c = self.cfg
        ptr, nbytes = rl_get_storage(self.ctx, which)
        T, Nn, A, Op = c.num_steps, c.num_envs, c.act_dim, c.obs_pad
        obs_dt = torch.bfloat16 if c.precision == RL_BF16 else torch.float32
        shapes = {0: ((T + 1, Nn, Op), obs_dt), 1: ((T, Nn, A), torch.float32), 2: ((T, Nn, A), torch.float32),
                  3: ((T, Nn), torch.float32), 4: ((T, Nn), torch.float32), 5: ((T, Nn), torch.float32),
                  6: ((T, Nn), torch.uint8), 7: ((T, Nn), torch.uint8), 8: ((Nn,), torch.float32),
                  9: ((T, Nn), torch.float32), 10: ((T, Nn), torch.float32), 11: ((Nn,), torch.int32),
                  12: ((RL_NSTATS,), torch.float32), 13: ((c.epochs, T * Nn), torch.int32),
                  14: ((c.epochs * c.minibatches, 2), torch.float32)}
        shape, dt = shapes[which]
        return _alias(ptr, shape, dt)

    def params(self):
        out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        rl_get_params(self.ctx, out)
        return out

    def adam_moments(self):
        m = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        v = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        rl_get_adam_moments(self.ctx, m, v)
        return m, v

    def set_params(self, p):
        rl_set_params(self.ctx, p.contiguous())

    def get_state(self):
        sf = torch.empty((RL_NF, self.cfg.num_envs), dtype=torch.float32, device="cuda")
        si = torch.empty((RL_NI, self.cfg.num_envs), dtype=torch.int32, device="cuda")
        rl_env_get_state(self.ctx, sf, si)
        return sf, si

    def set_state(self, sf, si):
        rl_env_set_state(self.ctx, sf.contiguous(), si.contiguous())

    def train_iteration(self, use_graph=True, stats_host=None):
        rl_train_iteration(self.ctx, use_graph, stats_host)


def _alias(ptr, shape, dtype):
    """A torch tensor over existing device memory (no copy, no ownership)."""
    numel = 1
    for s in shape:
        numel *= s
    esz = torch.tensor([], dtype=dtype).element_size()

    class _Mem:
        __cuda_array_interface__ = {
            "shape": (numel * esz,), "typestr": "|u1", "data": (ptr, False), "version": 3, "strides": None,
        }

    raw = torch.as_tensor(_Mem(), device="cuda")
    return raw.view(dtype).view(*shape)
