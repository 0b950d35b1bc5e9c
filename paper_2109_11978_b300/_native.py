"""ctypes binding of the C ABI declared in include/rl_b300.h (argument marshalling only).

Every function here forwards to the CUDA library; nothing computes on the host.  The library
is the in-tree build ``_lib/librl_b300.so``; importing this module without it raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "librl_b300.so")

RL_OK = 0
RL_ERR_INVALID_ARG = -1
RL_ERR_ALIGNMENT = -2
RL_ERR_CUDA = -3
RL_ERR_TIMEOUT = -4
RL_ERR_STATE = -5
RL_ERR_OOM = -6
RL_ERR_UNSUPPORTED = -7
RL_FP32 = 0
RL_BF16 = 1
RL_PROF_GEMM, RL_PROF_LOSS, RL_PROF_ADAM, RL_PROF_ENV, RL_PROF_ACT, RL_PROF_GATHER, RL_PROF_OTHER, RL_PROF_ALL = range(8)
RL_PROF_NAMES = ("gemm", "loss_head", "adam", "env_step", "act_head", "gather", "other")
RL_NF = 57
RL_ACT_INPUTS, RL_ACT_HIDDEN = 2, 32
RL_ACT_WEIGHTS = 4 * 32 * 2 + 4 * 32 * 32 + 4 * 32 + 32 + 1
RL_NI = 3
RL_NSTATS = 16


class rl_config(ctypes.Structure):
    _fields_ = [
        ("num_envs", ctypes.c_int32), ("num_steps", ctypes.c_int32), ("obs_dim", ctypes.c_int32),
        ("obs_pad", ctypes.c_int32), ("act_dim", ctypes.c_int32), ("num_hidden", ctypes.c_int32),
        ("hidden", ctypes.c_int32 * 4),
        ("gamma", ctypes.c_float), ("lam", ctypes.c_float), ("clip", ctypes.c_float),
        ("entropy_coef", ctypes.c_float), ("value_coef", ctypes.c_float), ("kl_target", ctypes.c_float),
        ("lr_init", ctypes.c_float), ("lr_min", ctypes.c_float), ("lr_max", ctypes.c_float),
        ("epochs", ctypes.c_int32), ("minibatches", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("kp", ctypes.c_float), ("kd", ctypes.c_float), ("action_scale", ctypes.c_float), ("dt", ctypes.c_float),
        ("sim_dt", ctypes.c_float), ("decimation", ctypes.c_int32), ("max_episode_len", ctypes.c_int32),
        ("num_levels", ctypes.c_int32), ("num_cols", ctypes.c_int32), ("tile_size", ctypes.c_float),
        ("hf_res", ctypes.c_float), ("grid_x", ctypes.c_int32), ("grid_y", ctypes.c_int32),
        ("grid_spacing", ctypes.c_float), ("noise_on", ctypes.c_int32), ("push_on", ctypes.c_int32),
        ("push_interval", ctypes.c_int32), ("push_vel", ctypes.c_float), ("cmd_range", ctypes.c_float * 3),
        ("crash_threshold", ctypes.c_uint32), ("q_def", ctypes.c_float * 12), ("reserved", ctypes.c_int32 * 2),
        ("seed", ctypes.c_uint64),
    ]


class RLError(RuntimeError):
    pass


_lib = None
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_f32 = ctypes.c_float

# name -> (restype, argtypes), exactly the entry points of include/rl_b300.h
SIGNATURES = {
    "rl_config_default": (None, [ctypes.POINTER(rl_config)]),
    "rl_param_count": (ctypes.c_int64, [ctypes.POINTER(rl_config)]),
    "rl_status_string": (ctypes.c_char_p, [_i32]),
    "rl_create": (_i32, [ctypes.POINTER(rl_config), _vp, _vp, ctypes.POINTER(_vp)]),
    "rl_destroy": (None, [_vp]),
    "rl_get_params": (_i32, [_vp, _vp, _vp]),
    "rl_set_params": (_i32, [_vp, _vp, _vp]),
    "rl_get_adam_moments": (_i32, [_vp, _vp, _vp, _vp]),
    "rl_get_scalars": (_i32, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "rl_set_scalars": (_i32, [_vp, ctypes.c_double, ctypes.c_int64, ctypes.c_int64, _vp]),
    "rl_actuator_lstm_step": (_i32, [_i32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "rl_terrain_generate": (_i32, [ctypes.POINTER(rl_config), _vp, _vp]),
    "rl_checkpoint_bytes": (ctypes.c_int64, [_vp]),
    "rl_checkpoint_save": (_i32, [_vp, _vp, ctypes.c_size_t, _vp]),
    "rl_checkpoint_load": (_i32, [_vp, _vp, ctypes.c_size_t, _vp]),
    "rl_env_get_state": (_i32, [_vp, _vp, _vp, _vp]),
    "rl_env_set_state": (_i32, [_vp, _vp, _vp, _vp]),
    "rl_env_reset_all": (_i32, [_vp, _vp, _vp]),
    "rl_env_step": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "rl_policy_act": (_i32, [_vp, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "rl_gae_workspace_bytes": (ctypes.c_size_t, [_i32, _i32]),
    "rl_gae": (_i32, [_i32, _i32, _f32, _f32, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp, _vp, ctypes.c_size_t, _vp]),
    "rl_gae_noalloc": (_i32, [_i32, _i32, _f32, _f32, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp, _vp]),
    "rl_ppo_update": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _i32, _f32, _vp, _vp]),
    "rl_ppo_loss_grad": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "rl_train_iteration": (_i32, [_vp, _i32, _vp, _vp]),
    "rl_get_storage": (_i32, [_vp, _i32, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_size_t)]),
    "rl_last_device_status": (_i32, [_vp]),
    "rl_clear_device_status": (_i32, [_vp, _vp]),
    "rl_diag_forced_timeout": (_i32, [_vp, _vp]),
    "rl_profile_enable": (_i32, [_vp, _i32, _i32]),
    "rl_profile_read": (_i32, [_vp, ctypes.POINTER(_f32), ctypes.POINTER(_i32)]),
    "rl_profile_read_class": (_i32, [_vp, _i32, ctypes.POINTER(_f32), ctypes.POINTER(_i32)]),
    "rl_launches_per_iteration": (_i32, [_vp]),
    "rl_autotune": (_i32, [_vp, ctypes.c_char_p, ctypes.c_size_t, _vp]),
    "rl_set_gemm_tiles": (_i32, [_vp, _i32, _i32, _i32, _i32, _i32]),
    "rl_set_gemm_ctas": (_i32, [_vp, _i32]),
    "rl_set_forward_fused": (_i32, [_vp, _i32, _i32]),
    "rl_get_forward_fused": (_i32, [_vp, _i32]),
    "rl_adam_step": (_i32, [ctypes.c_int64, _vp, _vp, _i32, _vp, _vp, _f32, _i32, _vp, _vp]),
    "rl_gemm_bf16": (_i32, [_i32, _i32, _i32, _vp, _vp, _vp, _vp]),
    "rl_gemm_bf16_tn": (_i32, [_i32, _i32, _i32, _vp, _vp, _vp, _vp]),
    "rl_gemm_bf16_shape": (_i32, [_i32, _i32, _i32, _vp, _vp, _vp, _i32, _i32, _i32, _vp]),
    "rl_group_create": (_i32, [_i32, ctypes.POINTER(rl_config), ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
    "rl_group_destroy": (None, [_vp]),
    "rl_group_learner": (_vp, [_vp, _i32]),
    "rl_group_train_iteration": (_i32, [_vp, _i32, _vp]),
}


def lib():
    """The loaded library (raises if the in-tree build is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RLError(f"CUDA library not built: {LIB_PATH} (run paper_2109_11978_b300.build)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status, what=""):
    if status != RL_OK:
        msg = lib().rl_status_string(status).decode()
        raise RLError(f"{what}: {msg} ({status})")
    return status


def default_config(**overrides):
    cfg = rl_config()
    lib().rl_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        if k == "hidden":
            cfg.num_hidden = len(v)
            for i in range(4):
                cfg.hidden[i] = v[i] if i < len(v) else 0
        elif k in ("cmd_range", "q_def"):
            arr = getattr(cfg, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(cfg, k, v)
    return cfg
