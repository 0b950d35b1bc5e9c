"""C ABI checks that need no GPU: the library loads, exports every entry point the header
declares, its config struct has the header's layout, and arguments are validated on the host
(invalid calls return a status and launch nothing)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2109_11978_b300 import _native as N
from paper_2109_11978_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rl_b300.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return N.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rl_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_four_hot_path_calls():
    names = declared_functions()
    for f in ("rl_env_step", "rl_policy_act", "rl_gae", "rl_ppo_update"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
        assert name in N.SIGNATURES, f"{name} has no binding"
    out = subprocess.run(["nm", "-D", "--defined-only", N.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (rl_[a-z0-9_]+)", out))
    assert set(names) <= exported


def test_config_struct_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "rl_b300.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(rl_config), offsetof(rl_config, seed),'
                   ' offsetof(rl_config, q_def), offsetof(rl_config, crash_threshold), offsetof(rl_config, gamma));'
                   'return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    C = N.rl_config
    want = [ctypes.sizeof(C), C.seed.offset, C.q_def.offset, C.crash_threshold.offset, C.gamma.offset]
    assert [int(x) for x in got] == want


def test_defaults_and_param_count(lib):
    cfg = N.default_config()
    assert (cfg.num_envs, cfg.num_steps, cfg.obs_dim, cfg.obs_pad, cfg.act_dim) == (4096, 24, 235, 256, 12)
    assert list(cfg.hidden)[:3] == [512, 256, 128] and cfg.num_hidden == 3
    assert abs(cfg.gamma - 0.99) < 1e-7 and abs(cfg.lam - 0.95) < 1e-7 and abs(cfg.clip - 0.2) < 1e-7
    assert (cfg.epochs, cfg.minibatches) == (5, 4)
    # actor 286,616 incl. log-std + critic 285,185 at obs 235, 512-256-128
    assert lib.rl_param_count(ctypes.byref(cfg)) == 571801
    from oracle import mlp
    assert mlp.param_count(235, (512, 256, 128), 12) == 571801


@pytest.mark.parametrize("field,value", [
    ("num_envs", 0), ("act_dim", 6), ("obs_dim", 100), ("obs_pad", 250), ("num_hidden", 0),
    ("precision", 7), ("minibatches", 5), ("decimation", 0), ("hf_res", 0.0), ("tile_size", 8.05),
])
def test_invalid_config_rejected_on_host(lib, field, value):
    cfg = N.default_config()
    setattr(cfg, field, value)
    hf = np.zeros((800, 1600), np.float32)
    params = np.zeros(571801 + 10000, np.float32)
    out = ctypes.c_void_p()
    st = lib.rl_create(ctypes.byref(cfg), hf.ctypes.data_as(ctypes.c_void_p), params.ctypes.data_as(ctypes.c_void_p),
                       ctypes.byref(out))
    assert st == N.RL_ERR_INVALID_ARG and not out.value


def test_null_arguments_rejected(lib):
    assert lib.rl_env_step(None, 0, None, None, None, None, None, None, None, None, None) == N.RL_ERR_INVALID_ARG
    assert lib.rl_policy_act(None, 0, 1, None, None, None, None, None, None) == N.RL_ERR_INVALID_ARG
    assert lib.rl_ppo_update(None, None, None, None, None, None, None, None, 1, 1, 0.2, None, None) == N.RL_ERR_INVALID_ARG
    assert lib.rl_gae(0, 5, 0.99, 0.95, None, None, None, None, None, None, 0, None, None, 0, None) == N.RL_ERR_INVALID_ARG
    assert lib.rl_gae_workspace_bytes(24, 4096) == (4096 // 256 + 1) * 16
    assert lib.rl_gae_workspace_bytes(0, 4096) == 0
    assert lib.rl_status_string(N.RL_ERR_TIMEOUT) == b"device wait timed out"
    lib.rl_destroy(None)


def test_create_without_gpu_reports_cuda_error(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    cfg = N.default_config(num_envs=64, num_steps=24, hidden=[64, 64], minibatches=2, grid_x=0, grid_y=0,
                           obs_dim=48, obs_pad=64)
    n = lib.rl_param_count(ctypes.byref(cfg))
    params = np.zeros(n, np.float32)
    out = ctypes.c_void_p()
    st = lib.rl_create(ctypes.byref(cfg), None, params.ctypes.data_as(ctypes.c_void_p), ctypes.byref(out))
    assert st in (N.RL_ERR_CUDA, N.RL_ERR_INVALID_ARG) and not out.value
