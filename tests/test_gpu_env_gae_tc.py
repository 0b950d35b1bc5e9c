"""GPU parity (through the C ABI) of the tensor-core GEMM, the env step and GAE against the
FP64 oracle.

* tcgen05 BF16 GEMM: against float64 products of the same bf16 values, several tiles, ragged M
  and K, all tile widths;
* env step: the fp32 stand-in state bit-exact, done / time-out / level / terrain index
  bit-exact, reward and observation within 1e-5 (norm-wise), on diverse states with ragged
  robot counts, for one step and for 8 chained steps (no teacher forcing of the state: both
  sides evolve their own state from the same start and the same actions); bf16 observations
  within bf16 rounding; the initial spawn;
* GAE: advantages, returns, normalisation statistics within 1e-5, ragged N, T = 1.
"""
import numpy as np
import pytest
import torch

from oracle import env as OE
from oracle import gae as OG
from oracle import train as OT
from paper_2109_11978_b300 import api, synth
from tests.helpers import TOL_FP32, lib_config, obs_dims, oracle_env_config, rel_err, workload

pytestmark = pytest.mark.gpu


def _bf16_round(x):
    return torch.as_tensor(np.asarray(x, np.float32)).to(torch.bfloat16).float().numpy()


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (300, 128, 256), (1000, 192, 72), (4096, 512, 256),
                                   (24576, 256, 512), (77, 256, 128)])
def test_tc_gemm_matches_fp64(M, N, K):
    g = torch.Generator().manual_seed(M + N + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    C = torch.full((M, N), float("nan"), device="cuda")
    api.rl_gemm_bf16(A.cuda(), B.cuda(), C)
    torch.cuda.synchronize()
    ref = A.double().numpy() @ B.double().numpy().T
    err = np.abs(C.cpu().double().numpy() - ref).max() / np.abs(ref).max()
    assert err < 2e-6, err


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (64, 128, 1000), (512, 256, 24576), (256, 512, 3000),
                                   (136, 192, 72), (8, 64, 5)])
def test_tc_gemm_mn_major_matches_fp64(M, N, K):
    """The weight-gradient form (both operands MN-major: K rows of M and N contiguous values),
    ragged in M (not a multiple of 128) and K (not a multiple of 64)."""
    g = torch.Generator().manual_seed(7 * M + N + K)
    At = torch.randn(K, M, generator=g).to(torch.bfloat16)
    Bt = torch.randn(K, N, generator=g).to(torch.bfloat16)
    C = torch.full((M, N), float("nan"), device="cuda")
    api.rl_gemm_bf16_tn(At.cuda(), Bt.cuda(), C)
    torch.cuda.synchronize()
    ref = At.double().numpy().T @ Bt.double().numpy()
    err = np.abs(C.cpu().double().numpy() - ref).max() / np.abs(ref).max()
    # FP32 accumulation in tensor memory, one rounding per 16-product block: the error of a sum
    # of K random products grows like sqrt(K)
    assert err < max(2e-6, 5e-7 * np.sqrt(K)), err


@pytest.mark.parametrize("operands,bn,cluster", [(0, 64, 1), (0, 256, 1), (0, 256, 3), (0, 128, 3), (1, 128, 1),
                                                 (1, 256, 1), (1, 256, 3), (1, 128, 3)])
@pytest.mark.parametrize("M,N,K", [(300, 512, 200), (1024, 256, 1000)])
def test_tc_gemm_tile_modes(operands, bn, cluster, M, N, K):
    """Every cluster mode of the tensor-core GEMM on both operand forms, with a ragged row count
    (the last pair has a CTA past the rows) and a ragged K: cluster 1 is one CTA per tile, cluster
    3 runs 256-row tiles on the cta_group::2 MMA with half of B in each CTA."""
    g = torch.Generator().manual_seed(M + 3 * N + K + bn + 11 * cluster + 97 * operands)
    if operands == 0:
        K8 = (K + 7) // 8 * 8
        A = torch.randn(M, K8, generator=g).to(torch.bfloat16)
        B = torch.randn(N, K8, generator=g).to(torch.bfloat16)
        ref = A.double().numpy() @ B.double().numpy().T
    else:
        M8 = (M + 7) // 8 * 8
        A = torch.randn(K, M8, generator=g).to(torch.bfloat16)
        B = torch.randn(K, N, generator=g).to(torch.bfloat16)
        ref = A.double().numpy().T @ B.double().numpy()
    C = torch.full(ref.shape, float("nan"), device="cuda")
    api.rl_gemm_bf16_shape(A.cuda(), B.cuda(), C, operands, bn, cluster)
    torch.cuda.synchronize()
    err = np.abs(C.cpu().double().numpy() - ref).max() / np.abs(ref).max()
    k_len = A.shape[1] if operands == 0 else A.shape[0]
    assert err < max(2e-6, 5e-7 * np.sqrt(k_len)), err     # FP32 accumulation, one rounding per 16 products


@pytest.mark.parametrize("operands,bn", [(2, 64), (2, 128), (3, 64), (3, 128)])
@pytest.mark.parametrize("M,N,K", [(300, 512, 192), (64, 128, 64), (1024, 256, 1088), (320, 128, 200), (512, 256, 24576)])
def test_tc_gemm_two_block_stages(operands, bn, M, N, K):
    """Stages of two K blocks (one 3D copy per operand): an odd K-block count multiplies only the
    first half of the last stage; K-major forms need whole 64-column K chunks, MN-major forms whole
    64-wide M chunks, so the ragged dimension is M (K-major) or K (MN-major)."""
    if operands == 3:
        M = (M + 63) // 64 * 64
    else:
        K = (K + 63) // 64 * 64
    g = torch.Generator().manual_seed(M + 5 * N + K + bn + 131 * operands)
    if operands == 2:
        A = torch.randn(M, K, generator=g).to(torch.bfloat16)
        B = torch.randn(N, K, generator=g).to(torch.bfloat16)
        ref = A.double().numpy() @ B.double().numpy().T
    else:
        A = torch.randn(K, M, generator=g).to(torch.bfloat16)
        B = torch.randn(K, N, generator=g).to(torch.bfloat16)
        ref = A.double().numpy().T @ B.double().numpy()
    C = torch.full(ref.shape, float("nan"), device="cuda")
    api.rl_gemm_bf16_shape(A.cuda(), B.cuda(), C, operands, bn, 1)
    torch.cuda.synchronize()
    err = np.abs(C.cpu().double().numpy() - ref).max() / np.abs(ref).max()
    assert err < max(2e-6, 5e-7 * np.sqrt(K)), err


def _learner(w, hf=None, params=None):
    cfg = lib_config(w)
    O, _ = obs_dims(w)
    if params is None:
        params = synth.xavier_params(w["seed"] + 1, O, w["hidden"], 12)
    if hf is None and w["grid"][0]:
        hf = synth.heightfield(w["seed"] + 2)
    return api.Learner(cfg, hf, params), hf


def _env_case(w, seed, n_steps=1):
    L, hf = _learner(w)
    N = w["num_envs"]
    O, Op = obs_dims(w)
    ecfg = oracle_env_config(w)
    sf0, si0 = synth.random_env_state(seed, N)
    L.set_state(torch.from_numpy(sf0).cuda(), torch.from_numpy(si0).cuda())
    rs = np.random.default_rng(seed + 7)
    sf, si = sf0, si0
    bf16 = w["precision"] == 1
    obs_dt = torch.bfloat16 if bf16 else torch.float32
    for t in range(n_steps):
        a = rs.normal(size=(N, 12)).astype(np.float32)
        v = rs.normal(size=N).astype(np.float32)
        obs = torch.full((N, Op), 7.0, dtype=obs_dt, device="cuda")
        rew = torch.empty(N, device="cuda")
        done = torch.empty(N, dtype=torch.uint8, device="cuda")
        tout = torch.empty(N, dtype=torch.uint8, device="cuda")
        lvl = torch.empty(N, dtype=torch.int32, device="cuda")
        tid = torch.empty(N, dtype=torch.int32, device="cuda")
        api.rl_env_step(L.ctx, t, torch.from_numpy(a).cuda(), torch.from_numpy(v).cuda(), obs, rew, done, tout, lvl, tid)
        gsf, gsi = L.get_state()
        torch.cuda.synchronize()
        ref = OE.step(ecfg, hf if hf is not None else np.zeros((800, 1600), np.float32), sf, si, a, v, 0, t)
        yield t, {"obs": obs.float().cpu().numpy(), "rew": rew.cpu().numpy(), "done": done.cpu().numpy(),
                  "timeout": tout.cpu().numpy(), "level": lvl.cpu().numpy(), "tidx": tid.cpu().numpy(),
                  "sf": gsf.cpu().numpy(), "si": gsi.cpu().numpy()}, ref
        sf, si = ref["sf"], ref["si"]
    L.close()


def _check_step(got, ref, O, bf16=False):
    assert np.array_equal(got["sf"], ref["sf"]), np.argwhere(got["sf"] != ref["sf"])[:10]
    assert np.array_equal(got["si"], ref["si"])
    assert np.array_equal(got["done"], ref["done"])
    assert np.array_equal(got["timeout"], ref["timeout"])
    assert np.array_equal(got["level"], ref["level"])
    assert np.array_equal(got["tidx"], ref["terrain_idx"])
    assert rel_err(got["rew"], ref["reward"]) < TOL_FP32
    assert np.all(got["obs"][:, O:] == 0)
    if bf16:
        want = _bf16_round(ref["obs"])
        assert np.all(np.abs(got["obs"][:, :O] - want) <= 2 ** -7 * np.abs(want) + 1e-6)
    else:
        assert rel_err(got["obs"][:, :O], ref["obs"]) < TOL_FP32


@pytest.mark.parametrize("n,grid", [(328, (17, 11)), (64, (0, 0)), (4096, (17, 11)), (328, (12, 9))])
def test_env_step_single(n, grid):
    w = workload("small_rough", num_envs=n, grid=grid, crash_threshold=2 ** 27)
    O, _ = obs_dims(w)
    for _, got, ref in _env_case(w, seed=3):
        assert ref["done"].any()
        _check_step(got, ref, O)


def test_env_step_chain_8_steps_bit_exact_state():
    w = workload("small_rough", num_envs=328, crash_threshold=2 ** 28)
    O, _ = obs_dims(w)
    resets = 0
    for _, got, ref in _env_case(w, seed=5, n_steps=8):
        _check_step(got, ref, O)
        resets += int(ref["done"].sum())
    assert resets > 50


@pytest.mark.parametrize("grid", [(17, 11), (12, 9)])
def test_env_step_bf16_observations(grid):
    w = workload("small_rough", num_envs=328, precision=1, grid=grid)
    O, _ = obs_dims(w)
    for _, got, ref in _env_case(w, seed=11):
        _check_step(got, ref, O, bf16=True)


def test_env_spawn_matches_oracle():
    w = workload("small_rough", num_envs=328)
    L, hf = _learner(w)
    O, Op = obs_dims(w)
    obs = torch.zeros((328, Op), device="cuda")
    api.rl_env_reset_all(L.ctx, obs)
    sf, si = L.get_state()
    torch.cuda.synchronize()
    ecfg = oracle_env_config(w)
    rsf, rsi = OE.initial_state(ecfg)
    assert np.array_equal(sf.cpu().numpy(), rsf) and np.array_equal(si.cpu().numpy(), rsi)
    ro = OT.initial_observation(ecfg, hf, rsf, rsi)
    assert rel_err(obs.cpu().numpy()[:, :O], ro) < TOL_FP32
    L.close()


@pytest.mark.parametrize("T,N", [(24, 4096), (24, 1000), (1, 1), (7, 33), (24, 16384)])
def test_gae_matches_oracle(T, N):
    rs = np.random.default_rng(T * 1000 + N)
    r = rs.normal(size=(T, N)).astype(np.float32)
    v = rs.normal(size=(T, N)).astype(np.float32)
    lv = rs.normal(size=N).astype(np.float32)
    d = (rs.random((T, N)) < 0.05).astype(np.uint8)
    cu = lambda x: torch.from_numpy(x).cuda()
    adv = torch.empty((T, N), device="cuda")
    ret = torch.empty((T, N), device="cuda")
    st = torch.empty(2, device="cuda")
    ws = torch.empty(api.rl_gae_workspace_bytes(T, N) // 4 + 4, device="cuda")
    api.rl_gae(0.99, 0.95, cu(r), cu(v), cu(lv), cu(d), adv, ret, normalize=False, adv_stats_out=st, workspace=ws)
    A, R = OG.gae(r, v, lv, d, 0.99, 0.95)
    assert rel_err(adv.cpu().numpy(), A) < TOL_FP32
    assert rel_err(ret.cpu().numpy(), R) < TOL_FP32
    An, m, s = OG.normalize(A)
    stats = st.cpu().numpy()
    assert abs(stats[0] - m) <= TOL_FP32 * max(abs(m), s) and abs(stats[1] - s) <= TOL_FP32 * s
    api.rl_gae(0.99, 0.95, cu(r), cu(v), cu(lv), cu(d), adv, ret, normalize=True, workspace=ws)
    if T * N > 1:
        assert rel_err(adv.cpu().numpy(), An) < TOL_FP32
    assert rel_err(ret.cpu().numpy(), R) < TOL_FP32


def test_gae_rejects_missing_workspace():
    x = torch.zeros((2, 4), device="cuda")
    with pytest.raises(api.RLError):
        api.rl_gae(0.99, 0.95, x, x, x[0], torch.zeros((2, 4), dtype=torch.uint8, device="cuda"), x.clone(),
                   x.clone(), normalize=True, workspace=None)
