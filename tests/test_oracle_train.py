"""Oracle training iteration end to end (CPU only): shapes, invariants, Algorithm 1 trace.

The rollout stores the time-out bootstrap in the reward (Sec. 2.2.2), GAE consumes it, and
the update runs epochs x minibatches with the learning rate adapted after every minibatch.
"""
import numpy as np

from oracle import config as C
from oracle import mlp, ppo
from oracle.train import Learner
from paper_2109_11978_b300 import synth


def test_learner_iteration_tiny():
    ecfg = C.EnvConfig(num_envs=32, grid_x=0, grid_y=0, crash_threshold=2 ** 27)
    pcfg = C.PPOConfig(epochs=2, minibatches=2)
    hidden = (16, 16)
    flat = synth.xavier_params(0, ecfg.obs_dim, hidden, 12)
    hf = synth.heightfield(0, flat=True)
    L = Learner(ecfg, pcfg, hidden, hf, flat)
    st, stats = L.iterate(8)
    assert st["obs"].shape == (8, 32, 48) and len(stats) == 4
    assert all(np.isfinite(s["loss"]) for s in stats)
    lr = pcfg.lr_init
    for s in stats:
        lr = ppo.adapt_lr(lr, s["kl"])
        assert s["lr"] == lr
    assert stats[0]["kl"] < 1e-12            # first minibatch: parameters equal the behaviour policy
    assert L.iteration == 1 and not np.array_equal(L.flat, flat.astype(np.float64))
    # logp stored at act time is the log density of the stored action
    p = mlp.unflatten(flat, 48, hidden, 12)
    np.testing.assert_allclose(st["logp"][0], mlp.log_prob(st["actions"][0], st["mu"][0], p["log_std"]), rtol=1e-12)
