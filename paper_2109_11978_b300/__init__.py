"""B300 (sm_103a) hot path of massively parallel PPO for legged locomotion.

The CUDA library (csrc/, C ABI in include/rl_b300.h) runs the env-side tensor math, batched
actor/critic inference, GAE and the PPO update; `api` binds it for torch tensors, `synth`
draws the seeded synthetic inputs, `build` compiles the library in-tree.
"""
__all__ = ["api", "synth", "build"]
