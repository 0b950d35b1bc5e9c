"""FP64 CPU oracle for the massively parallel PPO hot path (Rudin et al., CoRL 2021).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct restatement of
what the paper's training loop computes: the env-side tensor math (Sec. 3.1, 3.2, 3.3,
App. A.1.1, Table 2, Table 4), time-out bootstrapping (Sec. 2.2.2), generalized advantage
estimation (Sec. 2.2.1, Table 3), the clipped PPO update with the adaptive learning rate
(Sec. 2.2, Table 3, Algorithm 1) and Adam.  Floating point is float64 unless a passage
fixes the precision; the seeded physics stand-in (not part of the paper's method) is
defined as an fp32 recurrence and is evaluated in fp32 here so that both sides take every
integer decision on identical inputs.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import or execute anything in this package.  The product path
(the CUDA library and its Python binding) never imports it, and this package imports
nothing from the product.

Pins: every public function is checked by ``tests/test_oracle_*.py`` against closed forms,
hand-computed examples, brute force or invariants (see the docstrings).  The stand-in
transition has no paper passage to pin it against: parity unpinned (it is a documented
definition, compared bit-exactly with the CUDA path only).
"""
