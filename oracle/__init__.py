"""Plain FP64 CPU oracle of the DD-PPO rollout-then-update hot path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only code that may import it. It
shares no code with the CUDA library in ``paper_1911_00357_gb300``.

Modules:
  sim     -- ctypes wrapper of ``sim_oracle.c`` (scene generation, BFS
             geodesics, motion, reward/SPL, depth ray march), Sec. 4.
  policy  -- the agent network (App. "Agent Design") in float64 PyTorch CPU ops.
  rl      -- GAE (Sec. 4 "Training"), the PPO clipped surrogate (Eq. 2), the
             loss gradient (autograd in float64), Adam, and one PPO update.
"""
