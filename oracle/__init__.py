"""FP64 CPU oracle for the distilled multi-time-step (DMTS) hot path.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, links or runs
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it. It shares no code with the CUDA library.

It is the plain definition of every result the GPU path computes, written
with plain PyTorch CPU float64 operations:

* ``model``     brute-force O(N^2) neighbour pairs, the invariant
                message-passing potential (energy), forces F = -dE/dx,
                virial, and the force-matching loss gradient (double
                backward) of the distillation step;
* ``integrate`` velocity Verlet and the RESPA multiple-time-step step of
                Algorithm 1, NVE or with the Langevin O-step (BAOAB) and its
                counter-based noise; hydrogen mass repartitioning.

Pins (tests marked ``not gpu``) tie it to the mathematics: finite
differences, invariances, closed-form degenerate cases, textbook special cases
of RESPA and a closed-form harmonic RESPA map.
"""
from . import model, integrate  # noqa: F401
