"""System-specific distillation of the small model (section "Training
procedures"): frames from a short MD run of the reference (big) model,
labelled with its energies and forces, then the small model fit to them by
Adam on the energy and force loss.

Every step runs in the library through its C ABI: the frames come from
single-time-step velocity Verlet of a big-model-only context
(``dmts_respa_step`` with n_inner = 1, ``dmts_get_state``,
``dmts_forces``), the gradient from ``dmts_distill_grad`` and the update
from ``dmts_adam_step``. This module only sequences those calls.

The random-init stand-in models stay stable for about 120 fs of dynamics,
so the frames are taken from several short trajectories (independent
Maxwell-Boltzmann velocities) rather than from one long run.
"""
from __future__ import annotations

import numpy as np

from . import dmts as D
from . import inputs as I


def sample_frames(system, big_arch, big_params, n_frames: int, n_traj: int = 8, stride_fs: float = 10.0,
                  dt_fs: float = 1.0, temperature: float = 300.0, seed: int = 11, precision: int = D.FP32,
                  options: str | None = None):
    """n_frames frames of big-model MD: n_traj trajectories from the
    system's positions with Maxwell-Boltzmann velocities (seed + k), each
    sampled every stride_fs after one stride of equilibration. Returns
    (frames [M, N, 3], f_ref [M, N, 3], e_ref [M]): positions and the big
    model's forces and total energy at each frame."""
    if n_frames < 1 or n_traj < 1:
        raise ValueError("need n_frames >= 1 and n_traj >= 1")
    per = -(-n_frames // n_traj)
    steps = max(1, int(round(stride_fs / dt_fs)))
    frames, f_ref, e_ref = [], [], []
    with D.Context(system, big_arch, big_params, precision=precision, options=options) as ctx:
        for k in range(n_traj):
            if len(frames) >= n_frames:
                break
            v0 = I.maxwell_boltzmann(system.mass, temperature, seed + k, system.atom_offset)
            ctx.set_state(system.x, v0)
            ctx.respa_step(steps, dt_fs, 1, energies=False)
            for _ in range(per):
                if len(frames) >= n_frames:
                    break
                ctx.respa_step(steps, dt_fs, 1, energies=False)
                x, _ = ctx.get_state()
                E, F = ctx.forces(D.BIG)
                frames.append(x)
                f_ref.append(F)
                e_ref.append(float(np.sum(E)))
    return np.stack(frames), np.stack(f_ref), np.array(e_ref)


def train(ctx: "D.Context", frames, f_ref, e_ref, n_steps: int, lr: float = 1e-3, lambda_e: float = 1.0,
          beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """n_steps full-batch Adam steps of the small model of ``ctx`` on the
    energy and force loss; returns the loss before each step."""
    n = ctx.small_n_params
    m1, m2 = np.zeros(n), np.zeros(n)
    losses = []
    for t in range(1, n_steps + 1):
        loss, g = ctx.distill_grad(frames, f_ref, e_ref, lambda_e)
        losses.append(loss)
        ctx.adam_step(D.SMALL, g, m1, m2, t, lr, beta1, beta2, eps)
    return losses
