"""FP64 oracle of the integrators (test infrastructure only).

* ``respa`` is Algorithm 1 (the MTS integration step with force splitting)
  step by step, with the thermostat ``thermo`` the identity (NVE): an outer
  half-kick with the force difference F - F_small, n_slow inner steps of
  kick / half-drift / (thermostat) / half-drift / small force / kick, then the
  large force and a second half-kick with F - F_small.
* ``velocity_verlet`` is the textbook single-time-step scheme: half-kick,
  full drift, force, half-kick.

Positions of periodic systems are wrapped into [0, L) after every drift
(x - L floor(x / L)); the paper does not say where its engines wrap.

Units: x in A, v in A/fs, F in eV/A, masses in amu, t in fs; the kick
dv = dt F / m is converted from eV/(A amu) to A/fs^2.
"""
from __future__ import annotations

from typing import Callable

import numpy as np

# 1 eV/(A amu) in A/fs^2: (1.602176634e-19 J / 1e-10 m) / 1.66053906660e-27 kg
# = 9.6485e17 m/s^2, and 1 A/fs^2 = 1e20 m/s^2.
ACCEL = (1.602176634e-19 / 1e-10) / 1.66053906660e-27 / 1e20
# 1 amu (A/fs)^2 in eV: the inverse of ACCEL.
KE_EV = 1.0 / ACCEL

Force = Callable[[np.ndarray], np.ndarray]


def _wrap(x, box_per_atom):
    if box_per_atom is None:
        return x
    L = box_per_atom[:, None]
    per = L > 0
    Ls = np.where(per, L, 1.0)
    return np.where(per, x - Ls * np.floor(x / Ls), x)


def kinetic_energy(v, mass, atom_offset=None):
    """Per-system kinetic energy sum_i m_i |v_i|^2 / 2 in eV."""
    ke_i = 0.5 * mass * (v * v).sum(axis=1) * KE_EV
    if atom_offset is None:
        return np.array([ke_i.sum()])
    off = np.asarray(atom_offset)
    return np.array([ke_i[off[s]:off[s + 1]].sum() for s in range(len(off) - 1)])


def velocity_verlet(x, v, mass, f: Force, dt: float, n_steps: int,
                    box_per_atom=None, F=None):
    """n_steps of velocity Verlet with time step dt; returns (x, v, F)."""
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    a = ACCEL / np.asarray(mass, dtype=np.float64)[:, None]
    if F is None:
        F = f(x)
    for _ in range(n_steps):
        v = v + 0.5 * dt * a * F
        x = _wrap(x + dt * v, box_per_atom)
        F = f(x)
        v = v + 0.5 * dt * a * F
    return x, v, F


def respa(x, v, mass, f_small: Force, f_big: Force, dt: float, n_slow: int,
          n_outer: int, box_per_atom=None, F_small=None, F=None,
          energy_big: Callable[[np.ndarray], float] | None = None,
          atom_offset=None):
    """n_outer steps of Algorithm 1 (thermo = identity) with outer step dt and
    n_slow inner steps of dt / n_slow.

    ``F_small`` and ``F`` carry the forces at ``x`` between calls; when either
    is None this is the algorithm's first step and both are evaluated.
    Returns (x, v, F_small, F, energies) where energies is [n_outer, 3] with
    (E_pot of the big model, E_kin, E_pot + E_kin) after each outer step if
    ``energy_big`` is given, else None.
    """
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    mass = np.asarray(mass, dtype=np.float64)
    a = ACCEL / mass[:, None]
    if F_small is None or F is None:                        # first_step
        F_small = f_small(x)
        F = f_big(x)
    h = dt / n_slow
    out = []
    for _ in range(n_outer):
        v = v + (0.5 * dt) * a * (F - F_small)
        for _ in range(n_slow):
            v = v + (0.5 * h) * a * F_small
            x = _wrap(x + (0.5 * h) * v, box_per_atom)
            # thermo(v, h) = v  (NVE)
            x = _wrap(x + (0.5 * h) * v, box_per_atom)
            F_small = f_small(x)
            v = v + (0.5 * h) * a * F_small
        F = f_big(x)
        v = v + (0.5 * dt) * a * (F - F_small)
        if energy_big is not None:
            ep = np.asarray(energy_big(x), dtype=np.float64).reshape(-1)
            ek = kinetic_energy(v, mass, atom_offset)
            out.append(np.stack([ep, ek, ep + ek], axis=-1))
    energies = np.asarray(out) if energy_big is not None else None
    return x, v, F_small, F, energies
