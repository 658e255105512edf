"""FP64 oracle of the integrators (test infrastructure only).

* ``respa`` is the multiple-time-step integrator of Algorithm 1, written
  from its force splitting: the small model's force is the fast part, taken
  by n_inner velocity-Verlet substeps per outer step, and the remainder
  F - F_small is the slow part, applied as half-kicks at both ends of the
  outer step (NVE when ``thermo`` is None).
* ``velocity_verlet`` is the textbook single-time-step scheme: half-kick,
  full drift, force, half-kick.
* With ``thermo`` given, both become Langevin schemes: Algorithm 1's
  thermostat step (between the two half-drifts of each inner step) is the
  exact Ornstein-Uhlenbeck update of the velocities (the "O" of BAOAB), and
  velocity Verlet becomes BAOAB (half-kick, half-drift, O, half-drift,
  force, half-kick), the paper's single-time-step reference. The friction
  is 1 ps^-1 in the paper (section "Simulation details").
* ``hmr_masses`` is hydrogen mass repartitioning: each hydrogen's mass is
  raised to a target and the excess is taken from its bonded heavy atom.
* ``respa_monitored`` adds the force-difference monitor of the paper's
  active-learning section: after each outer step, if some atom's
  |F - F_small| exceeds the threshold (150 kcal/mol/A in the paper), the step
  is redone from its starting state with the single-time-step integrator
  (n_inner velocity-Verlet or BAOAB steps of dt / n_inner with the large model),
  and the small model is evaluated at the end for the next step's kicks.

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

# Boltzmann constant in eV/K (CODATA 2018, exact by the SI definitions).
KB_EV = 8.617333262e-5

Force = Callable[[np.ndarray], np.ndarray]

_M32 = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox-4x32 with 10 rounds (Salmon, Moraes, Dror and Shaw, "Parallel
    random numbers: as easy as 1, 2, 3", SC 2011): a counter-based generator
    whose output for a 128-bit counter and a 64-bit key is a fixed bijection
    of the counter. ``ctr`` [n, 4] and ``key`` [2] hold 32-bit words; returns
    [n, 4] uint32. Each round multiplies words 0 and 2 by the two Philox
    multipliers, crosses the high halves with words 1 and 3 and the key, and
    the key advances by the two Weyl constants between rounds."""
    c = np.asarray(ctr, dtype=np.uint64).reshape(-1, 4) & _M32
    k0, k1 = int(key[0]) & _M32, int(key[1]) & _M32
    m0, m1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
    for r in range(10):
        if r > 0:
            k0 = (k0 + 0x9E3779B9) & _M32
            k1 = (k1 + 0xBB67AE85) & _M32
        p0 = c[:, 0] * m0
        p1 = c[:, 2] * m1
        c = np.stack([(p1 >> np.uint64(32)) ^ c[:, 1] ^ np.uint64(k0), p1 & np.uint64(_M32),
                      (p0 >> np.uint64(32)) ^ c[:, 3] ^ np.uint64(k1), p0 & np.uint64(_M32)], axis=1)
    return c.astype(np.uint32)


def langevin_normals(n_atoms: int, step: int, seed: int) -> np.ndarray:
    """Three standard normal deviates per atom for inner step ``step``: one
    Philox call per atom with counter (atom, step low word, step high word, 0)
    and key (seed low word, seed high word); the four words become uniforms
    u = (w + 1/2) / 2^32 and the Box-Muller pairs (u0, u1) -> two normals,
    (u2, u3) -> one."""
    i = np.arange(n_atoms, dtype=np.uint64)
    ctr = np.stack([i, np.full_like(i, step & _M32), np.full_like(i, (step >> 32) & _M32),
                    np.zeros_like(i)], axis=1)
    w = philox4x32_10(ctr, (seed & _M32, (seed >> 32) & _M32)).astype(np.float64)
    u = (w + 0.5) / 4294967296.0
    r01 = np.sqrt(-2.0 * np.log(u[:, 0]))
    r23 = np.sqrt(-2.0 * np.log(u[:, 2]))
    return np.stack([r01 * np.cos(2.0 * np.pi * u[:, 1]), r01 * np.sin(2.0 * np.pi * u[:, 1]),
                     r23 * np.cos(2.0 * np.pi * u[:, 3])], axis=1)


def o_step(v, mass, h: float, thermo: dict, step: int):
    """Exact Ornstein-Uhlenbeck update over time h (fs) at friction
    thermo["gamma"] (1/fs) and temperature thermo["temperature"] (K):
    v <- c1 v + sqrt((1 - c1^2) k_B T / m) xi, c1 = exp(-gamma h)."""
    c1 = np.exp(-thermo["gamma"] * h)
    c2 = np.sqrt(1.0 - c1 * c1)
    sigma = np.sqrt(KB_EV * thermo["temperature"] * ACCEL / np.asarray(mass, dtype=np.float64))
    xi = langevin_normals(len(v), step, thermo["seed"])
    return c1 * v + (c2 * sigma)[:, None] * xi


def hmr_masses(mass, bonds, h_mass: float = 3.024, h_max: float = 1.5):
    """Hydrogen mass repartitioning: every atom lighter than ``h_max`` amu
    that is bonded to a heavier atom gets mass ``h_mass``; the difference is
    subtracted from that bonded heavy atom, so each molecule keeps its total
    mass. ``bonds`` [n_bonds, 2]; a hydrogen uses its first heavy partner."""
    m = np.array(mass, dtype=np.float64)
    m0 = np.asarray(mass, dtype=np.float64)
    done = np.zeros(len(m), dtype=bool)
    for a, b in np.asarray(bonds, dtype=np.int64).reshape(-1, 2):
        for h, heavy in ((a, b), (b, a)):
            if m0[h] < h_max and m0[heavy] >= h_max and not done[h]:
                m[heavy] -= h_mass - m0[h]
                m[h] = h_mass
                done[h] = True
    if np.any(m <= 0):
        raise ValueError("repartitioning leaves a non-positive mass")
    return m


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
                    box_per_atom=None, F=None, thermo: dict | None = None, step0: int = 0):
    """n_steps of velocity Verlet with time step dt; returns (x, v, F).
    With ``thermo``: BAOAB, step k drawing its noise at counter step0 + k."""
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    a = ACCEL / np.asarray(mass, dtype=np.float64)[:, None]
    if F is None:
        F = f(x)
    for k in range(n_steps):
        v = v + 0.5 * dt * a * F
        if thermo is None:
            x = _wrap(x + dt * v, box_per_atom)
        else:
            x = _wrap(x + (0.5 * dt) * v, box_per_atom)
            v = o_step(v, mass, dt, thermo, step0 + k)
            x = _wrap(x + (0.5 * dt) * v, box_per_atom)
        F = f(x)
        v = v + 0.5 * dt * a * F
    return x, v, F


def _kick(v, a, tau: float, F):
    """Velocity update by force F over time tau: v + tau F / m."""
    return v + tau * a * F


def _fast_substep(x, v, a, mass, h: float, F_fast, f_fast: Force, box_per_atom, thermo, step: int):
    """One substep of length h under the fast force alone: half-kick, two
    half-drifts (with the Ornstein-Uhlenbeck velocity update between them
    when ``thermo`` is given, drawing its noise at counter ``step``), the
    fast force at the new positions, half-kick. Returns (x, v, F_fast)."""
    v = _kick(v, a, 0.5 * h, F_fast)
    x = _wrap(x + (0.5 * h) * v, box_per_atom)
    if thermo is not None:
        v = o_step(v, mass, h, thermo, step)
    x = _wrap(x + (0.5 * h) * v, box_per_atom)
    F_fast = f_fast(x)
    v = _kick(v, a, 0.5 * h, F_fast)
    return x, v, F_fast


def respa(x, v, mass, f_small: Force, f_big: Force, dt: float, n_inner: int,
          n_outer: int, box_per_atom=None, F_small=None, F=None,
          energy_big: Callable[[np.ndarray], float] | None = None,
          atom_offset=None, thermo: dict | None = None, step0: int = 0):
    """n_outer outer steps of the multiple-time-step scheme of Algorithm 1.

    The large model's force is split as F = F_small + (F - F_small): the
    small model's force is the fast part, integrated by n_inner substeps of
    h = dt / n_inner (``_fast_substep``); the remainder is the slow part,
    applied as a half-kick of dt / 2 before and after them. thermo = None:
    NVE; else substep j of outer step s draws its noise at counter
    step0 + s n_inner + j.

    ``F_small`` and ``F`` carry the forces at ``x`` between calls; when either
    is None they are evaluated first (a start at new positions).
    Returns (x, v, F_small, F, energies) where energies is [n_outer, 3] with
    (E_pot of the big model, E_kin, E_pot + E_kin) after each outer step if
    ``energy_big`` is given, else None.
    """
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    mass = np.asarray(mass, dtype=np.float64)
    a = ACCEL / mass[:, None]
    if F_small is None or F is None:
        F_small = f_small(x)
        F = f_big(x)
    h = dt / n_inner
    out = []
    for s in range(n_outer):
        v = _kick(v, a, 0.5 * dt, F - F_small)                   # slow half-kick
        for j in range(n_inner):
            x, v, F_small = _fast_substep(x, v, a, mass, h, F_small, f_small, box_per_atom, thermo,
                                          step0 + s * n_inner + j)
        F = f_big(x)
        v = _kick(v, a, 0.5 * dt, F - F_small)                   # slow half-kick
        if energy_big is not None:
            ep = np.asarray(energy_big(x), dtype=np.float64).reshape(-1)
            ek = kinetic_energy(v, mass, atom_offset)
            out.append(np.stack([ep, ek, ep + ek], axis=-1))
    energies = np.asarray(out) if energy_big is not None else None
    return x, v, F_small, F, energies


def force_difference_norms(F, F_small):
    """Per-atom |F - F_small| (eV/A)."""
    d = np.asarray(F, dtype=np.float64) - np.asarray(F_small, dtype=np.float64)
    return np.sqrt((d * d).sum(axis=1))


def respa_monitored(x, v, mass, f_small: Force, f_big: Force, dt: float, n_inner: int, n_outer: int,
                    threshold: float, box_per_atom=None, thermo: dict | None = None, step0: int = 0,
                    df_out: list | None = None):
    """n_outer outer steps of Algorithm 1 with the force-difference monitor
    and single-time-step fallback. Returns (x, v, F_small, F, n_fallback,
    max_df) with max_df the largest |F - F_small| seen at the end of an
    outer step (before any fallback). If ``df_out`` is a list, each outer
    step's largest |F - F_small| is appended to it."""
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    F_small = f_small(x)
    F = f_big(x)
    h = dt / n_inner
    n_fallback, max_df = 0, 0.0
    for s_ in range(n_outer):
        t0 = step0 + s_ * n_inner
        x1, v1, Fs1, F1, _ = respa(x, v, mass, f_small, f_big, dt, n_inner, 1, box_per_atom=box_per_atom,
                                   F_small=F_small, F=F, thermo=thermo, step0=t0)
        df = force_difference_norms(F1, Fs1).max()
        if df_out is not None:
            df_out.append(float(df))
        max_df = max(max_df, df)
        if df > threshold:
            n_fallback += 1
            x1, v1, F1 = velocity_verlet(x, v, mass, f_big, h, n_inner, box_per_atom=box_per_atom, F=F,
                                         thermo=thermo, step0=t0)
            Fs1 = f_small(x1)
        x, v, F_small, F = x1, v1, Fs1, F1
    return x, v, F_small, F, n_fallback, max_df
