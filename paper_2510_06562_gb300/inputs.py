"""Seeded synthetic inputs: structures, velocities, masses and model parameters.

This module holds no arithmetic of the method itself (no basis, cutoff,
network or integrator): it only draws the numbers that the CUDA path and the
FP64 oracle both consume, so that either side can be fed identical inputs.

Units: Angstrom, eV, amu, fs.

Species indices are model-local: water systems use 0 = H, 1 = O
(``n_species = 2``); four-element systems use 0 = H, 1 = C, 2 = N, 3 = O.

Parameter vector layout (flat float64, in this order; ``S`` species, ``F``
features, ``K`` radial functions, ``Lr`` message-passing layers):

    A    [S, F]            species embedding, h0_i = A[Z_i]
    for each layer l < Lr:
      W_in [F, F]          u_i = h_i @ W_in
      W1   [K, F], b1 [F]  filter hidden layer (on the radial basis)
      W2   [F, F], b2 [F]  filter output layer
      U1   [F, F], c1 [F]  atom-update hidden layer (on the message)
      U2   [F, F], c2 [F]  atom-update output layer (residual)
    R1   [F, F], d1 [F]    readout hidden layer
    R2   [F],    d2 [1]    readout output
    e0   [S]               per-species energy offset

Matrices are row-major with the input index first (``y = x @ W``).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Masses in amu (IUPAC standard atomic weights).
MASS_H = 1.008
MASS_C = 12.011
MASS_N = 14.007
MASS_O = 15.999

# Boltzmann constant in eV/K and (eV/amu) -> (A/fs)^2 used only to draw
# Maxwell-Boltzmann velocities.
_KB_EV = 8.617333262e-5
_EV_PER_AMU_TO_A2_PER_FS2 = 1.602176634e-19 / 1.66053906660e-27 * 1e-10


# Short-range pair repulsion shared by both models: phi(d) = REP_A exp(-d /
# REP_RHO) fc(d; REP_CUTOFF). Random-init networks have no repulsive core, so
# atoms otherwise pass through each other and the dynamics blow up; the same
# term in both models is part of the fast forces and cancels in F_big - F_small.
REP_A = 50.0        # eV
REP_RHO = 0.2       # A
REP_CUTOFF = 2.0    # A


@dataclasses.dataclass(frozen=True)
class Arch:
    """Architecture of one invariant message-passing potential."""

    cutoff: float
    n_radial: int
    n_layers: int
    n_feat: int
    n_species: int
    rep_a: float = REP_A
    rep_rho: float = REP_RHO
    rep_cutoff: float = REP_CUTOFF

    def param_count(self) -> int:
        S, F, K, L = self.n_species, self.n_feat, self.n_radial, self.n_layers
        per_layer = F * F + K * F + F + F * F + F + F * F + F + F * F + F
        return S * F + L * per_layer + F * F + F + F + 1 + S


# The two architectures of the distilled multi-time-step pair: the big model
# (5.0 A cutoff, 16 radial functions, 2 layers, 64 features) and the distilled
# small model (3.5 A cutoff, 8 radial functions, 1 layer, 32 features).
def big_arch(n_species: int = 2) -> Arch:
    return Arch(cutoff=5.0, n_radial=16, n_layers=2, n_feat=64, n_species=n_species)


def small_arch(n_species: int = 2) -> Arch:
    return Arch(cutoff=3.5, n_radial=8, n_layers=1, n_feat=32, n_species=n_species)


def param_slices(arch: Arch) -> dict:
    """Offsets of every named block in the flat parameter vector.

    Keys: ``A``, ``R1``, ``d1``, ``R2``, ``d2``, ``e0`` and, per layer ``l``,
    ``(l, name)`` for name in W_in, W1, b1, W2, b2, U1, c1, U2, c2. Values are
    ``(offset, shape)``.
    """
    S, F, K = arch.n_species, arch.n_feat, arch.n_radial
    out = {}
    off = 0

    def take(key, shape):
        nonlocal off
        out[key] = (off, shape)
        off += int(np.prod(shape))

    take("A", (S, F))
    for l in range(arch.n_layers):
        take((l, "W_in"), (F, F))
        take((l, "W1"), (K, F))
        take((l, "b1"), (F,))
        take((l, "W2"), (F, F))
        take((l, "b2"), (F,))
        take((l, "U1"), (F, F))
        take((l, "c1"), (F,))
        take((l, "U2"), (F, F))
        take((l, "c2"), (F,))
    take("R1", (F, F))
    take("d1", (F,))
    take("R2", (F,))
    take("d2", (1,))
    take("e0", (S,))
    assert off == arch.param_count()
    return out


# Readout scale (eV). Together with the 1/k damping of the radial-filter
# weights W1 it is chosen so that 1 fs velocity Verlet with the random-init big
# model conserves energy on liquid-density water (about 1e-4 eV/atom over
# 100 fs), the regime the paper's integrators operate in; RMS force
# components are then about 0.17 eV/A (big) and 0.08 eV/A (small). With O(1)
# eV/A random forces the landscape is so rough that even 0.5 fs steps heat up.
ENERGY_SCALE = 1.0
BIAS_STD = 0.1


def init_params(arch: Arch, seed: int, energy_scale: float = ENERGY_SCALE) -> np.ndarray:
    """Random-init parameters (float64), drawn from PCG64(seed).

    Weights ~ N(0, 1/fan_in), except that row k (radial function k+1) of every
    filter matrix W1 is divided by k+1, a smoothness prior that keeps radial
    filters dominated by low Bessel frequencies; biases ~ N(0, BIAS_STD^2)
    (non-zero so that a dropped bias term changes the result); A ~ N(0, 1); the
    readout output layer, its bias and e0 are multiplied by ``energy_scale``.
    """
    rng = np.random.default_rng(seed)
    sl = param_slices(arch)
    p = np.empty(arch.param_count(), dtype=np.float64)
    for key, (off, shape) in sl.items():
        name = key[1] if isinstance(key, tuple) else key
        n = int(np.prod(shape))
        if name in ("b1", "b2", "c1", "c2", "d1"):
            vals = rng.normal(0.0, BIAS_STD, n)
        elif name == "A":
            vals = rng.normal(0.0, 1.0, n)
        elif name == "R2":
            vals = rng.normal(0.0, 1.0 / math.sqrt(arch.n_feat), n) * energy_scale
        elif name == "d2":
            vals = rng.normal(0.0, BIAS_STD, n) * energy_scale
        elif name == "e0":
            vals = rng.normal(0.0, 1.0, n) * energy_scale
        else:  # weight matrix, fan_in = first dimension
            vals = rng.normal(0.0, 1.0 / math.sqrt(shape[0]), n)
            if name == "W1":
                vals = (vals.reshape(shape) / np.arange(1, shape[0] + 1)[:, None]).ravel()
        p[off:off + n] = vals
    return p


def unpack_params(arch: Arch, p: np.ndarray) -> dict:
    """View the flat vector as named arrays (no copy)."""
    p = np.asarray(p, dtype=np.float64)
    return {k: p[o:o + int(np.prod(s))].reshape(s) for k, (o, s) in param_slices(arch).items()}


# --------------------------------------------------------------------------
# Structures
# --------------------------------------------------------------------------

def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotation matrices (Shoemake's subgroup algorithm)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    q = np.stack([
        np.sqrt(1 - u1) * np.sin(2 * np.pi * u2),
        np.sqrt(1 - u1) * np.cos(2 * np.pi * u2),
        np.sqrt(u1) * np.sin(2 * np.pi * u3),
        np.sqrt(u1) * np.cos(2 * np.pi * u3),
    ], axis=1)
    x, y, z, w = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


@dataclasses.dataclass
class System:
    """One batch of independent systems (a single periodic box or molecules).

    ``x`` [N, 3] float64; ``species`` [N] int32; ``mass`` [N] float64;
    ``atom_offset`` [n_systems + 1] int32; ``box`` [n_systems] float64 cubic
    edge length (<= 0 means non-periodic); ``bonds`` [n_bonds, 2] int32 atom
    indices of the generator's covalent bonds (used for hydrogen mass
    repartitioning only; the potentials do not use bonds).
    """

    x: np.ndarray
    species: np.ndarray
    mass: np.ndarray
    atom_offset: np.ndarray
    box: np.ndarray
    n_species: int
    name: str = ""
    bonds: np.ndarray | None = None

    @property
    def n_atoms(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_systems(self) -> int:
        return int(self.box.shape[0])


def make_water(n_side: int, box: float, seed: int = 0) -> System:
    """``n_side**3`` rigid water molecules (O-H 0.96 A, H-O-H 104.5 deg) with
    O at the lattice sites ``(i + 1/2) * box / n_side`` and uniformly random
    orientations, in a periodic cubic box; atoms ordered O, H, H per molecule
    and wrapped into ``[0, box)``.

    192 atoms: ``make_water(4, 12.42)``; 12,288 atoms: ``make_water(16, 49.7)``.
    """
    rng = np.random.default_rng(seed)
    n_mol = n_side ** 3
    a = box / n_side
    g = (np.arange(n_side) + 0.5) * a
    O = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    half = np.deg2rad(104.5) / 2
    r_oh = 0.96
    local = np.array([[0.0, 0.0, 0.0],
                      [r_oh * np.sin(half), 0.0, r_oh * np.cos(half)],
                      [-r_oh * np.sin(half), 0.0, r_oh * np.cos(half)]])
    R = _random_rotations(rng, n_mol)
    pos = O[:, None, :] + np.einsum("mab,kb->mka", R, local)
    x = pos.reshape(-1, 3)
    x = x - box * np.floor(x / box)
    species = np.tile(np.array([1, 0, 0], dtype=np.int32), n_mol)
    mass = np.where(species == 1, MASS_O, MASS_H).astype(np.float64)
    o_idx = 3 * np.arange(n_mol)
    bonds = np.stack([np.repeat(o_idx, 2), np.stack([o_idx + 1, o_idx + 2], axis=1).reshape(-1)],
                     axis=1).astype(np.int32)
    return System(x=x, species=species, mass=mass,
                  atom_offset=np.array([0, 3 * n_mol], dtype=np.int32),
                  box=np.array([box], dtype=np.float64), n_species=2,
                  name=f"water{3 * n_mol}", bonds=bonds)


def replicas(systems: list) -> System:
    """Independent systems stored back to back in one batch (periodic
    replicas must share one box edge); atom indices of the bonds shift with
    each system's offset."""
    xs, sp, ms, bonds, box, off = [], [], [], [], [], [0]
    for s in systems:
        if s.bonds is not None and len(s.bonds):
            bonds.append(np.asarray(s.bonds) + off[-1])
        xs.append(s.x)
        sp.append(s.species)
        ms.append(s.mass)
        box.append(s.box)
        off.extend(int(o) + off[-1] for o in np.asarray(s.atom_offset)[1:])
    return System(x=np.concatenate(xs), species=np.concatenate(sp).astype(np.int32), mass=np.concatenate(ms),
                  atom_offset=np.array(off, dtype=np.int32), box=np.concatenate(box).astype(np.float64),
                  n_species=max(s.n_species for s in systems), name=f"{len(systems)}x{systems[0].name}",
                  bonds=np.concatenate(bonds).astype(np.int32) if bonds else None)


def water_192(seed: int = 0) -> System:
    return make_water(4, 12.42, seed)


def water_12288(seed: int = 0) -> System:
    return make_water(16, 49.7, seed)


def make_vacuum_batch(n_mol: int = 512, n_min: int = 10, n_max: int = 60,
                      seed: int = 0) -> System:
    """``n_mol`` independent non-periodic molecules of ``U{n_min..n_max}``
    atoms: seeded random-walk chains with bond lengths ``U[1.1, 1.5]`` A in
    uniformly random directions, each new atom at least 1.0 A from all earlier
    atoms of its molecule; elements uniform over H/C/N/O."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(n_min, n_max + 1, n_mol)
    xs, zs = [], []
    for n in sizes:
        pts = [np.zeros(3)]
        while len(pts) < n:
            v = rng.normal(size=3)
            v /= np.linalg.norm(v)
            p = pts[-1] + rng.uniform(1.1, 1.5) * v
            if np.min(np.linalg.norm(np.asarray(pts) - p, axis=1)) >= 1.0:
                pts.append(p)
        xs.append(np.asarray(pts))
        zs.append(rng.integers(0, 4, n))
    masses = np.array([MASS_H, MASS_C, MASS_N, MASS_O])
    species = np.concatenate(zs).astype(np.int32)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    bonds = np.concatenate([np.stack([np.arange(off[k], off[k + 1] - 1), np.arange(off[k] + 1, off[k + 1])],
                                     axis=1) for k in range(n_mol)]).astype(np.int32)
    return System(x=np.concatenate(xs), species=species, mass=masses[species],
                  atom_offset=off, box=np.zeros(n_mol), n_species=4,
                  name=f"vacuum{n_mol}", bonds=bonds)


def make_solvated_polymer(n_heavy: int = 3000, n_total: int = 100_000, density: float = 1.0,
                          seed: int = 0) -> System:
    """A self-avoiding random-walk chain of ``n_heavy`` heavy atoms (C:N:O =
    6:2:2 in seeded random order, bonds 1.5 A, no heavy atom within 2.0 A of
    an earlier one except its chain neighbour), hydrogens added to fill each
    heavy atom's valence (C 4, N 3, O 2, minus its chain bonds) at C-H 1.09,
    N-H 1.01, O-H 0.96 A in random directions at least 1.0 A from every other
    atom, then rigid waters (as in ``make_water``) on a cubic lattice with
    random orientations, dropping sites within 2.5 A of the polymer, so that
    the total is ~``n_total`` atoms at ``density`` g/cm^3 in a periodic
    cubic box. Species: 0 = H, 1 = C, 2 = N, 3 = O."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    n_c = n_heavy * 6 // 10
    n_n = n_heavy * 2 // 10
    elem = rng.permutation(np.repeat(np.array([1, 2, 3]), [n_c, n_n, n_heavy - n_c - n_n]))
    valence = np.array([1, 4, 3, 2])          # by species index H, C, N, O
    chain_bonds = np.full(n_heavy, 2)
    chain_bonds[0] = chain_bonds[-1] = 1
    n_h = np.maximum(valence[elem] - chain_bonds, 0)
    heavy_mass = np.array([MASS_H, MASS_C, MASS_N, MASS_O])
    m_poly = heavy_mass[elem].sum() + n_h.sum() * MASS_H
    n_poly = n_heavy + int(n_h.sum())
    n_water = (n_total - n_poly) // 3
    m_total = m_poly + n_water * (MASS_O + 2 * MASS_H)
    L = (m_total * 1.66053906660 / density) ** (1.0 / 3.0)   # amu -> g is 1.6605e-24, A^3 -> cm^3 is 1e-24

    def wrap(p):
        return p - L * np.floor(p / L)

    def min_image(d):
        return d - L * np.round(d / L)

    # heavy-atom chain
    chain = np.empty((n_heavy, 3))
    chain[0] = rng.uniform(0, L, 3)
    k = 1
    while k < n_heavy:
        v = rng.normal(size=3)
        p = chain[k - 1] + 1.5 * v / np.linalg.norm(v)
        if k >= 2:
            d = np.linalg.norm(min_image(chain[:k - 1] - p), axis=1)
            if d.min() < 2.0:
                continue
        chain[k] = wrap(p)
        k += 1
    # hydrogens
    bond_h = np.array([0.0, 1.09, 1.01, 0.96])
    placed = [chain]
    tree = cKDTree(chain, boxsize=L)
    hs, h_parent = [], []
    for a in range(n_heavy):
        for _ in range(n_h[a]):
            for _try in range(200):
                v = rng.normal(size=3)
                p = wrap(chain[a] + bond_h[elem[a]] * v / np.linalg.norm(v))
                near = tree.query_ball_point(p, 1.0)
                if any(j != a for j in near):
                    continue
                if hs and np.min(np.linalg.norm(min_image(np.asarray(hs) - p), axis=1)) < 1.0:
                    continue
                hs.append(p)
                h_parent.append(a)
                break
            else:
                raise RuntimeError("could not place a hydrogen")
    poly = np.concatenate([chain, np.asarray(hs).reshape(-1, 3)])
    poly_species = np.concatenate([elem, np.zeros(len(hs), dtype=elem.dtype)])
    # waters on a lattice, away from the polymer
    n_side = int(np.ceil((n_water * 1.15) ** (1.0 / 3.0)))
    g = (np.arange(n_side) + 0.5) * (L / n_side)
    sites = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    ptree = cKDTree(poly, boxsize=L)
    free = np.array([len(x) == 0 for x in ptree.query_ball_point(sites, 2.5)])
    sites = sites[free]
    if len(sites) < n_water:
        raise RuntimeError("not enough free lattice sites for the water")
    sites = sites[rng.choice(len(sites), n_water, replace=False)]
    half = np.deg2rad(104.5) / 2
    local = np.array([[0.0, 0.0, 0.0], [0.96 * np.sin(half), 0.0, 0.96 * np.cos(half)],
                      [-0.96 * np.sin(half), 0.0, 0.96 * np.cos(half)]])
    R = _random_rotations(rng, n_water)
    wat = wrap((sites[:, None, :] + np.einsum("mab,kb->mka", R, local)).reshape(-1, 3))
    x = np.concatenate([poly, wat])
    species = np.concatenate([poly_species, np.tile(np.array([3, 0, 0]), n_water)]).astype(np.int32)
    mass = heavy_mass[species]
    n_p = len(poly)
    o_idx = n_p + 3 * np.arange(n_water)
    bonds = np.concatenate([
        np.stack([np.arange(n_heavy - 1), np.arange(1, n_heavy)], axis=1),              # chain
        np.stack([np.asarray(h_parent, dtype=np.int64), n_heavy + np.arange(len(hs))], axis=1),
        np.stack([np.repeat(o_idx, 2), np.stack([o_idx + 1, o_idx + 2], axis=1).reshape(-1)], axis=1),
    ]).astype(np.int32)
    return System(x=x, species=species, mass=mass, atom_offset=np.array([0, len(x)], dtype=np.int32),
                  box=np.array([L]), n_species=4, name=f"polymer{len(x)}", bonds=bonds)


def maxwell_boltzmann(mass: np.ndarray, temperature: float, seed: int = 1,
                      atom_offset: np.ndarray | None = None) -> np.ndarray:
    """Velocities (A/fs) from the Maxwell-Boltzmann distribution at
    ``temperature`` K, with the centre-of-mass momentum of every system
    removed (no rescaling)."""
    rng = np.random.default_rng(seed)
    sigma = np.sqrt(_KB_EV * temperature / mass * _EV_PER_AMU_TO_A2_PER_FS2)
    v = rng.normal(size=(mass.shape[0], 3)) * sigma[:, None]
    if atom_offset is None:
        atom_offset = np.array([0, mass.shape[0]])
    for s in range(len(atom_offset) - 1):
        a, b = atom_offset[s], atom_offset[s + 1]
        p = (mass[a:b, None] * v[a:b]).sum(0)
        v[a:b] -= p / mass[a:b].sum()
    return v
