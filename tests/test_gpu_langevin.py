"""Langevin thermostat of Algorithm 1 and HMR on the GPU (needs a GB300).

The GPU draws its noise from its own Philox-4x32-10 implementation with the
same counter layout as the oracle, so with the same seed both integrate the
same stochastic trajectory: the comparison is the NVE trajectory test's,
with a friction strong enough (20 ps^-1) that a wrong draw, a misplaced
O-step or a wrong c1/c2 moves the velocities by O(sqrt(k_B T / m)) at once.
"""
import json

import numpy as np
import pytest

from oracle import integrate as G
from oracle import model as M
from paper_2510_06562_gb300 import dmts as D
from paper_2510_06562_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FRICTION = 20.0          # ps^-1
SEED = 12345


def _ctx(s, mass=None, small=True, **opts):
    sa, ba = I.small_arch(s.n_species), I.big_arch(s.n_species)
    o = {"langevin_friction": FRICTION, "temperature": 300.0, "seed": SEED, "autotune": 0}
    o.update(opts)
    if mass is not None:
        s = I.System(x=s.x, species=s.species, mass=mass, atom_offset=s.atom_offset, box=s.box,
                     n_species=s.n_species, name=s.name, bonds=s.bonds)
    if small:
        return D.Context(s, ba, I.init_params(ba, 3), sa, I.init_params(sa, 2), options=json.dumps(o))
    return D.Context(s, ba, I.init_params(ba, 3), options=json.dumps(o))


def _forces(s, arch, par):
    spec = M.spec_of(arch)
    return lambda x: M.energy_forces(spec, par, x, s.species, s.atom_offset, s.box)[1]


def _thermo():
    return {"gamma": FRICTION * 1e-3, "temperature": 300.0, "seed": SEED}


def _dx(a, b, L):
    d = a - b
    return d - L * np.round(d / L)


def test_langevin_respa_matches_oracle():
    s = I.water_192(0)
    sa, ba = I.small_arch(2), I.big_arch(2)
    v0 = I.maxwell_boltzmann(s.mass, 300.0, 1)
    bpa = np.full(s.n_atoms, s.box[0])
    xr, vr, _, _, _ = G.respa(s.x, v0, s.mass, _forces(s, sa, I.init_params(sa, 2)),
                              _forces(s, ba, I.init_params(ba, 3)), 3.0, 3, 8, box_per_atom=bpa,
                              thermo=_thermo(), step0=0)
    with _ctx(s) as ctx:
        ctx.set_state(s.x, v0)
        ctx.respa_step(8, 3.0, 3)
        xg, vg = ctx.get_state()
    assert np.abs(_dx(xg, xr, s.box[0])).max() < 1e-4
    assert np.abs(vg - vr).max() < 1e-5
    # the thermostat acted: the NVE trajectory is far away
    xn, vn, _, _, _ = G.respa(s.x, v0, s.mass, _forces(s, sa, I.init_params(sa, 2)),
                              _forces(s, ba, I.init_params(ba, 3)), 3.0, 3, 8, box_per_atom=bpa)
    assert np.abs(vn - vr).max() > 100 * np.abs(vg - vr).max()


def test_baoab_velocity_verlet_matches_oracle():
    s = I.water_192(0)
    ba = I.big_arch(2)
    v0 = I.maxwell_boltzmann(s.mass, 300.0, 1)
    bpa = np.full(s.n_atoms, s.box[0])
    xr, vr, _ = G.velocity_verlet(s.x, v0, s.mass, _forces(s, ba, I.init_params(ba, 3)), 1.0, 12,
                                  box_per_atom=bpa, thermo=_thermo(), step0=0)
    with _ctx(s, small=False) as ctx:
        ctx.set_state(s.x, v0)
        ctx.respa_step(12, 1.0, 1)
        xg, vg = ctx.get_state()
    assert np.abs(_dx(xg, xr, s.box[0])).max() < 1e-5
    assert np.abs(vg - vr).max() < 1e-6


def test_noise_counter_is_continuous_and_restarts_with_set_state():
    s = I.water_192(0)
    v0 = I.maxwell_boltzmann(s.mass, 300.0, 1)
    with _ctx(s) as a, _ctx(s) as b:
        a.set_state(s.x, v0)
        a.respa_step(3, 3.0, 3)
        a.respa_step(2, 3.0, 3)
        xa, va = a.get_state()
        b.set_state(s.x, v0)
        b.respa_step(5, 3.0, 3)
        xb, vb = b.get_state()
        np.testing.assert_array_equal(xa, xb)
        np.testing.assert_array_equal(va, vb)
        b.set_state(s.x, v0)                        # the counter restarts: same trajectory again
        b.respa_step(5, 3.0, 3)
        xc, vc = b.get_state()
        np.testing.assert_array_equal(xc, xb)
        np.testing.assert_array_equal(vc, vb)
    with _ctx(s, seed=SEED + 1) as c:               # another seed: another trajectory
        c.set_state(s.x, v0)
        c.respa_step(5, 3.0, 3)
        assert np.abs(c.get_state()[1] - vb).max() > 1e-3


def test_hmr_respa_5fs_matches_oracle():
    """The paper's HMR setting: 1 fs inner / 5 fs outer steps with hydrogens
    at 3.024 amu and friction 1 ps^-1, against the oracle at the same
    masses."""
    s = I.water_192(0)
    sa, ba = I.small_arch(2), I.big_arch(2)
    m = D.hmr_masses(s.mass, s.bonds, 3.024)
    v0 = I.maxwell_boltzmann(m, 300.0, 1)
    bpa = np.full(s.n_atoms, s.box[0])
    th = {"gamma": 1e-3, "temperature": 300.0, "seed": SEED}
    xr, vr, _, _, _ = G.respa(s.x, v0, m, _forces(s, sa, I.init_params(sa, 2)),
                              _forces(s, ba, I.init_params(ba, 3)), 5.0, 5, 4, box_per_atom=bpa, thermo=th)
    with _ctx(s, mass=m, langevin_friction=1.0) as ctx:
        ctx.set_state(s.x, v0)
        e = ctx.respa_step(4, 5.0, 5)
        xg, vg = ctx.get_state()
    assert np.all(np.isfinite(e))
    assert np.abs(_dx(xg, xr, s.box[0])).max() < 1e-4
    assert np.abs(vg - vr).max() < 1e-5
