"""Pins of the oracle's integrators (CPU only).

``respa`` is Algorithm 1 with the thermostat the identity (NVE). Its special
cases reduce to textbook schemes: one inner step is velocity Verlet with the
big force; identical small and big forces make it velocity Verlet with step
dt / n_slow; a linear (harmonic) force split makes one outer step a product
of 2x2 kick and drift matrices; the scheme is time-reversible and its energy
error scales as dt^2.
"""
import numpy as np
import pytest

from oracle import integrate as G
from oracle import model as M
from paper_2510_06562_gb300 import inputs as I


def test_unit_conversion_constants():
    # 1 eV/(A amu) = 9.648533212e-3 A/fs^2; 1 amu (A/fs)^2 = 103.6427 eV
    assert abs(G.ACCEL - 9.6485332e-3) < 1e-10
    assert abs(G.KE_EV - 103.6427) < 1e-4
    ke = G.kinetic_energy(np.array([[1.0, 0.0, 0.0]]), np.array([2.0]))
    assert abs(ke[0] - G.KE_EV) < 1e-12


def _harmonic(k):
    return lambda x: -k * x


@pytest.mark.parametrize("n_slow", [1, 2, 3, 6])
def test_harmonic_split_closed_form(n_slow):
    """F = -k x split as F_small = -ks x: one outer step is
    K(dt/2, k-ks) [K(h/2, ks) D(h/2) D(h/2) K(h/2, ks)]^n K(dt/2, k-ks)
    acting on (x, v), with K(t, c) = [[1, 0], [-t c a, 1]], D(t) = [[1, t], [0, 1]]
    and a = ACCEL / m."""
    m, k, ks, dt = 2.0, 3.0, 2.2, 3.0
    a = G.ACCEL / m
    h = dt / n_slow

    def Kick(t, c):
        return np.array([[1.0, 0.0], [-t * c * a, 1.0]])

    def Drift(t):
        return np.array([[1.0, t], [0.0, 1.0]])

    inner = Kick(h / 2, ks) @ Drift(h / 2) @ Drift(h / 2) @ Kick(h / 2, ks)
    step = Kick(dt / 2, k - ks) @ np.linalg.matrix_power(inner, n_slow) @ Kick(dt / 2, k - ks)
    x0 = np.array([[0.3, -0.1, 0.2]])
    v0 = np.array([[0.01, 0.02, -0.03]])
    x, v, _, _, _ = G.respa(x0, v0, np.array([m]), _harmonic(ks), _harmonic(k), dt, n_slow, 4)
    S4 = np.linalg.matrix_power(step, 4)
    for c in range(3):
        ref = S4 @ np.array([x0[0, c], v0[0, c]])
        assert abs(x[0, c] - ref[0]) < 1e-14 and abs(v[0, c] - ref[1]) < 1e-15


@pytest.fixture(scope="module")
def water_small_model():
    s = I.make_water(2, 10.0, 0)
    spec = M.spec_of(I.small_arch())
    par = I.init_params(I.small_arch(), 2)
    specb = M.spec_of(I.big_arch())
    parb = I.init_params(I.big_arch(), 3)
    fs = lambda x: M.energy_forces(spec, par, x, s.species, s.atom_offset, s.box)[1]  # noqa: E731
    fb = lambda x: M.energy_forces(specb, parb, x, s.species, s.atom_offset, s.box)[1]  # noqa: E731
    v = I.maxwell_boltzmann(s.mass, 300.0, 1)
    return s, fs, fb, v


def test_one_inner_step_is_velocity_verlet(water_small_model):
    s, fs, fb, v = water_small_model
    bpa = np.full(s.n_atoms, s.box[0])
    x1, v1, _, _, _ = G.respa(s.x, v, s.mass, fs, fb, 1.0, 1, 5, box_per_atom=bpa)
    x2, v2, _ = G.velocity_verlet(s.x, v, s.mass, fb, 1.0, 5, box_per_atom=bpa)
    np.testing.assert_allclose(x1, x2, atol=1e-12)
    np.testing.assert_allclose(v1, v2, atol=1e-13)


def test_identical_forces_give_verlet_at_inner_step(water_small_model):
    s, fs, fb, v = water_small_model
    bpa = np.full(s.n_atoms, s.box[0])
    x1, v1, _, _, _ = G.respa(s.x, v, s.mass, fs, fs, 3.0, 3, 2, box_per_atom=bpa)
    x2, v2, _ = G.velocity_verlet(s.x, v, s.mass, fs, 1.0, 6, box_per_atom=bpa)
    np.testing.assert_allclose(x1, x2, atol=1e-12)
    np.testing.assert_allclose(v1, v2, atol=1e-13)


def test_time_reversibility(water_small_model):
    s, fs, fb, v = water_small_model
    bpa = np.full(s.n_atoms, s.box[0])
    x1, v1, Fs, Fb, _ = G.respa(s.x, v, s.mass, fs, fb, 3.0, 3, 4, box_per_atom=bpa)
    x2, v2, _, _, _ = G.respa(x1, -v1, s.mass, fs, fb, 3.0, 3, 4, box_per_atom=bpa, F_small=Fs, F=Fb)
    L = s.box[0]
    dx = x2 - s.x
    dx -= L * np.round(dx / L)
    assert np.abs(dx).max() < 1e-10
    np.testing.assert_allclose(-v2, v, atol=1e-12)


def test_energy_error_scales_as_dt_squared():
    """Velocity Verlet's total-energy fluctuation over a fixed time span drops
    by ~4x when dt is halved (second-order scheme)."""
    s = I.make_water(2, 10.0, 0)
    spec = M.spec_of(I.small_arch())
    par = I.init_params(I.small_arch(), 2)
    pairs_cache = {}

    def ef(x):
        return M.energy_forces(spec, par, x, s.species, s.atom_offset, s.box)

    v0 = I.maxwell_boltzmann(s.mass, 300.0, 1)
    bpa = np.full(s.n_atoms, s.box[0])
    spans = []
    for dt, n in ((0.5, 40), (0.25, 80)):
        x, v = s.x.copy(), v0.copy()
        E0, F = ef(x)
        tot = []
        for _ in range(n):
            x, v, F = G.velocity_verlet(x, v, s.mass, lambda y: ef(y)[1], dt, 1, box_per_atom=bpa, F=F)
            tot.append(ef(x)[0][0] + G.kinetic_energy(v, s.mass)[0])
        tot = np.array(tot)
        spans.append(tot.max() - tot.min())
    ratio = spans[0] / spans[1]
    assert 3.0 < ratio < 5.0, ratio
    del pairs_cache


def test_respa_energies_output(water_small_model):
    s, fs, fb, v = water_small_model
    specb = M.spec_of(I.big_arch())
    parb = I.init_params(I.big_arch(), 3)
    eb = lambda x: M.energy(specb, parb, x, s.species, s.atom_offset, s.box).numpy()  # noqa: E731
    bpa = np.full(s.n_atoms, s.box[0])
    x, vv, _, _, en = G.respa(s.x, v, s.mass, fs, fb, 3.0, 3, 2, box_per_atom=bpa, energy_big=eb)
    assert en.shape == (2, 1, 3)
    np.testing.assert_allclose(en[-1, 0, 0], eb(x)[0], rtol=1e-14)
    np.testing.assert_allclose(en[-1, 0, 1], G.kinetic_energy(vv, s.mass)[0], rtol=1e-14)
