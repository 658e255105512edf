"""Pins of the oracle's Langevin pieces (CPU only): the counter-based
generator, the Box-Muller normals, the exact Ornstein-Uhlenbeck O-step,
Algorithm 1 with the thermostat (BAOAB-RESPA) and velocity Verlet as BAOAB,
hydrogen mass repartitioning, and the force-difference monitor with its
single-time-step fallback.

The generator is pinned by its published known-answer vectors (stored in
tests/golden with their source) and by properties a mistake in a multiplier,
a shift, a word order or the key schedule destroys (injectivity on a sample,
avalanche, uniformity, bit balance); the thermostat by the exact moments of the
Ornstein-Uhlenbeck process, by equipartition, and by the temperature an
ensemble of harmonic oscillators reaches under the full integrator.
"""
import os

import numpy as np
import pytest

from oracle import integrate as G

KT300 = G.KB_EV * 300.0
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_philox_kat():
    """(counters [n, 4], keys [n, 2], outputs [n, 4]) of the published
    Philox-4x32-10 known-answer vectors."""
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(w, 16) for w in line.split()])
    a = np.array(rows, dtype=np.uint64)
    return a[:, 0:4], a[:, 4:6], a[:, 6:10]


def test_philox_known_answer_vectors():
    """The oracle's generator reproduces every published vector word for word:
    a wrong multiplier, Weyl constant, round count or output order fails."""
    ctr, key, out = load_philox_kat()
    assert len(ctr) == 3
    for c, k, o in zip(ctr, key, out):
        np.testing.assert_array_equal(G.philox4x32_10(c[None, :], k)[0].astype(np.uint64), o)


def _words(n, key=(7, 11), hi=0):
    i = np.arange(n, dtype=np.uint64)
    ctr = np.stack([i, np.full_like(i, hi), np.zeros_like(i), np.zeros_like(i)], axis=1)
    return G.philox4x32_10(ctr, key)


def test_philox_injective_on_a_sample_and_key_dependent():
    w = _words(1 << 16)
    packed = {tuple(r) for r in w.tolist()}
    assert len(packed) == 1 << 16
    w2 = _words(1 << 10, key=(8, 11))
    assert np.all(np.any(w2 != w[: 1 << 10], axis=1))
    # the high counter words matter too
    w3 = _words(1 << 10, hi=1)
    assert np.all(np.any(w3 != w[: 1 << 10], axis=1))


def test_philox_avalanche():
    rng = np.random.default_rng(0)
    base = rng.integers(0, 2 ** 32, size=(2000, 4), dtype=np.uint64)
    flips = []
    for bit in (0, 13, 31):
        for word in range(4):
            c2 = base.copy()
            c2[:, word] ^= np.uint64(1 << bit)
            a = G.philox4x32_10(base, (3, 5)).astype(np.uint64)
            b = G.philox4x32_10(c2, (3, 5)).astype(np.uint64)
            x = a ^ b
            n = sum(int(bin(int(v)).count("1")) for v in x.reshape(-1)) / len(base)
            flips.append(n)
    # a random 128-bit change flips 64 bits on average (sd of the mean ~0.13)
    assert all(abs(f - 64.0) < 1.0 for f in flips), flips


def test_philox_uniform_and_bit_balanced():
    w = _words(1 << 17).reshape(-1).astype(np.uint64)
    n = len(w)
    u = (w.astype(np.float64) + 0.5) / 2 ** 32
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    counts = np.bincount((u * 64).astype(int), minlength=64)
    exp = n / 64
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 63 + 6 * np.sqrt(2 * 63)              # 63 dof, ~6 sigma
    for b in range(32):
        frac = ((w >> np.uint64(b)) & np.uint64(1)).mean()
        assert abs(frac - 0.5) < 5 * 0.5 / np.sqrt(n)
    lag = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(lag) < 5 / np.sqrt(n)


def test_normals_moments():
    z = G.langevin_normals(200_000, step=3, seed=12345)
    n = len(z)
    for c in range(3):
        x = z[:, c]
        assert abs(x.mean()) < 5 / np.sqrt(n)
        assert abs(x.var() - 1.0) < 5 * np.sqrt(2 / n)
        assert abs((x ** 3).mean()) < 5 * np.sqrt(15 / n)
        assert abs((x ** 4).mean() - 3.0) < 5 * np.sqrt(96 / n)
    c01 = np.corrcoef(z[:, 0], z[:, 1])[0, 1]
    c02 = np.corrcoef(z[:, 0], z[:, 2])[0, 1]
    assert abs(c01) < 5 / np.sqrt(n) and abs(c02) < 5 / np.sqrt(n)
    # different inner steps and seeds give independent draws
    assert abs(np.corrcoef(z[:, 0], G.langevin_normals(n, 4, 12345)[:, 0])[0, 1]) < 5 / np.sqrt(n)
    assert abs(np.corrcoef(z[:, 0], G.langevin_normals(n, 3, 12346)[:, 0])[0, 1]) < 5 / np.sqrt(n)


def test_o_step_without_friction_is_the_identity():
    rng = np.random.default_rng(1)
    v = rng.normal(size=(50, 3))
    m = rng.uniform(1, 16, size=50)
    out = G.o_step(v, m, 1.0, {"gamma": 0.0, "temperature": 300.0, "seed": 9}, 5)
    np.testing.assert_array_equal(out, v)


@pytest.mark.parametrize("gamma_h", [0.05, 0.7, 3.0])
def test_o_step_exact_ou_moments(gamma_h):
    n = 200_000
    m = np.full(n, 12.0)
    v0 = np.tile(np.array([[0.01, -0.02, 0.005]]), (n, 1))
    h = 1.0
    th = {"gamma": gamma_h / h, "temperature": 300.0, "seed": 77}
    v = G.o_step(v0, m, h, th, step=0)
    c1 = np.exp(-gamma_h)
    var = (1 - c1 * c1) * KT300 * G.ACCEL / 12.0
    for c in range(3):
        assert abs(v[:, c].mean() - c1 * v0[0, c]) < 5 * np.sqrt(var / n)
        assert abs(v[:, c].var() / var - 1.0) < 5 * np.sqrt(2 / n)


def test_o_step_equipartition_from_rest():
    n = 100_000
    m = np.where(np.arange(n) % 3 == 0, 15.999, 1.008)
    v = np.zeros((n, 3))
    th = {"gamma": 0.5, "temperature": 300.0, "seed": 3}
    for s in range(12):                     # c1^12 = exp(-6)
        v = G.o_step(v, m, 1.0, th, step=s)
    ke = 0.5 * m[:, None] * v ** 2 * G.KE_EV          # per component
    for sel in (m > 2, m < 2):
        assert abs(ke[sel].mean() / (0.5 * KT300) - 1.0) < 0.02


def test_langevin_respa_at_zero_friction_equals_nve():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(30, 3))
    v = rng.normal(size=(30, 3)) * 0.01
    m = rng.uniform(1, 16, size=30)
    fs = lambda y: -0.5 * y
    fb = lambda y: -0.7 * y
    a = G.respa(x, v, m, fs, fb, 3.0, 3, 4)
    b = G.respa(x, v, m, fs, fb, 3.0, 3, 4, thermo={"gamma": 0.0, "temperature": 300.0, "seed": 1})
    for p, q in zip(a[:4], b[:4]):
        np.testing.assert_array_equal(p, q)


@pytest.mark.parametrize("scheme", ["respa", "baoab"])
def test_langevin_ensemble_reaches_the_bath_temperature(scheme):
    """Independent 3D harmonic oscillators (k = 1 eV/A^2, m = 16 amu, period
    ~256 fs) thermalised from rest: both the kinetic temperature and the
    configurational one (<k x^2> = k_B T per component) reach 300 K. A wrong
    unit factor, a misplaced O-step or a wrong c2 moves them far off."""
    n, k, m0 = 3000, 1.0, 16.0
    m = np.full(n, m0)
    f = lambda y: -k * y
    th = {"gamma": 0.02, "temperature": 300.0, "seed": 2024}
    x = np.zeros((n, 3))
    v = np.zeros((n, 3))
    ke, pe = [], []
    if scheme == "respa":
        Fs = F = None
        for s in range(400):
            x, v, Fs, F, _ = G.respa(x, v, m, f, f, 2.0, 2, 1, F_small=Fs, F=F, thermo=th, step0=2 * s)
            if s >= 200:
                ke.append((0.5 * m[:, None] * v ** 2 * G.KE_EV).mean())
                pe.append((0.5 * k * x ** 2).mean())
    else:
        F = None
        for s in range(400):
            x, v, F = G.velocity_verlet(x, v, m, f, 2.0, 2, F=F, thermo=th, step0=2 * s)
            if s >= 200:
                ke.append((0.5 * m[:, None] * v ** 2 * G.KE_EV).mean())
                pe.append((0.5 * k * x ** 2).mean())
    assert abs(np.mean(ke) / (0.5 * KT300) - 1.0) < 0.03
    assert abs(np.mean(pe) / (0.5 * KT300) - 1.0) < 0.03


def test_hmr_masses_water_and_conservation():
    # two waters O H H and a lone hydrogen and a hydrogen-hydrogen "bond"
    m = np.array([15.999, 1.008, 1.008, 15.999, 1.008, 1.008, 1.008, 1.008])
    bonds = np.array([[0, 1], [0, 2], [3, 4], [5, 3], [6, 7]])
    out = G.hmr_masses(m, bonds, h_mass=3.024)
    np.testing.assert_allclose(out[[1, 2, 4, 5]], 3.024)
    np.testing.assert_allclose(out[[0, 3]], 15.999 - 2 * (3.024 - 1.008))
    np.testing.assert_array_equal(out[[6, 7]], m[[6, 7]])
    assert abs(out.sum() - m.sum()) < 1e-12
    # a hydrogen bonded to two heavy atoms moves mass from the first only
    out2 = G.hmr_masses(np.array([12.011, 1.008, 14.007]), np.array([[1, 0], [1, 2]]))
    np.testing.assert_allclose(out2, [12.011 - 2.016, 3.024, 14.007])
    with pytest.raises(ValueError):
        G.hmr_masses(np.array([2.0, 1.0]), np.array([[0, 1]]), h_mass=3.5)


# ------------------------------------------------------------------ force-difference monitor

def _harmonic_pair(k_small, k_big):
    return (lambda y: -k_small * y), (lambda y: -k_big * y)


def test_monitor_never_tripping_is_plain_respa():
    rng = np.random.default_rng(5)
    x, v = rng.normal(size=(20, 3)), rng.normal(size=(20, 3)) * 0.02
    m = rng.uniform(1, 16, size=20)
    fs, fb = _harmonic_pair(0.4, 0.5)
    a = G.respa(x, v, m, fs, fb, 3.0, 3, 5)
    b = G.respa_monitored(x, v, m, fs, fb, 3.0, 3, 5, threshold=np.inf)
    for p, q in zip(a[:4], b[:4]):
        np.testing.assert_array_equal(p, q)
    assert b[4] == 0
    # the reported maximum is the largest end-of-step force difference
    assert abs(b[5] - max(G.force_difference_norms(fb(x_), fs(x_)).max()
                          for x_ in [G.respa(x, v, m, fs, fb, 3.0, 3, s)[0] for s in range(1, 6)])) < 1e-12


@pytest.mark.parametrize("thermo", [None, {"gamma": 0.05, "temperature": 300.0, "seed": 4}])
def test_monitor_always_tripping_is_single_time_step(thermo):
    """With a zero threshold every outer step falls back: the trajectory is
    n_slow x n_outer steps of the single-time-step integrator at dt / n_slow
    with the large model, drawing the same noise counters."""
    rng = np.random.default_rng(6)
    x, v = rng.normal(size=(20, 3)), rng.normal(size=(20, 3)) * 0.02
    m = rng.uniform(1, 16, size=20)
    fs, fb = _harmonic_pair(0.4, 0.9)
    xr, vr, Fr = G.velocity_verlet(x, v, m, fb, 1.0, 12, thermo=thermo, step0=0)
    xm, vm, Fsm, Fm, nf, _ = G.respa_monitored(x, v, m, fs, fb, 3.0, 3, 4, threshold=0.0, thermo=thermo)
    np.testing.assert_allclose(xm, xr, rtol=0, atol=1e-13)
    np.testing.assert_allclose(vm, vr, rtol=0, atol=1e-13)
    np.testing.assert_allclose(Fsm, fs(xm))
    assert nf == 4


def test_monitor_trips_only_on_large_differences():
    """A small model that is wrong only far from the origin: steps whose end
    state has an atom there fall back, the others do not."""
    rng = np.random.default_rng(7)
    n = 10
    x = rng.normal(size=(n, 3)) * 0.2
    x[0] = [2.0, 0.0, 0.0]                              # starts in the bad region, moving out of it
    v = np.zeros((n, 3))
    v[0] = [-0.2, 0.0, 0.0]
    m = np.full(n, 12.0)
    fb = lambda y: -0.5 * y
    fs = lambda y: -0.5 * y + np.where(np.linalg.norm(y, axis=1, keepdims=True) > 1.5, 3.0, 0.0)
    out = G.respa_monitored(x, v, m, fs, fb, 2.0, 2, 6, threshold=1.0)
    assert 1 <= out[4] < 6
