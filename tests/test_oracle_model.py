"""Pins of the oracle's potential: closed forms, finite differences and
invariances (CPU only).

The model is the invariant message-passing potential that stands in for the
paper's large and distilled small models (section "Neural Network
Architectures"); forces F = -dE/dx are what Algorithm 1 consumes.
"""
import math

import numpy as np
import pytest
import torch

from oracle import model as M
from paper_2510_06562_gb300 import inputs as I

SILU = lambda a: a / (1.0 + math.exp(-a))  # noqa: E731


def _small_water(seed=0):
    # 8 rigid waters in a 10 A box: periodic and at least twice the 5 A cutoff
    return I.make_water(2, 10.0, seed)


@pytest.fixture(scope="module")
def models():
    return [(M.spec_of(I.big_arch()), I.init_params(I.big_arch(), 3)),
            (M.spec_of(I.small_arch()), I.init_params(I.small_arch(), 2))]


# ---------------------------------------------------------------- basis ----

def test_bessel_closed_form_values():
    rc, K = 5.0, 16
    d = torch.tensor([rc / 2], dtype=torch.float64)
    e = M.bessel_basis(d, rc, K)[0].numpy()
    ref = [math.sqrt(2 / rc) * math.sin(k * math.pi / 2) / (rc / 2) for k in range(1, K + 1)]
    np.testing.assert_allclose(e, ref, rtol=1e-14, atol=1e-15)
    # d -> 0 limit is k pi / rc * sqrt(2 / rc)
    e0 = M.bessel_basis(torch.tensor([1e-9], dtype=torch.float64), rc, K)[0].numpy()
    np.testing.assert_allclose(e0, [k * math.pi / rc * math.sqrt(2 / rc) for k in range(1, K + 1)], rtol=1e-12)
    # zero at the cutoff
    ec = M.bessel_basis(torch.tensor([rc], dtype=torch.float64), rc, K)[0].numpy()
    assert np.max(np.abs(ec)) < 1e-14


def test_cosine_cutoff_values_and_smoothness():
    rc = 3.5
    d = torch.tensor([0.0, rc / 2, rc, rc + 1.0], dtype=torch.float64)
    np.testing.assert_allclose(M.cosine_cutoff(d, rc).numpy(), [1.0, 0.5, 0.0, 0.0], atol=1e-15)
    h = 1e-6  # C1 at rc: one-sided slopes vanish
    left = (M.cosine_cutoff(torch.tensor([rc], dtype=torch.float64), rc)
            - M.cosine_cutoff(torch.tensor([rc - h], dtype=torch.float64), rc)) / h
    assert abs(float(left)) < 1e-5


# ------------------------------------------------------ closed-form cases ---

def _one_feature_params(a, p, q, r, s, t, u1, v1, u2, v2, r1, dd1, r2, dd2, z):
    return np.array([a, p, q, r, s, t, u1, v1, u2, v2, r1, dd1, r2, dd2, z], dtype=np.float64)


@pytest.mark.parametrize("dist", [0.7, 1.9, 2.9, 3.2])
def test_two_atom_one_feature_closed_form(dist):
    """S=F=K=Lr=1: every block is a scalar, so E(d) of a dimer is a closed
    form; d >= rc leaves only the self terms."""
    rc = 3.0
    spec = M.Spec(rc, 1, 1, 1, 1)
    vals = dict(a=0.8, p=-1.3, q=1.7, r=0.2, s=-0.9, t=0.4, u1=1.1, v1=-0.3, u2=0.7,
                v2=0.05, r1=-1.2, dd1=0.1, r2=0.6, dd2=-0.2, z=0.35)
    par = _one_feature_params(**vals)
    x = np.array([[0.0, 0.0, 0.0], [dist, 0.0, 0.0]])
    E = float(M.energy(spec, par, x, np.array([0, 0]), [0, 2], [0.0])[0])
    v = vals
    if dist < rc:
        e = math.sqrt(2 / rc) * math.sin(math.pi * dist / rc) / dist
        fc = 0.5 * (math.cos(math.pi * dist / rc) + 1)
        w = fc * (SILU(v["q"] * e + v["r"]) * v["s"] + v["t"])
        m = w * v["a"] * v["p"]
    else:
        m = 0.0
    h1 = v["a"] + SILU(m * v["u1"] + v["v1"]) * v["u2"] + v["v2"]
    Ei = SILU(h1 * v["r1"] + v["dd1"]) * v["r2"] + v["dd2"] + v["z"]
    assert abs(E - 2 * Ei) < 1e-13


def test_two_feature_routing_closed_form():
    """F=2 with off-diagonal 0/1 matrices: each product routes one feature
    into the other, so a transposed operand or a misplaced bias zeroes or
    changes the closed-form result E = 2 SiLU(SiLU(fc(d) t alpha))."""
    rc, d, alpha, t = 4.0, 1.6, 1.4, 0.9
    spec = M.Spec(rc, 1, 1, 2, 1)
    A = [alpha, 0.0]
    W_in = [[0, 1], [0, 0]]
    W1, b1 = [[0, 2.0]], [0, 0]
    W2, b2 = [[0, 0], [1, 0]], [0, t]
    U1, c1 = [[0, 0], [1, 0]], [0, 0]
    U2, c2 = [[0, 1], [0, 0]], [0, 0]
    R1, d1 = [[0, 0], [1, 0]], [0, 0]
    R2, d2, e0 = [1, 0], [0], [0]
    par = np.concatenate([np.ravel(b) for b in (A, W_in, W1, b1, W2, b2, U1, c1, U2, c2, R1, d1, R2, d2, e0)]).astype(float)
    x = np.array([[0.0, 0, 0], [0, d, 0]])
    E = float(M.energy(spec, par, x, np.array([0, 0]), [0, 2], [0.0])[0])
    fc = 0.5 * (math.cos(math.pi * d / rc) + 1)
    assert abs(E - 2 * SILU(SILU(fc * t * alpha))) < 1e-14


def test_parameter_layout_matches_generator():
    for arch in (I.big_arch(), I.small_arch(), I.big_arch(4)):
        spec = M.spec_of(arch)
        p = np.arange(arch.param_count(), dtype=np.float64)
        P = M.parse_params(spec, p)
        sl = I.param_slices(arch)
        for key, (off, shape) in sl.items():
            if isinstance(key, tuple):
                got = P["layers"][key[0]][key[1]]
            else:
                got = P[key]
            np.testing.assert_array_equal(got.numpy().reshape(shape), p[off:off + int(np.prod(shape))].reshape(shape))
    with pytest.raises(ValueError):
        M.parse_params(M.spec_of(I.small_arch()), np.zeros(10))


# ------------------------------------------------------- derivatives -------

@pytest.mark.parametrize("which", [0, 1])
def test_forces_match_central_differences(models, which):
    spec, par = models[which]
    s = _small_water()
    E, F = M.energy_forces(spec, par, s.x, s.species, s.atom_offset, s.box)
    rng = np.random.default_rng(5)
    h = 1e-4
    pairs = M.pair_list(s.x, s.atom_offset, s.box, spec.cutoff)
    # individual coordinates and random directions
    dirs = []
    for k in rng.choice(s.n_atoms * 3, 6, replace=False):
        dv = np.zeros(s.n_atoms * 3)
        dv[k] = 1.0
        dirs.append(dv)
    for _ in range(3):
        dv = rng.normal(size=s.n_atoms * 3)
        dirs.append(dv / np.linalg.norm(dv))
    for dv in dirs:
        dv = dv.reshape(-1, 3)
        Ep = float(M.energy(spec, par, s.x + h * dv, s.species, s.atom_offset, s.box, pairs)[0])
        Em = float(M.energy(spec, par, s.x - h * dv, s.species, s.atom_offset, s.box, pairs)[0])
        fd = -(Ep - Em) / (2 * h)
        an = float((F * dv).sum())
        assert abs(fd - an) <= 1e-7 * max(1.0, np.abs(F).max()), (fd, an)


def test_forces_fd_vacuum_molecule(models):
    spec, par = models[0]
    b = I.make_vacuum_batch(3, 12, 20, seed=4)
    spec4 = spec._replace(n_species=4)
    par4 = I.init_params(I.big_arch(4), 9)
    E, F = M.energy_forces(spec4, par4, b.x, b.species, b.atom_offset, b.box)
    assert E.shape == (3,)
    h = 1e-4
    rng = np.random.default_rng(0)
    for _ in range(4):
        dv = rng.normal(size=b.x.shape)
        dv /= np.linalg.norm(dv)
        Ep = M.energy(spec4, par4, b.x + h * dv, b.species, b.atom_offset, b.box).sum()
        Em = M.energy(spec4, par4, b.x - h * dv, b.species, b.atom_offset, b.box).sum()
        assert abs(-(float(Ep) - float(Em)) / (2 * h) - float((F * dv).sum())) < 1e-7 * max(1, np.abs(F).max())


# ------------------------------------------------------- invariances -------

def test_translation_invariance_across_wrap(models):
    s = _small_water()
    for spec, par in models:
        E0, F0 = M.energy_forces(spec, par, s.x, s.species, s.atom_offset, s.box)
        shift = np.array([7.3, -2.9, 4.45])
        xs = s.x + shift
        xs = xs - s.box[0] * np.floor(xs / s.box[0])
        E1, F1 = M.energy_forces(spec, par, xs, s.species, s.atom_offset, s.box)
        assert abs(E1[0] - E0[0]) <= 1e-12 * abs(E0[0]) + 1e-12
        np.testing.assert_allclose(F1, F0, atol=1e-11)
        # zero net force (consequence of translation invariance)
        assert np.abs(F0.sum(0)).max() <= 1e-12 * s.n_atoms * np.abs(F0).max()


def test_permutation_invariance(models):
    s = _small_water()
    rng = np.random.default_rng(3)
    perm = rng.permutation(s.n_atoms)
    for spec, par in models:
        E0, F0 = M.energy_forces(spec, par, s.x, s.species, s.atom_offset, s.box)
        E1, F1 = M.energy_forces(spec, par, s.x[perm], s.species[perm], s.atom_offset, s.box)
        assert abs(E1[0] - E0[0]) <= 1e-12 * abs(E0[0])
        np.testing.assert_allclose(F1, F0[perm], atol=1e-12)


def _cubic_ops():
    import itertools
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3))
            for a in range(3):
                R[a, perm[a]] = signs[a]
            yield R


def test_cubic_symmetry_invariance_periodic(models):
    s = _small_water()
    L = s.box[0]
    c = np.full(3, L / 2)
    spec, par = models[1]
    E0, F0 = M.energy_forces(spec, par, s.x, s.species, s.atom_offset, s.box)
    ops = list(_cubic_ops())
    assert len(ops) == 48
    for R in ops:
        xr = (s.x - c) @ R.T + c
        xr = xr - L * np.floor(xr / L)
        E1, F1 = M.energy_forces(spec, par, xr, s.species, s.atom_offset, s.box)
        assert abs(E1[0] - E0[0]) <= 1e-12 * abs(E0[0])
        np.testing.assert_allclose(F1, F0 @ R.T, atol=1e-11)
    specb, parb = models[0]
    Eb, _ = M.energy_forces(specb, parb, s.x, s.species, s.atom_offset, s.box)
    for R in ops[::7]:
        xr = (s.x - c) @ R.T + c
        xr = xr - L * np.floor(xr / L)
        assert abs(M.energy(specb, parb, xr, s.species, s.atom_offset, s.box)[0] - Eb[0]) <= 1e-12 * abs(Eb[0])


def test_rotation_invariance_vacuum():
    b = I.make_vacuum_batch(2, 20, 30, seed=7)
    spec = M.spec_of(I.big_arch(4))
    par = I.init_params(I.big_arch(4), 11)
    E0, F0 = M.energy_forces(spec, par, b.x, b.species, b.atom_offset, b.box)
    rng = np.random.default_rng(1)
    for _ in range(3):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        if np.linalg.det(Q) < 0:
            Q[:, 0] *= -1
        E1, F1 = M.energy_forces(spec, par, b.x @ Q.T + 3.0, b.species, b.atom_offset, b.box)
        np.testing.assert_allclose(E1, E0, rtol=1e-12)
        np.testing.assert_allclose(F1, F0 @ Q.T, atol=1e-11)


# ------------------------------------------------------------ virial -------

def test_virial_matches_strain_differences(models):
    s = _small_water()
    spec, par = models[0]
    pairs = M.pair_list(s.x, s.atom_offset, s.box, spec.cutoff)
    W = M.virial(spec, par, s.x, s.species, s.atom_offset, s.box, pairs)[0]
    h = 1e-6
    for a in range(3):
        for b in range(3):
            eps = np.zeros((3, 3))
            eps[a, b] = h
            Ep = M.strained_energy(spec, par, s.x, s.species, s.atom_offset, s.box, eps, pairs)
            Em = M.strained_energy(spec, par, s.x, s.species, s.atom_offset, s.box, -eps, pairs)
            assert abs(-(Ep - Em) / (2 * h) - W[a, b]) < 1e-6 * max(1.0, np.abs(W).max())
    # symmetric (rotation invariance of the energy)
    np.testing.assert_allclose(W, W.T, atol=1e-10 * np.abs(W).max())


def test_virial_equals_sum_r_outer_f_in_vacuum():
    b = I.make_vacuum_batch(2, 15, 25, seed=2)
    spec = M.spec_of(I.small_arch(4))
    par = I.init_params(I.small_arch(4), 5)
    W = M.virial(spec, par, b.x, b.species, b.atom_offset, b.box)
    _, F = M.energy_forces(spec, par, b.x, b.species, b.atom_offset, b.box)
    for sidx in range(2):
        a, e = b.atom_offset[sidx], b.atom_offset[sidx + 1]
        np.testing.assert_allclose(W[sidx], b.x[a:e].T @ F[a:e], atol=1e-11)


# ------------------------------------------------- distillation gradient ---

def test_force_matching_gradient_finite_differences():
    s = _small_water()
    spec = M.spec_of(I.small_arch())
    par = I.init_params(I.small_arch(), 2)
    rng = np.random.default_rng(0)
    frames = np.stack([s.x, s.x + rng.normal(scale=0.05, size=s.x.shape)])
    f_ref = rng.normal(scale=0.5, size=frames.shape)
    L, g = M.force_matching_grad(spec, par, frames, s.species, s.atom_offset, s.box, f_ref)
    assert L > 0 and g.shape == par.shape
    h = 1e-5
    for _ in range(3):
        dv = rng.normal(size=par.shape)
        dv /= np.linalg.norm(dv)
        Lp = float(M.force_matching_loss(spec, par + h * dv, frames, s.species, s.atom_offset, s.box, f_ref))
        Lm = float(M.force_matching_loss(spec, par - h * dv, frames, s.species, s.atom_offset, s.box, f_ref))
        assert abs((Lp - Lm) / (2 * h) - g @ dv) < 1e-7 * max(1.0, np.abs(g).max())
    # single-coordinate checks on a few parameters, including biases and e0
    for k in [0, 70, len(par) - 1, len(par) - 3]:
        dv = np.zeros_like(par)
        dv[k] = 1
        Lp = float(M.force_matching_loss(spec, par + h * dv, frames, s.species, s.atom_offset, s.box, f_ref))
        Lm = float(M.force_matching_loss(spec, par - h * dv, frames, s.species, s.atom_offset, s.box, f_ref))
        assert abs((Lp - Lm) / (2 * h) - g[k]) < 1e-7 * max(1.0, np.abs(g).max())
    # e0 shifts energies only, never forces: its gradient is exactly zero
    assert np.all(g[-2:] == 0.0)


def test_force_matching_gradient_is_tangent_of_energy_gradient():
    """dL/dtheta = (2 / (3 N M)) sum_m (F_m - F_ref_m) . dF_m/dtheta and, since
    F = -dE/dx, (g . dF/dtheta) = -d/deps [dE/dtheta(x + eps g)] at eps = 0."""
    s = _small_water(1)
    spec = M.spec_of(I.small_arch())
    par = I.init_params(I.small_arch(), 2)
    rng = np.random.default_rng(2)
    frames = s.x[None]
    f_ref = rng.normal(scale=0.5, size=frames.shape)
    _, grad = M.force_matching_grad(spec, par, frames, s.species, s.atom_offset, s.box, f_ref)
    _, F = M.energy_forces(spec, par, s.x, s.species, s.atom_offset, s.box)
    g = 2.0 * (F - f_ref[0]) / (3.0 * s.n_atoms)
    pairs = M.pair_list(s.x, s.atom_offset, s.box, spec.cutoff)

    def dE_dtheta(x):
        th = torch.tensor(par, requires_grad=True)
        E = M.energy(spec, th, x, s.species, s.atom_offset, s.box, pairs).sum()
        return torch.autograd.grad(E, th)[0].numpy()

    eps = 1e-5
    tang = -(dE_dtheta(s.x + eps * g) - dE_dtheta(s.x - eps * g)) / (2 * eps)
    np.testing.assert_allclose(grad, tang, atol=1e-8 * max(1.0, np.abs(grad).max()))


@pytest.mark.parametrize("dist", [0.3, 0.96, 1.7, 2.5])
def test_pair_repulsion_closed_form(dist):
    """With every network parameter zero the energy of a dimer is the pair
    repulsion alone: E = a exp(-d/rho) (cos(pi d/r) + 1)/2 for d < r, else 0
    (each directed pair contributes half)."""
    a, rho, r = 50.0, 0.2, 2.0
    spec = M.Spec(3.0, 2, 1, 2, 1, a, rho, r)
    n = 2 + (4 * 4 + 2 * 2 + 4 * 2) + 4 + 2 + 2 + 1 + 1
    par = np.zeros(n)
    x = np.array([[0.0, 0, 0], [dist, 0, 0]])
    E, F = M.energy_forces(spec, par, x, np.array([0, 0]), [0, 2], [0.0])
    ref = a * math.exp(-dist / rho) * 0.5 * (math.cos(math.pi * dist / r) + 1) if dist < r else 0.0
    assert abs(E[0] - ref) <= 1e-12 * max(1.0, ref)
    # force on atom 1 along +x is -dE/dd
    dref = 0.0
    if dist < r:
        dref = a * math.exp(-dist / rho) * (-0.5 * (math.cos(math.pi * dist / r) + 1) / rho
                                            - 0.5 * math.pi / r * math.sin(math.pi * dist / r))
    assert abs(F[1, 0] + dref) <= 1e-10 * max(1.0, abs(dref))
    assert abs(F[0, 0] - dref) <= 1e-10 * max(1.0, abs(dref))


def test_distill_gradient_finite_differences():
    """Energy + force loss: dL/dtheta against central differences of L in
    theta, along random directions and for single parameters including d2
    and e0 (which the energy term moves and the force term does not)."""
    s = _small_water()
    spec = M.spec_of(I.small_arch())
    par = I.init_params(I.small_arch(), 2)
    rng = np.random.default_rng(4)
    frames = np.stack([s.x, s.x + rng.normal(scale=0.05, size=s.x.shape)])
    f_ref = rng.normal(scale=0.5, size=frames.shape)
    e_ref = np.array([1.5, -2.0]) * s.n_atoms
    lam = 0.7
    L, g = M.distill_grad(spec, par, frames, s.species, s.atom_offset, s.box, f_ref, e_ref, lam)
    h = 1e-5

    def loss(p):
        return float(M.distill_loss(spec, p, frames, s.species, s.atom_offset, s.box, f_ref, e_ref, lam))

    for _ in range(3):
        dv = rng.normal(size=par.shape)
        dv /= np.linalg.norm(dv)
        assert abs((loss(par + h * dv) - loss(par - h * dv)) / (2 * h) - g @ dv) < 1e-7 * max(1.0, np.abs(g).max())
    for k in [0, 70, len(par) - 1, len(par) - 2, len(par) - 3]:
        dv = np.zeros_like(par)
        dv[k] = 1
        assert abs((loss(par + h * dv) - loss(par - h * dv)) / (2 * h) - g[k]) < 1e-7 * max(1.0, np.abs(g).max())
    assert abs(L - loss(par)) <= 1e-12 * L


def test_distill_energy_term_closed_forms():
    """lambda_e = 0 is the force-matching loss; the gradient's d2 and e0
    entries come from the energy term alone and have closed forms:
    dL/dd2 = 2 lambda_e / M sum_m (E_m - E_ref,m) / N (every atom adds d2
    once) and dL/de0[s] = 2 lambda_e / M sum_m (E_m - E_ref,m) n_s / N^2."""
    s = _small_water(1)
    spec = M.spec_of(I.small_arch())
    par = I.init_params(I.small_arch(), 2)
    rng = np.random.default_rng(5)
    frames = np.stack([s.x, s.x + rng.normal(scale=0.05, size=s.x.shape)])
    f_ref = rng.normal(scale=0.5, size=frames.shape)
    e_ref = np.array([0.3, -0.4]) * s.n_atoms
    L0, g0 = M.distill_grad(spec, par, frames, s.species, s.atom_offset, s.box, f_ref, e_ref, 0.0)
    Lf, gf = M.force_matching_grad(spec, par, frames, s.species, s.atom_offset, s.box, f_ref)
    assert abs(L0 - Lf) <= 1e-12 * Lf
    np.testing.assert_allclose(g0, gf, rtol=0, atol=1e-13 * np.abs(gf).max())
    lam = 2.0
    _, g = M.distill_grad(spec, par, frames, s.species, s.atom_offset, s.box, f_ref, e_ref, lam)
    E = np.array([M.energy(spec, par, f, s.species, s.atom_offset, s.box).sum().item() for f in frames])
    N, Mf = s.n_atoms, len(frames)
    r = (E - e_ref) / N
    n_s = np.bincount(s.species, minlength=spec.n_species)
    S = spec.n_species
    assert abs(g[-1 - S] - 2 * lam / Mf * r.sum()) <= 1e-12 * max(1.0, abs(g[-1 - S]))
    np.testing.assert_allclose(g[-S:], 2 * lam / Mf * r.sum() * n_s / N, rtol=1e-12, atol=0)


def test_adam_first_step_and_constant_gradient():
    """Adam's first step moves each parameter by lr g / (|g| + eps) against
    its gradient (both bias corrections are exact at t = 1); under a constant
    gradient every later step does the same, since m_hat = g and
    v_hat = g^2 at every t."""
    rng = np.random.default_rng(0)
    th = rng.normal(size=50)
    g = rng.normal(size=50)
    m = np.zeros(50)
    v = np.zeros(50)
    lr, eps = 1e-3, 1e-8
    t1, m, v = M.adam_step(th, g, m, v, 1, lr, eps=eps)
    np.testing.assert_allclose(t1, th - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    t = t1
    for k in range(2, 6):
        t_new, m, v = M.adam_step(t, g, m, v, k, lr, eps=eps)
        np.testing.assert_allclose(t_new, t - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-14)
        t = t_new

