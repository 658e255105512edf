"""GPU parity of the CUDA path against the FP64 oracle (needs a GB300).

Tolerances (FP32 path): energy |E_gpu - E_ref| / N <= 1e-6 eV/atom and force
RMSE over all 3N components <= 1e-5 eV/A. Neighbour pair sets are compared
bit-exactly (the FP64 cutoff decision is reproduced on the GPU).
"""
import json

import numpy as np
import pytest

from oracle import integrate as G
from oracle import model as M
from paper_2510_06562_gb300 import dmts as D
from paper_2510_06562_gb300 import inputs as I

pytestmark = pytest.mark.gpu

E_TOL = 1e-6     # eV / atom
F_TOL = 1e-5     # eV / A, RMSE


def _models(n_species):
    return (I.small_arch(n_species), I.init_params(I.small_arch(n_species), 2),
            I.big_arch(n_species), I.init_params(I.big_arch(n_species), 3))


def _ctx(s, options=None, small=True):
    sa, sp, ba, bp = _models(s.n_species)
    if small:
        return D.Context(s, ba, bp, sa, sp, options=options)
    return D.Context(s, ba, bp, options=options)


def _pairs(row_ptr, col):
    n = len(row_ptr) - 1
    return np.repeat(np.arange(n), np.diff(row_ptr)), col.astype(np.int64)


def _rmse(a, b):
    return float(np.sqrt(np.mean((np.asarray(a) - np.asarray(b)) ** 2)))


def _with_isolated_atoms():
    """Molecules of 1 to 12 atoms (single-atom molecules have no pairs), and
    in one larger molecule the last atom moved 30 A away: an atom without
    neighbours inside a system that has pairs. Exercises the empty rows of
    every pass (pair lists, tiles and their fix-up, per-atom MLPs)."""
    s = I.make_vacuum_batch(40, 1, 12, seed=5)
    x = s.x.copy()
    sizes = np.diff(s.atom_offset)
    k = int(np.nonzero(sizes >= 4)[0][0])
    x[s.atom_offset[k + 1] - 1] += np.array([30.0, 0.0, 0.0])
    return I.System(x=x, species=s.species, mass=s.mass, atom_offset=s.atom_offset, box=s.box,
                    n_species=s.n_species, name="isolated40", bonds=s.bonds)


def _tiny_molecules():
    """Three non-periodic systems in one context: a dimer (1.2 A), a bent
    triatomic (bonds 1.0 and 1.4 A, 2.1 A apart at the ends) and one rigid
    water molecule; the smallest cases of every pass, with rows of one and
    two pairs."""
    dimer = np.array([[0.0, 0.0, 0.0], [1.2, 0.0, 0.0]])
    tri = np.array([[10.0, 0.0, 0.0], [11.0, 0.0, 0.0], [11.3, 1.37, 0.0]])
    w = I.water_192(0)
    water = w.x[:3] - w.x[0] + np.array([20.0, 0.0, 0.0])
    x = np.concatenate([dimer, tri, water])
    return I.System(x=x, species=np.array([0, 1, 1, 0, 0, 1, 0, 0], np.int32),
                    mass=np.array([1.008, 15.999, 15.999, 1.008, 1.008, 15.999, 1.008, 1.008]),
                    atom_offset=np.array([0, 2, 5, 8], np.int32), box=np.zeros(3), n_species=2, name="tiny3")


SYSTEMS = {
    "tiny3": _tiny_molecules,
    "water192": lambda: I.water_192(0),
    "water12288": lambda: I.water_12288(0),
    "vacuum64": lambda: I.make_vacuum_batch(64, 10, 60, seed=0),
    "isolated40": _with_isolated_atoms,
}


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_neighbor_pairs_bit_exact(name):
    s = SYSTEMS[name]()
    sa, _, ba, _ = _models(s.n_species)
    with _ctx(s) as ctx:
        ctx.set_state(s.x)
        for which, arch in ((D.SMALL, sa), (D.BIG, ba)):
            row_ptr, col = ctx.neighbors(which)
            gi, gj = _pairs(row_ptr, col)
            oi, oj = M.pair_list(s.x, s.atom_offset, s.box, arch.cutoff)
            assert len(gi) == len(oi), (which, len(gi), len(oi))
            np.testing.assert_array_equal(gi, oi)
            np.testing.assert_array_equal(gj, oj)


def test_neighbor_ties_at_the_cutoff():
    """Distances exactly equal to rc (representable) are excluded; distances
    a hair below are included; across the periodic boundary too."""
    L = 16.0
    x = np.array([[1.0, 1.0, 1.0], [6.0, 1.0, 1.0], [1.0, 4.5, 1.0], [1.0, 1.0, 5.999999999],
                  [12.0, 1.0, 1.0], [1.0, 13.5, 1.0], [9.0, 9.0, 9.0], [9.0, 9.0, 12.5],
                  [9.0, 12.49999999, 9.0]])
    s = I.System(x=x, species=np.zeros(len(x), np.int32), mass=np.ones(len(x)),
                 atom_offset=np.array([0, len(x)], np.int32), box=np.array([L]), n_species=2)
    sa, _, ba, _ = _models(2)
    with _ctx(s) as ctx:
        ctx.set_state(x)
        for which, arch in ((D.SMALL, sa), (D.BIG, ba)):
            gi, gj = _pairs(*ctx.neighbors(which))
            oi, oj = M.pair_list(x, s.atom_offset, s.box, arch.cutoff)
            np.testing.assert_array_equal(gi, oi)
            np.testing.assert_array_equal(gj, oj)
        got = set(zip(*_pairs(*ctx.neighbors(D.BIG))))
        assert (0, 1) not in got and (0, 3) in got and (0, 4) not in got


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_energy_forces_fp32(name):
    s = SYSTEMS[name]()
    sa, sp, ba, bp = _models(s.n_species)
    with _ctx(s) as ctx:
        ctx.set_state(s.x)
        for which, arch, par in ((D.SMALL, sa, sp), (D.BIG, ba, bp)):
            E, F = ctx.forces(which)
            Er, Fr = M.energy_forces(M.spec_of(arch), par, s.x, s.species, s.atom_offset, s.box)
            err_e = np.abs(E - Er).max() / max(1, s.n_atoms // s.n_systems)
            err_f = _rmse(F, Fr)
            print(json.dumps({"system": name, "model": "small" if which == 0 else "big",
                              "dE_per_atom": float(np.abs(E - Er).sum() / s.n_atoms),
                              "force_rmse": err_f, "force_rms": float(np.sqrt(np.mean(Fr ** 2)))}))
            assert np.abs(E - Er).sum() / s.n_atoms <= E_TOL
            assert err_e <= E_TOL or s.n_systems > 1
            assert err_f <= F_TOL


def test_virial_fp32():
    s = I.water_192(0)
    sa, sp, ba, bp = _models(2)
    with _ctx(s) as ctx:
        ctx.set_state(s.x)
        for which, arch, par in ((D.SMALL, sa, sp), (D.BIG, ba, bp)):
            _, _, W = ctx.forces(which, virial=True)
            Wr = M.virial(M.spec_of(arch), par, s.x, s.species, s.atom_offset, s.box)
            assert np.abs(W - Wr).max() <= 1e-4 * max(1.0, np.abs(Wr).max())


def test_state_roundtrip_and_device_pointers():
    torch = pytest.importorskip("torch")
    s = I.water_192(0)
    v = I.maxwell_boltzmann(s.mass, 300.0, 1)
    with _ctx(s) as ctx:
        ctx.set_state(s.x, v)
        x1, v1 = ctx.get_state()
        np.testing.assert_array_equal(x1, s.x)
        np.testing.assert_array_equal(v1, v)
        xd = torch.tensor(s.x, device="cuda")
        vd = torch.tensor(v, device="cuda")
        ctx.set_state(xd, vd)
        xo = torch.empty_like(xd)
        vo = torch.empty_like(vd)
        ctx.get_state(xo, vo)
        np.testing.assert_array_equal(xo.cpu().numpy(), s.x)
        Fd = torch.empty_like(xd)
        Ed = torch.empty(1, dtype=torch.float64, device="cuda")
        ctx.forces(D.BIG, f_out=Fd, e_out=Ed)
        E, F = ctx.forces(D.BIG)
        np.testing.assert_array_equal(Fd.cpu().numpy(), F)
        np.testing.assert_array_equal(Ed.cpu().numpy(), E)


def test_wraps_positions_into_box():
    s = I.water_192(0)
    x = s.x + np.array([12.42, -12.42, 2 * 12.42])
    with _ctx(s) as ctx:
        ctx.set_state(x)
        xw, _ = ctx.get_state()
        assert np.all(xw >= 0) and np.all(xw < 12.42)
        E, F = ctx.forces(D.BIG)
        ctx.set_state(s.x)
        E0, F0 = ctx.forces(D.BIG)
        # x + L - L differs from x by FP64 rounding: agreement at FP32 level
        assert abs(E[0] - E0[0]) / s.n_atoms < E_TOL
        assert _rmse(F, F0) < F_TOL


# ------------------------------------------------------------------ dynamics

def _oracle_forces(s, arch, par):
    spec = M.spec_of(arch)
    return lambda x: M.energy_forces(spec, par, x, s.species, s.atom_offset, s.box)[1]


def test_respa_trajectory_water192():
    """Algorithm 1 (3 fs outer, 3 inner steps) on the 192-atom box.

    After 10 outer steps the positions match the oracle to 1e-4 A: a
    relative force perturbation of 1e-6 (the FP32 force error scale) moves
    the oracle's own trajectory by ~1e-6 A there, while a wrong or missing
    kick moves it by >1e-3 A. The dynamics are chaotic (a 1e-6 perturbation
    grows to ~4 A by 100 steps), so over 40 outer steps (120 fs, the window in
    which the random-init models conserve energy) the test compares energy
    conservation with the oracle's own run, and up to 100 steps it checks that
    every reported energy is the oracle's at the GPU's own state."""
    s = I.water_192(0)
    sa, sp, ba, bp = _models(2)
    v0 = I.maxwell_boltzmann(s.mass, 300.0, 1)
    bpa = np.full(s.n_atoms, s.box[0])
    fs, fb = _oracle_forces(s, sa, sp), _oracle_forces(s, ba, bp)
    eb = lambda x: M.energy(M.spec_of(ba), bp, x, s.species, s.atom_offset, s.box).numpy()  # noqa: E731
    xr, vr, Fs, Fb, er = G.respa(s.x, v0, s.mass, fs, fb, 3.0, 3, 10, box_per_atom=bpa, energy_big=eb)
    _, _, _, _, er2 = G.respa(xr, vr, s.mass, fs, fb, 3.0, 3, 30, box_per_atom=bpa,
                              F_small=Fs, F=Fb, energy_big=eb)
    with _ctx(s) as ctx:
        ctx.set_state(s.x, v0)
        eg = ctx.respa_step(10, 3.0, 3)
        xg, vg = ctx.get_state()
        dx = xg - xr
        dx -= s.box[0] * np.round(dx / s.box[0])
        assert np.abs(dx).max() < 1e-4, np.abs(dx).max()
        assert np.abs(vg - vr).max() < 1e-5
        assert np.abs(eg[:, 0, 0] - er[:, 0, 0]).max() / s.n_atoms < E_TOL
        eg2 = ctx.respa_step(30, 3.0, 3)
        etot = np.concatenate([eg[:, 0, 2], eg2[:, 0, 2]])
        etot_ref = np.concatenate([er[:, 0, 2], er2[:, 0, 2]])
        span, span_ref = etot.max() - etot.min(), etot_ref.max() - etot_ref.min()
        print(json.dumps({"etot_span_gpu_120fs": float(span), "etot_span_oracle_120fs": float(span_ref)}))
        assert span < 3.0 * span_ref + 0.05
        eg3 = ctx.respa_step(60, 3.0, 3)
        xg, vg = ctx.get_state()
        assert abs(eg3[-1, 0, 0] - eb(xg)[0]) / s.n_atoms < E_TOL
        assert abs(eg3[-1, 0, 1] - G.kinetic_energy(vg, s.mass)[0]) < 1e-9 * eg3[-1, 0, 1]


def test_velocity_verlet_matches_oracle():
    s = I.water_192(0)
    _, _, ba, bp = _models(2)
    v0 = I.maxwell_boltzmann(s.mass, 300.0, 1)
    bpa = np.full(s.n_atoms, s.box[0])
    xr, vr, _ = G.velocity_verlet(s.x, v0, s.mass, _oracle_forces(s, ba, bp), 1.0, 20, box_per_atom=bpa)
    with _ctx(s, small=False) as ctx:
        ctx.set_state(s.x, v0)
        e = ctx.respa_step(20, 1.0, 1)
        xg, vg = ctx.get_state()
    dx = xg - xr
    dx -= s.box[0] * np.round(dx / s.box[0])
    assert np.abs(dx).max() < 1e-5
    assert e.shape == (20, 1, 3)


def test_one_inner_step_equals_verlet_on_gpu():
    s = I.water_192(0)
    v0 = I.maxwell_boltzmann(s.mass, 300.0, 1)
    with _ctx(s) as a, _ctx(s, small=False) as b:
        a.set_state(s.x, v0)
        b.set_state(s.x, v0)
        a.respa_step(5, 1.0, 1)
        b.respa_step(5, 1.0, 1)
        xa, va = a.get_state()
        xb, vb = b.get_state()
    assert np.abs(xa - xb).max() < 1e-9 and np.abs(va - vb).max() < 1e-9


def test_checkpoint_resume_is_exact():
    s = I.water_192(0)
    v0 = I.maxwell_boltzmann(s.mass, 300.0, 1)
    with _ctx(s) as a:
        a.set_state(s.x, v0)
        a.respa_step(6, 3.0, 3)
        xm, vm = a.get_state()
        a.respa_step(6, 3.0, 3)
        x1, v1 = a.get_state()
    with _ctx(s) as b:
        b.set_state(xm, vm)
        b.respa_step(6, 3.0, 3)
        x2, v2 = b.get_state()
    np.testing.assert_array_equal(x1, x2)
    np.testing.assert_array_equal(v1, v2)


@pytest.mark.parametrize("name", ["water192", "water12288"])
def test_capacity_overflow_retry_gives_identical_results(name):
    """Row, pair-list and cell capacities far too small at the start: every
    overflow is detected on the device, the capacities grow and the work is
    redone, with results identical to a context that never overflowed."""
    s = SYSTEMS[name]()
    v0 = I.maxwell_boltzmann(s.mass, 300.0, 1)
    opts = '{"row_capacity": 4, "edge_capacity_factor": 0.05, "cell_capacity": 2}'
    with _ctx(s) as a, _ctx(s, options=opts) as b:
        a.set_state(s.x, v0)
        b.set_state(s.x, v0)
        Ea, Fa = a.forces(D.BIG)
        Eb, Fb = b.forces(D.BIG)
        np.testing.assert_array_equal(Fa, Fb)
        ea = a.respa_step(4, 3.0, 3)
        eb = b.respa_step(4, 3.0, 3)
        np.testing.assert_array_equal(ea, eb)
        np.testing.assert_array_equal(a.get_state()[0], b.get_state()[0])


def test_nonfinite_state_is_reported():
    s = I.water_192(0)
    v = I.maxwell_boltzmann(s.mass, 300.0, 1)
    v[5, 1] = np.nan
    with _ctx(s) as ctx:
        ctx.set_state(s.x, v)
        with pytest.raises(D.DmtsError) as ei:
            ctx.respa_step(1, 3.0, 3)
        assert ei.value.code == -5
        ctx.set_state(s.x, np.zeros_like(v))       # still usable
        ctx.respa_step(1, 3.0, 3)


def test_argument_errors():
    s = I.water_192(0)
    with _ctx(s) as ctx:
        with pytest.raises(D.DmtsError) as ei:
            ctx.respa_step(1, 3.0, 3)              # no state yet
        assert ei.value.code == -7
        ctx.set_state(s.x)
        for bad in ((1, -1.0, 3), (1, 3.0, 0), (-1, 3.0, 3)):
            with pytest.raises(D.DmtsError) as ei:
                ctx.respa_step(*bad)
            assert ei.value.code == -1
        with pytest.raises(D.DmtsError):
            ctx.forces(7)
    with _ctx(s, small=False) as ctx:
        ctx.set_state(s.x)
        with pytest.raises(D.DmtsError):
            ctx.respa_step(1, 3.0, 3)              # n_inner > 1 needs a small model
    small_box = I.System(x=s.x, species=s.species, mass=s.mass, atom_offset=s.atom_offset,
                         box=np.array([9.0]), n_species=2)
    with pytest.raises(D.DmtsError):
        _ctx(small_box)


def test_launch_count_grows():
    s = I.water_192(0)
    with _ctx(s) as ctx:
        ctx.set_state(s.x)
        n0 = ctx.launch_count
        ctx.respa_step(3, 3.0, 3)
        assert ctx.launch_count > n0 + 3 * 20


# ------------------------------------------------------------ BF16 tensor-core path

F_TOL_BF16 = 5e-3   # eV / A, RMSE


def _ctx_bf16(s, small=True):
    sa, sp, ba, bp = _models(s.n_species)
    if small:
        return D.Context(s, ba, bp, sa, sp, precision=D.BF16_MLP)
    return D.Context(s, ba, bp, precision=D.BF16_MLP)


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_atom_mlp_tensor_cores_match_fp32_kernels(name):
    """BF16 mode: the per-atom MLPs of the big model (F = 64) on the tensor
    cores, with operands split into two BF16 parts and FP32 accumulation,
    against the FP32 SIMT kernels, everything else identical. They differ
    only by the split-operand rounding, at most about 2^-17 relative per
    product, compounded over six stages and the edge backward: measured
    4e-6 eV/atom and 5e-5 eV/A on 192 waters, ten times below the BF16
    filter MLPs' own error; a wrong tile, transpose, bias or stage shows at
    the 1e-1 level. The molecules of two and three atoms average no rounding
    over many atoms (measured 1.7e-4 eV/A, virial 4e-4 of its largest entry),
    hence bounds of 5e-4 and 1e-3 relative."""
    s = SYSTEMS[name]()
    sa, sp, ba, bp = _models(s.n_species)
    out = []
    for tc in (1, 0):
        with D.Context(s, ba, bp, sa, sp, precision=D.BF16_MLP,
                       options=json.dumps({"atom_tensor_cores": tc})) as ctx:
            ctx.set_state(s.x)
            E, F = ctx.forces(D.BIG)
            _, _, W = ctx.forces(D.BIG, virial=True)
            out.append((np.asarray(E, dtype=np.float64), F, W))
    (E1, F1, W1), (E0, F0, W0) = out
    de = float(np.abs(E1 - E0).max() / s.n_atoms)
    err_f = _rmse(F1, F0)
    print(json.dumps({"system": name, "atom_tc_vs_fp32_dE_per_atom": de, "force_rmse": err_f}))
    assert de <= 2e-5
    assert err_f <= 5e-4 * max(1.0, float(np.sqrt(np.mean(F0 ** 2))))
    assert np.abs(W1 - W0).max() <= 1e-3 * max(1.0, np.abs(W0).max())


def test_bf16_other_radial_counts():
    """The BF16 kernels have the shipped radial-function counts (16 at F = 64,
    8 at F = 32) compiled in and take any other count at run time: K = 10
    and K = 12 against the oracle."""
    s = I.water_192(0)
    ba = I.Arch(cutoff=5.0, n_radial=10, n_layers=2, n_feat=64, n_species=2)
    sa = I.Arch(cutoff=3.5, n_radial=12, n_layers=1, n_feat=32, n_species=2)
    bp, sp = I.init_params(ba, 3), I.init_params(sa, 2)
    with D.Context(s, ba, bp, sa, sp, precision=D.BF16_MLP) as ctx:
        ctx.set_state(s.x)
        for which, arch, par in ((D.SMALL, sa, sp), (D.BIG, ba, bp)):
            E, F = ctx.forces(which)
            Er, Fr = M.energy_forces(M.spec_of(arch), par, s.x, s.species, s.atom_offset, s.box)
            de, err_f = float(np.abs(E - Er).sum() / s.n_atoms), _rmse(F, Fr)
            print(json.dumps({"model": "small" if which == 0 else "big", "K": arch.n_radial,
                              "dE_per_atom": de, "force_rmse": err_f}))
            assert de <= 5e-3 and err_f <= F_TOL_BF16


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_energy_forces_bf16(name):
    """Filter MLPs on tensor cores with BF16 operands and FP32 accumulation."""
    s = SYSTEMS[name]()
    sa, sp, ba, bp = _models(s.n_species)
    with _ctx_bf16(s) as ctx:
        ctx.set_state(s.x)
        for which, arch, par in ((D.SMALL, sa, sp), (D.BIG, ba, bp)):
            E, F = ctx.forces(which)
            Er, Fr = M.energy_forces(M.spec_of(arch), par, s.x, s.species, s.atom_offset, s.box)
            err_f = _rmse(F, Fr)
            de = float(np.abs(E - Er).sum() / s.n_atoms)
            print(json.dumps({"system": name, "model": "small" if which == 0 else "big", "precision": "bf16",
                              "dE_per_atom": de, "force_rmse": err_f,
                              "force_rms": float(np.sqrt(np.mean(Fr ** 2)))}))
            assert err_f <= F_TOL_BF16
            # energies: BF16 operands carry ~2^-9 relative rounding per product
            assert de <= 5e-3


@pytest.mark.parametrize("name", ["water192", "water12288"])
@pytest.mark.parametrize("prec", [D.FP32, D.BF16_MLP])
def test_energy_forces_network_only(name, prec):
    """The same comparisons with the pair repulsion switched off (rep_a = 0):
    the forces are then the networks' alone (RMS about 0.17 eV/A on water,
    against 0.84 with the repulsion), so the error of the MLP path is
    measured undiluted. Absolute bounds as above, and relative to the
    network force: FP32 1e-4, BF16 3e-2 of its RMS."""
    import dataclasses
    s = SYSTEMS[name]()
    sa = dataclasses.replace(I.small_arch(s.n_species), rep_a=0.0)
    ba = dataclasses.replace(I.big_arch(s.n_species), rep_a=0.0)
    sp, bp = I.init_params(sa, 2), I.init_params(ba, 3)
    with D.Context(s, ba, bp, sa, sp, precision=prec) as ctx:
        ctx.set_state(s.x)
        for which, arch, par in ((D.SMALL, sa, sp), (D.BIG, ba, bp)):
            E, F = ctx.forces(which)
            Er, Fr = M.energy_forces(M.spec_of(arch), par, s.x, s.species, s.atom_offset, s.box)
            de, err_f = float(np.abs(E - Er).sum() / s.n_atoms), _rmse(F, Fr)
            rms = float(np.sqrt(np.mean(Fr ** 2)))
            print(json.dumps({"system": name, "precision": int(prec), "model": int(which), "rep_a": 0.0,
                              "dE_per_atom": de, "force_rmse": err_f, "force_rms": rms,
                              "rel_force_rmse": err_f / rms}))
            if prec == D.FP32:
                assert de <= E_TOL and err_f <= F_TOL and err_f <= 1e-4 * rms
            else:
                assert de <= 5e-3 and err_f <= F_TOL_BF16 and err_f <= 3e-2 * rms


@pytest.mark.parametrize("prec", [D.FP32, D.BF16_MLP])
def test_every_tuning_candidate_gives_identical_forces(prec):
    """The autotuner's candidates (persistent CTAs per SM and one or two
    tiles in flight per backward CTA for the tensor-core kernels, atoms per
    CTA for the FP32 kernels) change only how the same fixed work is spread
    over the GPU: forces and energies are bit-identical for every choice, on
    a system large enough for every grid to differ."""
    s = I.water_12288(0)
    cands = [(k, t) for t in (1, 2) for k in (1, 2, 3, 4, 5, 6)] if prec == D.BF16_MLP else \
        [(k, 0) for k in (8, 16, 24, 32, 48)]
    ref = None
    with _ctx_bf16(s) if prec == D.BF16_MLP else _ctx(s) as ctx:
        ctx.set_state(s.x)
        for k, t in cands:
            out = []
            for which in (D.SMALL, D.BIG):
                ctx.set_tuning(which, k, k, t)
                if t:
                    assert ctx.tuning(which)["bwd_tiles"] == t
                E, F = ctx.forces(which)
                out.append((E, F))
            if ref is None:
                ref = out
                continue
            for (E, F), (E0, F0) in zip(out, ref):
                np.testing.assert_array_equal(E, E0)
                np.testing.assert_array_equal(F, F0)


def test_bf16_virial_and_dynamics():
    s = I.water_192(0)
    sa, sp, ba, bp = _models(2)
    v0 = I.maxwell_boltzmann(s.mass, 300.0, 1)
    with _ctx_bf16(s) as ctx:
        ctx.set_state(s.x, v0)
        _, _, W = ctx.forces(D.BIG, virial=True)
        Wr = M.virial(M.spec_of(ba), bp, s.x, s.species, s.atom_offset, s.box)
        assert np.abs(W - Wr).max() <= 2e-2 * max(1.0, np.abs(Wr).max())
        e = ctx.respa_step(40, 3.0, 3)
        span = float(e[:, 0, 2].max() - e[:, 0, 2].min())
        print(json.dumps({"bf16_etot_span_120fs": span}))
        assert np.all(np.isfinite(e)) and span < 5.0


# ------------------------------------------------------------ distillation gradient (double backward)

def _fm_frames(s, ba, bp, n_frames=2, seed=7):
    """Frames: the structure and a copy displaced by 0.03 A per component;
    reference forces from the big model (FP64 oracle)."""
    rng = np.random.default_rng(seed)
    frames = np.stack([s.x] + [s.x + rng.normal(scale=0.03, size=s.x.shape) for _ in range(n_frames - 1)])
    frames = frames - s.box[0] * np.floor(frames / s.box[0])
    f_ref = np.stack([M.energy_forces(M.spec_of(ba), bp, f, s.species, s.atom_offset, s.box)[1] for f in frames])
    return frames, f_ref


@pytest.mark.parametrize("name,rel", [("water192", 1e-6), ("water12288", 1e-5)])
def test_force_matching_gradient_matches_oracle(name, rel):
    """dL/dtheta of the force-matching loss through the forces, by the
    library's FP32 adjoint kernels, against the FP64 oracle (autograd double
    backward) on two frames, entry by entry:
    |g - g_ref| <= rel * max|g_ref| + 1e-9. Each entry is a fixed-order FP32
    sum over all pairs of all frames, so its rounding error grows like the
    square root of the term count: measured 2.6e-7 of max|g_ref| on 192 atoms;
    64 times the terms on 12,288 atoms allow 8 times that, hence 1e-5 there.
    A wrong entry (a dropped term, a transposed weight gradient) is off by
    the size of the entry itself, far above either bound."""
    s = SYSTEMS[name]()
    sa, sp, ba, bp = _models(2)
    frames, f_ref = _fm_frames(s, ba, bp)
    L_ref, g_ref = M.force_matching_grad(M.spec_of(sa), sp, frames, s.species, s.atom_offset, s.box, f_ref)
    with _ctx(s) as ctx:
        ctx.set_state(s.x)
        L, g = ctx.force_matching_grad(frames, f_ref)
    rel_L = abs(L - L_ref) / L_ref
    err = np.abs(g - g_ref)
    bound = rel * np.abs(g_ref).max() + 1e-9
    print(json.dumps({"system": name, "loss": L, "loss_ref": L_ref, "rel_loss_err": rel_L,
                      "grad_max_abs_err": float(err.max()), "grad_max_abs": float(np.abs(g_ref).max()),
                      "bound": float(bound), "worst_entry": int(err.argmax())}))
    assert rel_L < 1e-5
    assert np.all(err <= bound), (int(err.argmax()), float(err.max()), float(bound))
    assert np.all(g[-(1 + s.n_species):] == 0.0)          # d2 and e0 do not move forces


def test_force_matching_autograd_function():
    """ForceMatchingLoss (a torch.autograd.Function around the library call)
    returns the oracle's loss and, through backward, the oracle's gradient
    scaled by the incoming gradient."""
    torch = pytest.importorskip("torch")
    s = I.water_192(0)
    sa, sp, ba, bp = _models(2)
    frames, f_ref = _fm_frames(s, ba, bp, n_frames=1)
    L_ref, g_ref = M.force_matching_grad(M.spec_of(sa), sp, frames, s.species, s.atom_offset, s.box, f_ref)
    with _ctx(s) as ctx:
        ctx.set_state(s.x)
        theta = torch.tensor(sp, requires_grad=True)
        loss = D.ForceMatchingLoss.apply(theta, ctx, frames, f_ref)
        (2.5 * loss).backward()
    assert abs(float(loss.detach()) - L_ref) <= 1e-5 * L_ref
    err = np.abs(theta.grad.numpy() - 2.5 * g_ref)
    assert np.all(err <= 2.5 * (1e-6 * np.abs(g_ref).max() + 1e-9)), float(err.max())


# ------------------------------------------------------------ solvated polymer (4 species)

@pytest.mark.parametrize("prec", [D.FP32, D.BF16_MLP])
def test_polymer6000_energy_forces(prec):
    pytest.importorskip("scipy")
    s = I.make_solvated_polymer(n_heavy=300, n_total=6000, seed=1)
    sa, sp, ba, bp = _models(4)
    with D.Context(s, ba, bp, sa, sp, precision=prec) as ctx:
        ctx.set_state(s.x)
        for which, arch, par in ((D.SMALL, sa, sp), (D.BIG, ba, bp)):
            gi, gj = _pairs(*ctx.neighbors(which))
            oi, oj = M.pair_list(s.x, s.atom_offset, s.box, arch.cutoff)
            np.testing.assert_array_equal(gi, oi)
            np.testing.assert_array_equal(gj, oj)
            E, F = ctx.forces(which)
            Er, Fr = M.energy_forces(M.spec_of(arch), par, s.x, s.species, s.atom_offset, s.box, (oi, oj))
            de, err = float(abs(E[0] - Er[0]) / s.n_atoms), _rmse(F, Fr)
            print(json.dumps({"system": "polymer6000", "precision": int(prec), "model": int(which),
                              "dE_per_atom": de, "force_rmse": err}))
            if prec == D.FP32:
                assert de <= E_TOL and err <= F_TOL
            else:
                assert de <= 5e-3 and err <= F_TOL_BF16


@pytest.mark.parametrize("prec", [D.FP32, D.BF16_MLP])
def test_polymer100k_sampled_rows_and_invariants(prec):
    """~100k atoms: too many for the O(N^2) oracle, so sampled neighbour rows
    are compared bit-exactly with the oracle's row, and forces and energies
    are checked against properties that hold at any size."""
    pytest.importorskip("scipy")
    s = I.make_solvated_polymer()
    sa, sp, ba, bp = _models(4)
    rng = np.random.default_rng(0)
    sample = np.concatenate([[0, 1, 2999, 3000, s.n_atoms - 1], rng.choice(s.n_atoms, 40, replace=False)])
    with D.Context(s, ba, bp, sa, sp, precision=prec) as ctx:
        ctx.set_state(s.x)
        for which, arch in ((D.SMALL, sa), (D.BIG, ba)):
            rp, col = ctx.neighbors(which)
            for i in sample:
                np.testing.assert_array_equal(col[rp[i]:rp[i + 1]], M.pair_row(s.x, int(i), s.atom_offset, s.box, arch.cutoff))
        E0, F0 = ctx.forces(D.BIG)
        rms = float(np.sqrt(np.mean(F0 ** 2)))
        net = np.abs(F0.sum(axis=0)).max()
        shift = np.array([3.3, -1.7, 2.2])
        xs = s.x + shift
        xs -= s.box[0] * np.floor(xs / s.box[0])
        ctx.set_state(xs)
        E1, F1 = ctx.forces(D.BIG)
        print(json.dumps({"system": "polymer100k", "precision": int(prec), "n_atoms": s.n_atoms,
                          "net_force_rel": float(net / (s.n_atoms * rms)), "dE_shift_per_atom": float(abs(E1[0] - E0[0]) / s.n_atoms),
                          "force_rmse_shift": _rmse(F1, F0)}))
        assert net <= (1e-5 if prec == D.FP32 else 1e-3) * s.n_atoms * rms
        assert abs(E1[0] - E0[0]) / s.n_atoms <= (E_TOL if prec == D.FP32 else 5e-4)
        assert _rmse(F1, F0) <= (F_TOL if prec == D.FP32 else F_TOL_BF16)
        e = ctx.respa_step(3, 3.0, 3)
        assert np.all(np.isfinite(e))


# ------------------------------------------------------------ periodic replicas in one context

def test_periodic_replicas_match_oracle_and_single_boxes():
    """Four 192-atom water boxes (different orientations) as periodic
    replicas of one context: bit-exact pair sets, per-replica energies and
    forces against the oracle (FP32 and BF16 bounds), and an Algorithm 1
    trajectory of the batch equal, replica by replica, to the trajectory of
    each box in its own context (FP32 sums every row in edge order, so the
    batching changes no bit)."""
    boxes = [I.water_192(k) for k in range(4)]
    s = I.replicas(boxes)
    assert s.n_systems == 4 and s.n_atoms == 768
    sa, sp, ba, bp = _models(2)
    v0 = [I.maxwell_boltzmann(b.mass, 300.0, 1 + k) for k, b in enumerate(boxes)]
    for prec, f_tol in ((D.FP32, F_TOL), (D.BF16_MLP, F_TOL_BF16)):
        with D.Context(s, ba, bp, sa, sp, precision=prec) as ctx:
            ctx.set_state(s.x)
            for which, arch, par in ((D.SMALL, sa, sp), (D.BIG, ba, bp)):
                gi, gj = _pairs(*ctx.neighbors(which))
                oi, oj = M.pair_list(s.x, s.atom_offset, s.box, arch.cutoff)
                np.testing.assert_array_equal(gi, oi)
                np.testing.assert_array_equal(gj, oj)
                E, F = ctx.forces(which)
                Er, Fr = M.energy_forces(M.spec_of(arch), par, s.x, s.species, s.atom_offset, s.box, (oi, oj))
                assert E.shape == (4,)
                de = float(np.abs(E - Er).max() / 192)
                print(json.dumps({"replicas": 4, "precision": int(prec), "model": int(which), "dE_per_atom": de,
                                  "force_rmse": _rmse(F, Fr)}))
                assert de <= (E_TOL if prec == D.FP32 else 5e-3) and _rmse(F, Fr) <= f_tol
    with D.Context(s, ba, bp, sa, sp) as ctx:
        ctx.set_state(s.x, np.concatenate(v0))
        ctx.respa_step(5, 3.0, 3)
        xb, vb = ctx.get_state()
    for k, b in enumerate(boxes):
        with _ctx(b) as one:
            one.set_state(b.x, v0[k])
            one.respa_step(5, 3.0, 3)
            x1, v1 = one.get_state()
        np.testing.assert_array_equal(xb[192 * k:192 * (k + 1)], x1)
        np.testing.assert_array_equal(vb[192 * k:192 * (k + 1)], v1)


def test_periodic_replicas_must_share_a_box():
    a, b = I.water_192(0), I.make_water(4, 12.5, 1)
    with pytest.raises(D.DmtsError) as ei:
        _ctx(I.replicas([a, b]))
    assert ei.value.code == -1
