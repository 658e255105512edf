"""The seeded workload generators produce what their docstrings state (CPU)."""
import numpy as np
import pytest

from paper_2510_06562_gb300 import inputs as I


def test_water_boxes():
    for s, L in ((I.water_192(0), 12.42), (I.water_12288(0), 49.7)):
        n_mol = s.n_atoms // 3
        assert s.box[0] == L and np.all(s.x >= 0) and np.all(s.x < L)
        dens = s.mass.sum() * 1.66053906660 / L ** 3
        assert abs(dens - 0.998) < 0.003
        x = s.x.reshape(n_mol, 3, 3)
        d = x[:, 1:, :] - x[:, :1, :]
        d -= L * np.round(d / L)
        np.testing.assert_allclose(np.linalg.norm(d, axis=2), 0.96, atol=1e-12)
        cosang = (d[:, 0] * d[:, 1]).sum(1) / 0.96 ** 2
        np.testing.assert_allclose(np.degrees(np.arccos(cosang)), 104.5, atol=1e-9)


def test_vacuum_batch():
    b = I.make_vacuum_batch(20, 10, 60, seed=3)
    sizes = np.diff(b.atom_offset)
    assert b.n_systems == 20 and np.all((sizes >= 10) & (sizes <= 60)) and np.all(b.box == 0)
    for s in range(20):
        p = b.x[b.atom_offset[s]:b.atom_offset[s + 1]]
        bonds = np.linalg.norm(np.diff(p, axis=0), axis=1)
        assert np.all((bonds >= 1.1 - 1e-12) & (bonds <= 1.5 + 1e-12))
        dd = np.linalg.norm(p[:, None] - p[None], axis=2) + np.eye(len(p)) * 9
        assert dd.min() >= 1.0 - 1e-12


def test_solvated_polymer():
    pytest.importorskip("scipy")
    from scipy.spatial import cKDTree
    s = I.make_solvated_polymer(n_heavy=300, n_total=6000, seed=1)
    L = s.box[0]
    assert abs(s.n_atoms - 6000) <= 3
    assert abs(s.mass.sum() * 1.66053906660 / L ** 3 - 1.0) < 1e-9
    heavy = s.species[:300]
    assert (heavy == 1).sum() == 180 and (heavy == 2).sum() == 60 and (heavy == 3).sum() == 60
    # chain bonds of 1.5 A
    d = np.diff(s.x[:300], axis=0)
    d -= L * np.round(d / L)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.5, atol=1e-9)
    # hydrogens fill valences: C 4, N 3, O 2 minus chain bonds
    n_h_poly = int((s.species[300:] == 0).sum()) - 2 * int((s.species[300:] == 3).sum())
    val = np.array([0, 4, 3, 2])[heavy] - np.r_[1, np.full(298, 2), 1]
    assert n_h_poly == np.maximum(val, 0).sum()
    tr = cKDTree(s.x, boxsize=L)
    dist, _ = tr.query(s.x, k=2)
    assert dist[:, 1].min() >= 0.95
