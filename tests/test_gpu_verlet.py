"""Verlet-skin neighbour lists on the GPU (needs a GB300).

Candidate rows of all j within rc + skin are kept from the last rebuild and
filtered with the exact cutoff test at every evaluation. While no atom has
moved by skin / 2 since the rebuild, that must give exactly the oracle's
FP64 pair set; once one has, both models' rows are rebuilt. The pair set is
the same as a fresh build at every evaluation, so forces and whole RESPA
trajectories must be bit-identical to running with skin 0 (fresh build at
every evaluation).
"""
import json

import numpy as np
import pytest

from oracle import model as M
from paper_2510_06562_gb300 import dmts as D
from paper_2510_06562_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SKIN = 1.0


def _ctx(s, skin, precision=D.FP32, extra=None):
    sa, ba = I.small_arch(s.n_species), I.big_arch(s.n_species)
    opts = {"skin": skin, "autotune": 0}
    opts.update(extra or {})
    return D.Context(s, ba, I.init_params(ba, 3), sa, I.init_params(sa, 2), precision=precision,
                     options=json.dumps(opts))


def _check_pairs(ctx, s, x):
    for which, arch in ((D.SMALL, I.small_arch(s.n_species)), (D.BIG, I.big_arch(s.n_species))):
        row_ptr, col = ctx.neighbors(which)
        gi = np.repeat(np.arange(len(row_ptr) - 1), np.diff(row_ptr))
        oi, oj = M.pair_list(x, s.atom_offset, s.box, arch.cutoff)
        assert len(gi) == len(oi), (which, len(gi), len(oi))
        np.testing.assert_array_equal(gi, oi)
        np.testing.assert_array_equal(col.astype(np.int64), oj)


def _displace(x, max_len, seed):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=x.shape)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return x + d * rng.uniform(0.0, max_len, size=(len(x), 1))


SYSTEMS = {
    "water192": lambda: I.water_192(0),
    "water12288": lambda: I.water_12288(0),
    "vacuum64": lambda: I.make_vacuum_batch(64, 10, 60, seed=0),
}


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_filtered_candidates_equal_oracle_pairs(name):
    s = SYSTEMS[name]()
    with _ctx(s, SKIN) as ctx:
        ctx.set_state(s.x)
        _check_pairs(ctx, s, ctx.get_state()[0])
        checks0, rebuilds0 = ctx.neighbor_stats()
        assert rebuilds0 == 1 and checks0 >= 2       # the first check rebuilds, the later ones find nothing moved
        # every atom moves by less than skin / 2: the rows are filtered, not rebuilt
        ctx.set_state(_displace(s.x, 0.49 * SKIN, seed=5))
        _check_pairs(ctx, s, ctx.get_state()[0])
        checks1, rebuilds1 = ctx.neighbor_stats()
        assert checks1 > checks0 and rebuilds1 == 1
        # one atom moves by more than skin / 2: rebuilt once, at the first check
        x2 = _displace(s.x, 0.49 * SKIN, seed=5)
        x2[7] += np.array([0.8, -0.7, 0.6]) * SKIN     # 1.22 skin: beyond skin / 2 whatever the first move
        ctx.set_state(x2)
        _check_pairs(ctx, s, ctx.get_state()[0])
        checks2, rebuilds2 = ctx.neighbor_stats()
        assert checks2 > checks1 and rebuilds2 == 2


def test_row_capacity_overflow_of_candidate_rows_recovers():
    s = I.water_192(0)
    with _ctx(s, SKIN, extra={"row_capacity": 8}) as ctx:
        ctx.set_state(s.x)
        _check_pairs(ctx, s, ctx.get_state()[0])


@pytest.mark.parametrize("precision", [D.FP32, D.BF16_MLP])
def test_trajectory_bit_identical_to_fresh_builds(precision):
    s = I.water_12288(0)
    v0 = I.maxwell_boltzmann(s.mass, 300.0, seed=1, atom_offset=s.atom_offset)
    out = []
    for skin in (0.0, SKIN):
        with _ctx(s, skin, precision) as ctx:
            ctx.set_state(s.x, v0)
            e = ctx.respa_step(12, 3.0, 3)
            x, v = ctx.get_state()
            _, f = ctx.forces(D.BIG)
            out.append((x, v, f, e, ctx.neighbor_stats()))
    (x0, v0_, f0, e0, st0), (x1, v1, f1, e1, st1) = out
    assert st0 == (0, 0)
    checks, rebuilds = st1
    assert checks >= 12 * 3 and 1 <= rebuilds < checks
    np.testing.assert_array_equal(x0, x1)
    np.testing.assert_array_equal(v0_, v1)
    np.testing.assert_array_equal(f0, f1)
    np.testing.assert_array_equal(e0, e1)
