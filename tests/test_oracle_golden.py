"""The oracle still reproduces its stored regression record (CPU only)."""
import json
import os

import numpy as np

from oracle import model as M
from paper_2510_06562_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


def test_water192_record():
    with open(os.path.join(HERE, "golden", "water192_oracle.json")) as f:
        rec = json.load(f)
    s = I.water_192(0)
    for name, arch in (("big", I.big_arch()), ("small", I.small_arch())):
        r = rec["models"][name]
        par = I.init_params(arch, r["param_seed"])
        i, j = M.pair_list(s.x, s.atom_offset, s.box, arch.cutoff)
        assert len(i) == r["n_pairs"]
        E, F = M.energy_forces(M.spec_of(arch), par, s.x, s.species, s.atom_offset, s.box, (i, j))
        assert abs(E[0] - r["energy"]) <= 1e-12 * abs(r["energy"])
        np.testing.assert_allclose(F[:4], np.array(r["forces_first4"]), atol=1e-12)
