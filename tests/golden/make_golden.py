"""Writes the stored oracle values under tests/golden/ (calls only oracle/
and the seeded input generators). The paper prints no worked example of the
potential or of Algorithm 1, so these files are regression records of the
oracle itself, not values quoted from the paper.

Run from the repository root: python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import model as M  # noqa: E402
from paper_2510_06562_gb300 import inputs as I  # noqa: E402


def main():
    s = I.water_192(0)
    out = {"system": "water192 seed 0 (64 rigid waters, L = 12.42 A)", "models": {}}
    for name, arch, seed in (("big", I.big_arch(), 3), ("small", I.small_arch(), 2)):
        spec = M.spec_of(arch)
        par = I.init_params(arch, seed)
        i, j = M.pair_list(s.x, s.atom_offset, s.box, arch.cutoff)
        E, F = M.energy_forces(spec, par, s.x, s.species, s.atom_offset, s.box, (i, j))
        out["models"][name] = {
            "param_seed": seed, "n_pairs": int(len(i)), "energy": float(E[0]),
            "forces_first4": F[:4].tolist(), "force_rms": float(np.sqrt((F ** 2).mean())),
        }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "water192_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
