"""The bounds-checked build (libdmts_check.so, compiled with -DDMTS_CHECK).

Its kernels test every pair, row and cell index they gather with against the
array it indexes; an index outside records the source line and the call
fails. The main paths run through it here in a child process (the library is
chosen by DMTS_LIBRARY): pair lists, forces in both precisions, RESPA steps,
the distillation gradient and periodic replicas, on systems from two atoms
to 12,288. Every call must succeed, and the energies equal those of the
ordinary build (the checks change no arithmetic).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2510_06562_gb300 import build as B

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + "/tests")
from paper_2510_06562_gb300 import dmts as D, inputs as I
from test_gpu_parity import _tiny_molecules
out = {"library": D.LIB_PATH}
systems = {"tiny3": _tiny_molecules(), "vacuum64": I.make_vacuum_batch(64, 10, 60, seed=0),
           "water192": I.water_192(0), "water12288": I.water_12288(0),
           "replicas4": I.replicas([I.water_192(k) for k in range(4)])}
for name, s in systems.items():
    sa, ba = I.small_arch(s.n_species), I.big_arch(s.n_species)
    sp, bp = I.init_params(sa, 2), I.init_params(ba, 3)
    for prec in (D.FP32, D.BF16_MLP):
        with D.Context(s, ba, bp, sa, sp, precision=prec) as ctx:
            ctx.set_state(s.x, I.maxwell_boltzmann(s.mass, 300.0, 1, s.atom_offset))
            for which in (D.SMALL, D.BIG):
                ctx.neighbors(which)
                E, F = ctx.forces(which)
                out[f"{name}/{prec}/{which}"] = [float(e) for e in E]
            e = ctx.respa_step(3, 3.0, 3)
            out[f"{name}/{prec}/respa"] = float(e[-1, :, 2].sum())
            if name == "water192" and prec == D.FP32:
                frames = s.x[None].copy()
                L, g = ctx.distill_grad(frames, F[None], np.array([float(np.sum(E))]), 1.0)
                out["distill_loss"] = L
print(json.dumps(out))
"""


def _run(lib):
    env = dict(os.environ, DMTS_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], capture_output=True, text=True,
                       env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_runs_every_path_without_an_index_violation():
    lib_check = B.build(check=True)
    lib = B.build()
    got = _run(lib_check)
    ref = _run(lib)
    assert got["library"].endswith("libdmts_check.so") and ref["library"].endswith("libdmts.so")
    for k, v in ref.items():
        if k == "library":
            continue
        np.testing.assert_allclose(np.asarray(got[k]), np.asarray(v), rtol=1e-6, atol=1e-9, err_msg=k)
