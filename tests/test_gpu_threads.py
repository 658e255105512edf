"""Two contexts driven from two host threads at once, on one device.

The launch set-up of every kernel (its shared-memory limit, the persistent
grid's CTAs per SM) is process state taken once per kernel and device under
a lock; the contexts themselves share nothing. Each thread creates its own
context, so the first launches of the kernels race. The results must equal
those of the same runs made one after the other (the tuner is off, so both
runs use the same work granularity).
"""
import threading

import numpy as np
import pytest

from paper_2510_06562_gb300 import dmts as D
from paper_2510_06562_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _run(prec):
    s = I.water_192(0)
    sa, ba = I.small_arch(s.n_species), I.big_arch(s.n_species)
    v0 = I.maxwell_boltzmann(s.mass, 300.0, 1)
    with D.Context(s, ba, I.init_params(ba, 3), sa, I.init_params(sa, 2), precision=prec,
                   options='{"autotune": 0}') as ctx:
        ctx.set_state(s.x, v0)
        e = ctx.respa_step(10, 3.0, 3)
        _, f = ctx.forces(D.BIG)
        x, v = ctx.get_state()
    return e, f, x, v


def test_two_threads_two_contexts_match_serial_runs():
    precs = (D.BF16_MLP, D.FP32, D.BF16_MLP)
    serial = [_run(p) for p in precs]
    got = [None] * len(precs)
    errors = []

    def work(k):
        try:
            got[k] = _run(precs[k])
        except Exception as exc:          # reported by the main thread
            errors.append(exc)

    threads = [threading.Thread(target=work, args=(k,)) for k in range(len(precs))]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not any(t.is_alive() for t in threads)
    assert not errors, errors
    for ref, out in zip(serial, got):
        for a, b in zip(ref, out):
            np.testing.assert_allclose(b, a, rtol=1e-9, atol=1e-9)
