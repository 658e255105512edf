"""GPU checks of the library's diagnostics and of cached-force continuity.

* The device's Philox-4x32-10 (the thermostat's noise generator) against the
  generator's published known-answer vectors, word for word.
* The bounded completion wait of the tensor-core kernels, exercised by a
  self-test kernel that issues no MMA: a wait nothing arrives at gives up,
  the call reports DMTS_ERR_TIMEOUT, and the same context then evaluates
  forces identical to those it gave before.
* dmts_set_state keeps the cached forces when the positions are unchanged
  (Algorithm 1's first step is a restart at new positions only), and
  recomputes them when a position changed.
* dmts_time_stages reads 0 for the stages that launch nothing.
"""
import os
import sys

import numpy as np
import pytest

from paper_2510_06562_gb300 import dmts as D
from paper_2510_06562_gb300 import inputs as I

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from test_oracle_langevin import load_philox_kat  # noqa: E402

pytestmark = pytest.mark.gpu


def _ctx(s, precision=D.FP32, options=None):
    sa, sp = I.small_arch(s.n_species), I.init_params(I.small_arch(s.n_species), 2)
    ba, bp = I.big_arch(s.n_species), I.init_params(I.big_arch(s.n_species), 3)
    return D.Context(s, ba, bp, sa, sp, precision=precision, options=options)


def test_device_philox_known_answer_vectors():
    ctr, key, out = load_philox_kat()
    for c, k, o in zip(ctr, key, out):
        got = D.philox4x32_10(c[None, :].astype(np.uint32), k.astype(np.uint32))
        np.testing.assert_array_equal(got[0].astype(np.uint64), o)


def test_device_philox_matches_oracle_on_many_counters():
    from oracle import integrate as G
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    key = np.array([0x12345678, 0x9ABCDEF0], dtype=np.uint32)
    np.testing.assert_array_equal(D.philox4x32_10(ctr, key), G.philox4x32_10(ctr, key))


@pytest.mark.parametrize("precision", [D.FP32, D.BF16_MLP])
def test_wait_timeout_is_reported_and_context_stays_usable(precision):
    s = I.water_192(0)
    with _ctx(s, precision) as ctx:
        ctx.set_state(s.x)
        E0, F0 = ctx.forces(D.BIG)
        assert ctx.wait_selftest(True, 1000) == 0          # an arrival completes the wait
        code = ctx.wait_selftest(False, 2000)              # nothing arrives: the wait gives up
        assert code == -6
        assert b"gave up" in D.load_library().dmts_last_error()
        assert ctx.wait_selftest(True, 1000) == 0          # the flag was cleared
        E1, F1 = ctx.forces(D.BIG)
        np.testing.assert_array_equal(E1, E0)
        np.testing.assert_array_equal(F1, F0)
        e = ctx.respa_step(2, 3.0, 3)
        assert np.all(np.isfinite(e))


def test_set_state_with_unchanged_positions_keeps_cached_forces():
    """A caller that reads the state back and uploads it again every step
    pays no extra force evaluation, and its trajectory is the uninterrupted
    one bit for bit; a changed position recomputes both models' forces."""
    s = I.water_192(0)
    v0 = I.maxwell_boltzmann(s.mass, 300.0, 1)
    with _ctx(s, D.BF16_MLP) as a, _ctx(s, D.BF16_MLP) as b:
        a.set_state(s.x, v0)
        b.set_state(s.x, v0)
        a.respa_step(3, 3.0, 3)
        b.respa_step(2, 3.0, 3)
        n0 = b.launch_count
        b.respa_step(1, 3.0, 3)
        per_step = b.launch_count - n0                    # both contexts have taken 3 steps
        for _ in range(3):
            x, v = a.get_state()
            a.set_state(x, v)
            n0 = a.launch_count
            a.respa_step(1, 3.0, 3)
            assert a.launch_count - n0 == per_step          # no first-step evaluation
            b.respa_step(1, 3.0, 3)
        xa, va = a.get_state()
        xb, vb = b.get_state()
        np.testing.assert_array_equal(xa, xb)
        np.testing.assert_array_equal(va, vb)
        # velocities alone changed: forces still valid
        a.set_state(xa, -va)
        n0 = a.launch_count
        a.respa_step(1, 3.0, 3)
        assert a.launch_count - n0 == per_step
        # one position changed: both models are evaluated first
        x, v = a.get_state()
        x[7, 1] = np.nextafter(x[7, 1], np.inf)
        a.set_state(x, v)
        n0 = a.launch_count
        a.respa_step(1, 3.0, 3)
        assert a.launch_count - n0 > per_step


@pytest.mark.parametrize("precision", [D.FP32, D.BF16_MLP])
def test_stage_timing_reads_zero_for_stages_without_work(precision):
    """dmts_time_stages: the species embedding (built at parameter upload)
    and the layer-0 per-atom adjoint launch nothing and read 0; every other
    stage of both models is timed (> 0)."""
    s = I.water_192(0)
    with _ctx(s, precision) as ctx:
        ctx.set_state(s.x)
        for which in (D.SMALL, D.BIG):
            st = ctx.time_stages(which, reps=2)
            assert st["embed"] == 0.0 and st["atom_bwd_l0"] == 0.0
            others = {k: v for k, v in st.items() if k not in ("embed", "atom_bwd_l0")}
            assert all(v > 0.0 for v in others.values()), others
