"""The Python binding's argument marshalling, on the CPU with a stand-in for
the library: every buffer the library reads or writes is checked for type,
contiguity and size before its address is passed (the library trusts the
sizes it is given)."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2510_06562_gb300 import dmts as D

N, NS, NP = 5, 1, 11


class _FakeLib:
    """Records each call's arguments and returns DMTS_OK."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def call(*args):
            self.calls.append((name, args))
            if name == "dmts_set_state":            # what the library would copy, read during the call
                p = C.cast(args[1], C.POINTER(C.c_double))
                self.x_seen = [p[i] for i in range(3 * args[3])]
            return D.DMTS_OK
        return call


@pytest.fixture
def ctx(monkeypatch):
    lib = _FakeLib()
    monkeypatch.setattr(D, "load_library", lambda *a: lib)
    c = object.__new__(D.Context)
    c._keep, c._h = [], C.c_void_p(1)
    c.n_atoms, c.n_systems, c.small_n_params, c.has_small = N, NS, NP, True
    c.lib = lib
    yield c
    c._h = None                     # never handed to the real library


def _last(c, name):
    calls = [a for n, a in c.lib.calls if n == name]
    assert calls, name
    return calls[-1]


def test_inputs_are_converted_and_sized(ctx):
    x = np.arange(3 * N, dtype=np.float32).reshape(N, 3)
    ctx.set_state(x)                                    # NumPy data is converted to float64
    args = _last(ctx, "dmts_set_state")
    assert args[2] is None and args[3] == N
    assert ctx.lib.x_seen == list(range(3 * N))
    ctx.set_state(np.zeros(3 * N), np.ones((N, 3)))     # any shape with 3N values
    with pytest.raises(ValueError):
        ctx.set_state(np.zeros((N - 1, 3)))
    with pytest.raises(ValueError):
        ctx.set_state(np.zeros((N, 3)), np.zeros((N + 1, 3)))
    with pytest.raises(ValueError):
        ctx.set_state(None)
    with pytest.raises(TypeError):
        ctx.set_state(torch.zeros(N, 3, dtype=torch.float32))
    t = torch.zeros(N, 3, dtype=torch.float64)
    ctx.set_state(t)
    assert _last(ctx, "dmts_set_state")[1] == t.data_ptr()


def test_output_buffers_must_match_exactly(ctx):
    xo, vo = np.empty((N, 3)), np.empty((N, 3))
    ctx.get_state(xo, vo)
    args = _last(ctx, "dmts_get_state")
    assert args[1] == xo.ctypes.data and args[2] == vo.ctypes.data
    for bad, err in ((np.empty((N, 3), np.float32), TypeError),
                     (np.empty((N, 6))[:, :3], TypeError),        # not contiguous
                     (np.empty((N - 1, 3)), ValueError),
                     (torch.empty(N, 3, dtype=torch.float32), TypeError),
                     ([0.0] * (3 * N), TypeError)):
        with pytest.raises(err):
            ctx.get_state(bad, vo)
    ro = np.empty((N, 3))
    ro.flags.writeable = False
    with pytest.raises(TypeError):
        ctx.get_state(ro, vo)
    t = torch.empty(N, 3, dtype=torch.float64)
    ctx.get_state(t, vo)
    assert _last(ctx, "dmts_get_state")[1] == t.data_ptr()


def test_forces_outputs(ctx):
    f, e = np.empty((N, 3)), np.empty(NS)
    assert ctx.forces(D.BIG, f_out=f, e_out=e) == (e, f)
    with pytest.raises(ValueError):
        ctx.forces(D.BIG, e_out=np.empty(NS + 1))
    with pytest.raises(TypeError):
        ctx.forces(D.BIG, f_out=np.empty((N, 3), np.float32))
    e2, f2, w = ctx.forces(D.SMALL, virial=True)
    assert f2.shape == (N, 3) and e2.shape == (NS,) and w.shape == (NS, 3, 3)
    assert _last(ctx, "dmts_forces")[1] == D.SMALL


def test_respa_and_gradient_outputs(ctx):
    out = np.empty((4, NS, 3))
    assert ctx.respa_step(4, 3.0, 3, out=out) is out
    with pytest.raises(ValueError):
        ctx.respa_step(5, 3.0, 3, out=out)
    assert ctx.respa_step(2, 3.0, 3).shape == (2, NS, 3)
    assert ctx.respa_step(2, 3.0, 3, energies=False) is None
    assert _last(ctx, "dmts_respa_step")[4] is None
    ctx.respa_step(-1, 3.0, 3)                          # the library reports the bad count
    assert _last(ctx, "dmts_respa_step")[1] == -1
    frames = np.zeros((2, N, 3))
    loss, g = ctx.force_matching_grad(frames, frames)
    assert g.shape == (NP,)
    with pytest.raises(ValueError):
        ctx.force_matching_grad(frames, frames, grad_out=np.empty(NP - 1))
    with pytest.raises(ValueError):
        ctx.force_matching_grad(frames, np.zeros((3, N, 3)))
