"""The allocation-free neighbour list, dmts_neighbors_noalloc.

It serves callers that cannot allocate device memory themselves or let a
library do so: an MD engine that owns all device memory through its own pool,
or code under a fixed memory budget. Its scratch
is a static device array, so these checks call it twice in a row on different
systems (the second call sees the first call's leftovers) and compare each
result, through the C ABI, with the context-based dmts_neighbors: the pair
sets must be identical (integer output, bit-exact). Here the test allocates
the input and output buffers with torch, as such a caller's pool would.

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from oracle import model as M
from paper_2510_06562_gb300 import build as B
from paper_2510_06562_gb300 import dmts as D
from paper_2510_06562_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _noalloc(lib, torch, s, cutoff, capacity):
    x = torch.tensor(s.x, dtype=torch.float64, device="cuda")
    row_ptr = torch.full((s.n_atoms + 1,), -7, dtype=torch.int32, device="cuda")
    col = torch.full((max(1, capacity),), -7, dtype=torch.int32, device="cuda")
    n = ctypes.c_longlong(-1)
    code = lib.dmts_neighbors_noalloc(x.data_ptr(), s.n_atoms, float(s.box[0]), cutoff, row_ptr.data_ptr(),
                                      col.data_ptr(), capacity, ctypes.byref(n), None)
    torch.cuda.synchronize()
    return code, row_ptr.cpu().numpy(), col.cpu().numpy()[:max(0, n.value)], n.value


def _context(s, which):
    sa, sp, ba, bp = (I.small_arch(s.n_species), I.init_params(I.small_arch(s.n_species), 2),
                      I.big_arch(s.n_species), I.init_params(I.big_arch(s.n_species), 3))
    with D.Context(s, ba, bp, sa, sp) as ctx:
        ctx.set_state(s.x)
        return ctx.neighbors(which)


def test_noalloc_neighbors_match_context_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    B.build()
    lib = D.load_library()
    cases = [(I.water_12288(0), 5.0, D.BIG), (I.water_192(0), 3.5, D.SMALL)]
    for s, rc, which in cases:
        code, rp, col, n = _noalloc(lib, torch, s, rc, 64 * s.n_atoms + 1024)
        assert code == 0, lib.dmts_last_error()
        ref_rp, ref_col = _context(s, which)
        assert n == ref_rp[-1]
        np.testing.assert_array_equal(rp, ref_rp)
        np.testing.assert_array_equal(col, ref_col)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    pytest.importorskip("torch")
    lib = D.load_library()
    n = ctypes.c_longlong(0)
    code = lib.dmts_neighbors_noalloc(ctypes.c_void_p(16), 16385, 50.0, 5.0, ctypes.c_void_p(16),
                                      ctypes.c_void_p(16), 1, ctypes.byref(n), None)
    assert code == -1
    assert b"16384" in lib.dmts_last_error()


def _pairs(rp, col):
    return np.repeat(np.arange(len(rp) - 1), np.diff(rp)), col.astype(np.int64)


def test_noalloc_open_boundaries_and_all_pairs_path():
    """The branches the periodic cell-list case does not take: one molecule
    without a box (its own fixed-point frame) and the 192-atom box at 5.0 A,
    where fewer than three cells fit per edge and every pair is tested;
    each against the oracle's brute-force pair list, twice in a row."""
    torch = pytest.importorskip("torch")
    lib = D.load_library()
    mol = I.make_vacuum_batch(1, 60, 60, seed=4)
    assert mol.box[0] <= 0
    cases = [(mol, 5.0), (I.water_192(0), 5.0), (mol, 3.5), (I.water_192(0), 5.0)]
    for s, rc in cases:
        code, rp, col, n = _noalloc(lib, torch, s, rc, 64 * s.n_atoms + 1024)
        assert code == 0, lib.dmts_last_error()
        oi, oj = M.pair_list(s.x, s.atom_offset, s.box, rc)
        gi, gj = _pairs(rp, col)
        assert n == len(oi)
        np.testing.assert_array_equal(gi, oi)
        np.testing.assert_array_equal(gj, oj)


def test_noalloc_capacity_errors_still_write_the_counts():
    """Too small an output: DMTS_ERR_CAPACITY, with *n_pairs and row_ptr
    written; a row longer than the 256 neighbours the fill pass sorts:
    DMTS_ERR_CAPACITY with a message."""
    torch = pytest.importorskip("torch")
    lib = D.load_library()
    s = I.water_192(0)
    code, rp, _, n = _noalloc(lib, torch, s, 3.5, 100)
    assert code == -4
    oi, _ = M.pair_list(s.x, s.atom_offset, s.box, 3.5)
    assert n == len(oi) > 100
    np.testing.assert_array_equal(np.diff(rp), np.bincount(oi, minlength=s.n_atoms))
    rng = np.random.default_rng(2)
    x = rng.uniform(0.0, 3.0, size=(300, 3))           # every atom within 5.2 A of every other
    dense = I.System(x=x, species=np.zeros(300, np.int32), mass=np.ones(300),
                     atom_offset=np.array([0, 300], np.int32), box=np.array([0.0]), n_species=1)
    code, _, _, n = _noalloc(lib, torch, dense, 6.0, 300 * 300)
    assert code == -4
    assert b"256" in lib.dmts_last_error()
    # and the entry point still works afterwards
    code, rp, col, n = _noalloc(lib, torch, s, 3.5, 64 * s.n_atoms)
    assert code == 0 and n == len(oi)
