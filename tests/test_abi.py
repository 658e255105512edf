"""The C ABI library builds, loads and exports every declared symbol; argument
validation that needs no GPU (CPU only, no compute calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2510_06562_gb300 import build as B
from paper_2510_06562_gb300 import dmts as D
from paper_2510_06562_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return D.load_library()


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dmts_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared("dmts.h")
    for n in ("dmts_create", "dmts_set_state", "dmts_forces", "dmts_respa_step", "dmts_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for header in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if header.endswith(".h"):
            for name in _declared(header):
                assert hasattr(lib, name), f"{name} declared in {header} but not exported"
    assert set(D.EXPORTED) <= set(_declared("dmts.h"))


def test_missing_library_fails_loudly(tmp_path):
    saved = D._lib
    D._lib = None
    try:
        with pytest.raises(ImportError):
            D.load_library(str(tmp_path / "nope.so"))
    finally:
        D._lib = saved


def test_null_and_bad_arguments_rejected_before_device_use(lib):
    out = ctypes.c_void_p(1)
    assert lib.dmts_create(None, None, None, None, ctypes.byref(out)) == -1
    assert out.value is None
    assert b"NULL" in lib.dmts_last_error() or b"big" in lib.dmts_last_error()
    arch = I.big_arch()
    p = I.init_params(arch, 3)
    bad = D.ModelDesc(arch.cutoff, arch.n_radial, arch.n_layers, arch.n_feat, arch.n_species,
                      p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), p.size - 1, 0)
    assert lib.dmts_create(None, ctypes.byref(bad), None, None, ctypes.byref(out)) == -1
    assert b"n_params" in lib.dmts_last_error()
    odd = D.ModelDesc(arch.cutoff, arch.n_radial, arch.n_layers, 48, arch.n_species,
                      p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), p.size, 0)
    assert lib.dmts_create(None, ctypes.byref(odd), None, None, ctypes.byref(out)) == -1
    lib.dmts_destroy(None)                                   # NULL-safe
    assert lib.dmts_set_state(None, None, None, 0) == -1
    assert lib.dmts_forces(None, 1, None, None, None) == -1
    assert lib.dmts_respa_step(None, 1, 1.0, 1, None) == -1
    assert lib.dmts_stream(None) is None
    assert lib.dmts_launch_count(None) == -1


def test_system_validation(lib):
    arch = I.big_arch()
    p = I.init_params(arch, 3)
    big = D.ModelDesc(arch.cutoff, arch.n_radial, arch.n_layers, arch.n_feat, arch.n_species,
                      p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), p.size, 0)
    s = I.water_192(0)
    off = np.array([0, 192], np.int32)
    sp = s.species.astype(np.int32).copy()
    ms = s.mass.copy()
    for box, species, code in ((9.0, sp, -1), (12.42, np.full(192, 5, np.int32), -1)):
        bx = np.array([box])
        sd = D.SystemDesc(1, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                          species.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                          ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          bx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        out = ctypes.c_void_p()
        assert lib.dmts_create(None, ctypes.byref(big), ctypes.byref(sd), None, ctypes.byref(out)) == code


# ------------------------------------------------------------------ host-only entry points

@pytest.mark.parametrize("make", [lambda: I.water_192(0), lambda: I.make_vacuum_batch(64, 10, 60, seed=0)])
def test_hmr_masses_equal_the_oracle(lib, make):
    """dmts_hmr_masses (host code, no GPU) against the oracle's definition,
    bit for bit, on the generators' bond lists."""
    from oracle import integrate as G
    s = make()
    got = D.hmr_masses(s.mass, s.bonds, 3.024)
    np.testing.assert_array_equal(got, G.hmr_masses(s.mass, s.bonds, 3.024))
    off = s.atom_offset
    for k in range(len(off) - 1):
        assert abs(got[off[k]:off[k + 1]].sum() - s.mass[off[k]:off[k + 1]].sum()) < 1e-9
    if s.box[0] > 0:                                   # water: O 15.999 - 2 (3.024 - 1.008)
        np.testing.assert_allclose(got[0::3], 11.967)
        np.testing.assert_allclose(got[1::3], 3.024)


def test_hmr_masses_rejects_bad_input(lib):
    with pytest.raises(D.DmtsError):
        D.hmr_masses(np.array([16.0, 1.0]), np.array([[0, 2]]))
    with pytest.raises(D.DmtsError):
        D.hmr_masses(np.array([2.0, 1.0]), np.array([[0, 1]]), h_mass=3.5)
