"""The C ABI library builds, loads and exports every declared symbol; argument
validation that needs no GPU (CPU only, no compute calls)."""
import ctypes
import json
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


# ------------------------------------------------------------------ options

def _create_rc(lib, options):
    """dmts_create on 192 waters with `options`; returns its status (a
    context created on a machine with a GPU is destroyed at once)."""
    arch = I.big_arch()
    p = I.init_params(arch, 3)
    big = D.ModelDesc(arch.cutoff, arch.n_radial, arch.n_layers, arch.n_feat, arch.n_species,
                      p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), p.size, 0)
    s = I.water_192(0)
    off = np.array([0, s.n_atoms], np.int32)
    sp = s.species.astype(np.int32).copy()
    ms = s.mass.copy()
    bx = np.array(s.box, dtype=np.float64)
    sd = D.SystemDesc(1, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                      sp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                      ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      bx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    out = ctypes.c_void_p()
    rc = lib.dmts_create(None, ctypes.byref(big), ctypes.byref(sd),
                         options.encode() if options is not None else None, ctypes.byref(out))
    if rc == 0:
        lib.dmts_destroy(out)
    return rc


# every option set the tests and the benchmark pass, and the documented forms
GOOD_OPTIONS = [
    None, "", "  ", "{}", ' { } ',
    '{"autotune": 0}', '{"autotune": false}', '{"autotune": true, "concurrent_models": false}',
    json.dumps({"langevin_friction": 20.0, "temperature": 300.0, "seed": 12345, "autotune": 0}),
    json.dumps({"langevin_friction": 1.0, "temperature": 300.0, "seed": 7, "fallback_threshold": 6.505}),
    json.dumps({"fallback_threshold": 1e-9, "langevin_friction": 1.0, "seed": 5}),
    '{"row_capacity": 4, "edge_capacity_factor": 0.05, "cell_capacity": 2}',
    json.dumps({"skin": 1.0, "autotune": 0, "row_capacity": 8}),
    json.dumps({"atom_tensor_cores": 0}), json.dumps({"atom_tensor_cores": True}),
    '{"atoms_per_cta_big": 8, "atoms_per_cta_small": 16}',
    '{\n  "skin": 2e0,\n  "seed": 0\n}',
]

BAD_OPTIONS = [
    '{"autotun": 0}',                          # misspelt key
    '{"Skin": 1.0}',                           # keys are case-sensitive
    '{"skin": "1.0"}',                         # string value
    '{"skin": null}',
    '{"skin": [1]}',
    '{"skin": 1.0, "skin": 2.0}',              # repeated key
    '{"skin": 1.0',                            # unterminated object
    '{"skin" 1.0}',
    '{"skin": 1.0,}',                          # trailing comma
    '{"skin": 1.0} x',                         # text after the object
    '"skin": 1.0',
    '{skin: 1.0}',
    '{"skin": .5}',
    '{"skin": nan}',
    '{"skin": 1e999}',                         # not finite
    '{"ski\\n": 1}',                           # escapes are not option keys
]


@pytest.mark.parametrize("opts", GOOD_OPTIONS)
def test_options_accepted(lib, opts):
    """Accepted options pass on to the device check: DMTS_ERR_CUDA without a
    GPU, success with one."""
    assert _create_rc(lib, opts) in (0, -3), lib.dmts_last_error()


@pytest.mark.parametrize("opts", BAD_OPTIONS)
def test_options_rejected_before_device_use(lib, opts):
    assert _create_rc(lib, opts) == -1
    assert b"options" in lib.dmts_last_error()


def test_option_keys_match_the_header():
    """Every option key the library accepts is documented in the header, and
    every quoted key the header documents as an option is accepted."""
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = open(os.path.join(root, "paper_2510_06562_gb300", "csrc", "dmts.cu")).read()
    block = src[src.index("kOptionKeys[] = {"):]
    keys = set(re.findall(r'"([a-z_]+)"', block[:block.index("};")]))
    header = open(os.path.join(root, "include", "dmts.h")).read()
    for k in keys:
        assert f'"{k}"' in header, k
    assert len(keys) == 13


def test_options_parser_survives_arbitrary_text(lib):
    """Whatever the options string, dmts_create returns a status: an
    argument error, or (valid options) the device check's result."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")
    keys = ["skin", "autotune", "seed", "temperature", "cell_capacity", "bogus", ""]
    values = st.one_of(st.floats(allow_nan=True, allow_infinity=True).map(repr), st.integers().map(str),
                       st.sampled_from(["true", "false", "null", '"x"', "[]", "{}", "-", "1e", ".5", "0x10"]))
    pairs = st.lists(st.tuples(st.sampled_from(keys), values), max_size=4)
    objects = pairs.map(lambda kv: "{" + ", ".join(f'"{k}": {v}' for k, v in kv) + "}")
    texts = st.one_of(st.text(max_size=40), objects, objects.map(lambda s: s[:-1]), objects.map(lambda s: s + ","))

    @hyp.settings(max_examples=300, deadline=None, derandomize=True)
    @hyp.given(texts)
    def check(opts):
        if "\x00" in opts:
            return                                   # a C string ends at the first NUL
        assert _create_rc(lib, opts) in (-1, -3, 0)

    check()
