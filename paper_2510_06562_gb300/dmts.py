"""ctypes binding of the DMTS C ABI (``include/dmts.h``, ``libdmts.so``).

Argument marshalling only: every step of the force evaluation and of the
integration runs in the library's CUDA kernels. Arrays may be NumPy arrays
(host memory) or torch tensors (host or CUDA memory); they are passed to the
library as raw pointers and the library tells host from device memory
itself. There is no CPU fallback: if the compiled library is missing, or
has no GPU to run on, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import inputs as _inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
# DMTS_LIBRARY selects another build of the library (e.g. the bounds-checked
# libdmts_check.so) for this process.
LIB_PATH = os.environ.get("DMTS_LIBRARY") or os.path.join(_HERE, "libdmts.so")

DMTS_OK = 0
STATUS = {0: "DMTS_OK", -1: "DMTS_ERR_ARG", -2: "DMTS_ERR_OOM", -3: "DMTS_ERR_CUDA",
          -4: "DMTS_ERR_CAPACITY", -5: "DMTS_ERR_NONFINITE", -6: "DMTS_ERR_TIMEOUT",
          -7: "DMTS_ERR_STATE"}
FP32, BF16_MLP = 0, 1
SMALL, BIG = 0, 1

EXPORTED = ("dmts_create", "dmts_set_state", "dmts_get_state", "dmts_forces", "dmts_respa_step",
            "dmts_destroy", "dmts_last_error", "dmts_neighbors", "dmts_set_params", "dmts_stream",
            "dmts_launch_count", "dmts_time_stages", "dmts_neighbors_noalloc",
            "dmts_force_matching_grad", "dmts_get_tuning", "dmts_neighbor_stats", "dmts_hmr_masses",
            "dmts_monitor", "dmts_monitor_reset", "dmts_set_tuning", "dmts_wait_selftest",
            "dmts_philox4x32_10", "dmts_distill_grad", "dmts_adam_step", "dmts_get_params",
            "dmts_get_bwd_tiles")


class DmtsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class ModelDesc(C.Structure):
    _fields_ = [("cutoff", C.c_double), ("n_radial", C.c_int), ("n_layers", C.c_int),
                ("n_feat", C.c_int), ("n_species", C.c_int), ("params", C.POINTER(C.c_double)),
                ("n_params", C.c_size_t), ("precision", C.c_int), ("rep_a", C.c_double),
                ("rep_rho", C.c_double), ("rep_cutoff", C.c_double)]


class SystemDesc(C.Structure):
    _fields_ = [("n_systems", C.c_int), ("atom_offset", C.POINTER(C.c_int)),
                ("species", C.POINTER(C.c_int)), ("mass", C.POINTER(C.c_double)),
                ("box", C.POINTER(C.c_double))]


_lib = None


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load ``libdmts.so`` (built by ``paper_2510_06562_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2510_06562_gb300.build.build()")
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.dmts_create.argtypes = [C.POINTER(ModelDesc), C.POINTER(ModelDesc), C.POINTER(SystemDesc),
                                C.c_char_p, C.POINTER(P)]
    lib.dmts_create.restype = C.c_int
    lib.dmts_set_state.argtypes = [P, P, P, C.c_int]
    lib.dmts_get_state.argtypes = [P, P, P]
    lib.dmts_forces.argtypes = [P, C.c_int, P, P, P]
    lib.dmts_respa_step.argtypes = [P, C.c_int, C.c_double, C.c_int, P]
    lib.dmts_destroy.argtypes = [P]
    lib.dmts_destroy.restype = None
    lib.dmts_last_error.argtypes = []
    lib.dmts_last_error.restype = C.c_char_p
    lib.dmts_neighbors.argtypes = [P, C.c_int, P, P, C.c_longlong, C.POINTER(C.c_longlong)]
    lib.dmts_set_params.argtypes = [P, C.c_int, P, C.c_size_t]
    lib.dmts_stream.argtypes = [P]
    lib.dmts_stream.restype = C.c_void_p
    lib.dmts_launch_count.argtypes = [P]
    lib.dmts_launch_count.restype = C.c_longlong
    lib.dmts_time_stages.argtypes = [P, C.c_int, C.c_int, P, C.c_int]
    lib.dmts_time_stages.restype = C.c_int
    lib.dmts_neighbors_noalloc.argtypes = [P, C.c_int, C.c_double, C.c_double, P, P, C.c_longlong,
                                           C.POINTER(C.c_longlong), P]
    lib.dmts_neighbors_noalloc.restype = C.c_int
    lib.dmts_force_matching_grad.argtypes = [P, C.c_int, P, P, P, P]
    lib.dmts_force_matching_grad.restype = C.c_int
    lib.dmts_get_tuning.argtypes = [P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.dmts_get_tuning.restype = C.c_int
    lib.dmts_neighbor_stats.argtypes = [P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
    lib.dmts_neighbor_stats.restype = C.c_int
    lib.dmts_hmr_masses.argtypes = [C.c_int, P, C.c_int, P, C.c_double, P]
    lib.dmts_hmr_masses.restype = C.c_int
    lib.dmts_monitor.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), P,
                                 C.c_int]
    lib.dmts_monitor.restype = C.c_int
    lib.dmts_monitor_reset.argtypes = [P]
    lib.dmts_monitor_reset.restype = C.c_int
    lib.dmts_set_tuning.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int]
    lib.dmts_get_bwd_tiles.argtypes = [P, C.c_int]
    lib.dmts_get_bwd_tiles.restype = C.c_int
    lib.dmts_set_tuning.restype = C.c_int
    lib.dmts_wait_selftest.argtypes = [P, C.c_int, C.c_int]
    lib.dmts_wait_selftest.restype = C.c_int
    lib.dmts_philox4x32_10.argtypes = [C.c_int, P, P, P]
    lib.dmts_philox4x32_10.restype = C.c_int
    lib.dmts_distill_grad.argtypes = [P, C.c_int, P, P, P, C.c_double, P, P]
    lib.dmts_distill_grad.restype = C.c_int
    lib.dmts_adam_step.argtypes = [P, C.c_int, P, P, P, C.c_longlong, C.c_double, C.c_double, C.c_double,
                                   C.c_double]
    lib.dmts_adam_step.restype = C.c_int
    lib.dmts_get_params.argtypes = [P, C.c_int, P, C.c_size_t]
    lib.dmts_get_params.restype = C.c_int
    for name in ("dmts_set_state", "dmts_get_state", "dmts_forces", "dmts_respa_step",
                 "dmts_neighbors", "dmts_set_params"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(code: int):
    if code != DMTS_OK:
        raise DmtsError(code, load_library().dmts_last_error().decode())


def _ptr(a):
    """Raw address of a NumPy array or torch tensor (contiguous), or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _f64(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.float64)
    import torch
    if a.dtype != torch.float64:
        raise TypeError("tensors must be float64")
    return a.contiguous()


def _numel(a) -> int:
    return int(a.size) if isinstance(a, np.ndarray) else int(a.numel())


def _in_f64(a, n: int, name: str):
    """An input of n float64 values: NumPy data is converted, a torch tensor
    must be float64 (made contiguous). The library reads exactly n values."""
    a = _f64(a)
    if a is not None and _numel(a) != n:
        raise ValueError(f"{name} must hold {n} values, got {_numel(a)}")
    return a


def _out_f64(a, n: int, name: str):
    """An output buffer the library writes n float64 values into: it must be
    float64, contiguous and of exactly that size (no conversion: the caller
    reads the buffer it passed)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        ok = a.dtype == np.float64 and a.flags.c_contiguous and a.flags.writeable
    elif hasattr(a, "data_ptr"):
        import torch
        ok = a.dtype == torch.float64 and a.is_contiguous()
    else:
        raise TypeError(f"{name}: unsupported array type {type(a)}")
    if not ok:
        raise TypeError(f"{name} must be a writable, contiguous float64 buffer")
    if _numel(a) != n:
        raise ValueError(f"{name} must hold {n} values, got {_numel(a)}")
    return a


def philox4x32_10(ctr, key) -> np.ndarray:
    """Raw Philox-4x32-10 words of the thermostat's generator, run on the
    current GPU (``dmts_philox4x32_10``): ctr [n, 4] and key [2] 32-bit words;
    returns [n, 4] uint32."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.zeros_like(c)
    _check(load_library().dmts_philox4x32_10(len(c), _ptr(c), _ptr(k), _ptr(out)))
    return out


def hmr_masses(mass, bonds, h_mass: float = 3.024) -> np.ndarray:
    """Hydrogen mass repartitioning (``dmts_hmr_masses``): hydrogens (< 1.5
    amu) bonded to a heavy atom get ``h_mass``; the heavy partner loses the
    difference. ``bonds`` [n_bonds, 2] atom indices."""
    m = np.ascontiguousarray(mass, dtype=np.float64)
    b = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1, 2))
    out = np.empty_like(m)
    _check(load_library().dmts_hmr_masses(len(m), _ptr(m), len(b), _ptr(b) if len(b) else None, float(h_mass),
                                          _ptr(out)))
    return out


class Context:
    """One simulation context: the big model, optionally the small model, and
    the systems (Algorithm 1's x, v, m and the two force fields)."""

    def __init__(self, system: "_inputs.System", big_arch, big_params, small_arch=None,
                 small_params=None, precision: int = FP32, options: str | None = None):
        lib = load_library()
        self._keep = []
        self.n_atoms = system.n_atoms
        self.n_systems = system.n_systems

        def desc(arch, params):
            p = np.ascontiguousarray(params, dtype=np.float64)
            self._keep.append(p)
            return ModelDesc(arch.cutoff, arch.n_radial, arch.n_layers, arch.n_feat, arch.n_species,
                             p.ctypes.data_as(C.POINTER(C.c_double)), p.size, precision,
                             getattr(arch, "rep_a", 0.0), getattr(arch, "rep_rho", 1.0),
                             getattr(arch, "rep_cutoff", 0.0))

        big = desc(big_arch, big_params)
        small = desc(small_arch, small_params) if small_arch is not None else None
        off = np.ascontiguousarray(system.atom_offset, dtype=np.int32)
        sp = np.ascontiguousarray(system.species, dtype=np.int32)
        ms = np.ascontiguousarray(system.mass, dtype=np.float64)
        bx = np.ascontiguousarray(system.box, dtype=np.float64)
        self._keep += [off, sp, ms, bx]
        sd = SystemDesc(system.n_systems, off.ctypes.data_as(C.POINTER(C.c_int)),
                        sp.ctypes.data_as(C.POINTER(C.c_int)), ms.ctypes.data_as(C.POINTER(C.c_double)),
                        bx.ctypes.data_as(C.POINTER(C.c_double)))
        h = C.c_void_p()
        _check(lib.dmts_create(C.byref(small) if small is not None else None, C.byref(big), C.byref(sd),
                               options.encode() if options else None, C.byref(h)))
        self._h = h
        self.has_small = small_arch is not None
        self.small_n_params = small_arch.param_count() if small_arch is not None else 0
        self.big_n_params = big_arch.param_count()

    # ---------------------------------------------------------------- state
    def set_state(self, x, v=None):
        if x is None:
            raise ValueError("x is required")
        x = _in_f64(x, 3 * self.n_atoms, "x")
        v = _in_f64(v, 3 * self.n_atoms, "v")
        _check(load_library().dmts_set_state(self._h, _ptr(x), _ptr(v), self.n_atoms))

    def get_state(self, x_out=None, v_out=None):
        x_out = np.empty((self.n_atoms, 3)) if x_out is None else _out_f64(x_out, 3 * self.n_atoms, "x_out")
        v_out = np.empty((self.n_atoms, 3)) if v_out is None else _out_f64(v_out, 3 * self.n_atoms, "v_out")
        _check(load_library().dmts_get_state(self._h, _ptr(x_out), _ptr(v_out)))
        return x_out, v_out

    # ---------------------------------------------------------------- forces
    def forces(self, which: int = BIG, virial: bool = False, f_out=None, e_out=None):
        f_out = np.empty((self.n_atoms, 3)) if f_out is None else _out_f64(f_out, 3 * self.n_atoms, "f_out")
        e_out = np.empty(self.n_systems) if e_out is None else _out_f64(e_out, self.n_systems, "e_out")
        w_out = np.empty((self.n_systems, 3, 3)) if virial else None
        _check(load_library().dmts_forces(self._h, which, _ptr(f_out), _ptr(e_out), _ptr(w_out)))
        return (e_out, f_out, w_out) if virial else (e_out, f_out)

    def neighbors(self, which: int = BIG):
        row_ptr = np.empty(self.n_atoms + 1, dtype=np.int32)
        n = C.c_longlong(0)
        lib = load_library()
        code = lib.dmts_neighbors(self._h, which, _ptr(row_ptr), None, 0, C.byref(n))
        if code not in (DMTS_OK, -4):
            _check(code)
        col = np.empty(max(1, n.value), dtype=np.int32)
        _check(lib.dmts_neighbors(self._h, which, _ptr(row_ptr), _ptr(col), col.size, C.byref(n)))
        return row_ptr, col[:n.value]

    def set_params(self, which: int, params):
        p = np.ascontiguousarray(params, dtype=np.float64)
        _check(load_library().dmts_set_params(self._h, which, _ptr(p), p.size))

    # ---------------------------------------------------------------- dynamics
    def respa_step(self, n_outer: int, dt_outer: float, n_inner: int, energies: bool = True, out=None):
        """n_outer steps of Algorithm 1; returns [n_outer, n_systems, 3]
        (E_pot big, E_kin, E_tot) or None."""
        if energies and out is None and n_outer >= 0:
            out = np.empty((n_outer, self.n_systems, 3))
        elif energies and out is not None and n_outer >= 0:
            out = _out_f64(out, 3 * n_outer * self.n_systems, "out")
        _check(load_library().dmts_respa_step(self._h, n_outer, float(dt_outer), n_inner,
                                              _ptr(out) if energies else None))
        return out if energies else None

    def force_matching_grad(self, frames, f_ref, grad_out=None):
        """Distillation loss of the small model against reference forces and
        its parameter gradient: (loss, grad [n_params]). frames, f_ref:
        [M, N, 3] float64 (NumPy or torch, host or device)."""
        frames = _f64(frames)
        f_ref = _f64(f_ref)
        m = frames.shape[0]
        if tuple(f_ref.shape) != tuple(frames.shape) or frames.shape[1:] != (self.n_atoms, 3):
            raise ValueError("frames and f_ref must both be [M, N, 3]")
        loss = np.zeros(1)
        grad = np.empty(self.small_n_params) if grad_out is None else _out_f64(grad_out, self.small_n_params,
                                                                               "grad_out")
        _check(load_library().dmts_force_matching_grad(self._h, m, _ptr(frames), _ptr(f_ref), _ptr(loss),
                                                       _ptr(grad)))
        return float(loss[0]), grad

    def distill_grad(self, frames, f_ref, e_ref, lambda_e: float, grad_out=None):
        """Energy and force distillation loss of the small model and its
        parameter gradient (``dmts_distill_grad``): (loss, grad [n_params]).
        frames, f_ref: [M, N, 3]; e_ref: [M] float64 (host or device)."""
        frames = _f64(frames)
        f_ref = _f64(f_ref)
        e_ref = _f64(e_ref)
        m = frames.shape[0]
        if tuple(f_ref.shape) != tuple(frames.shape) or frames.shape[1:] != (self.n_atoms, 3):
            raise ValueError("frames and f_ref must both be [M, N, 3]")
        if _numel(e_ref) != m:
            raise ValueError("e_ref must hold one energy per frame")
        loss = np.zeros(1)
        grad = np.empty(self.small_n_params) if grad_out is None else _out_f64(grad_out, self.small_n_params,
                                                                               "grad_out")
        _check(load_library().dmts_distill_grad(self._h, m, _ptr(frames), _ptr(f_ref), _ptr(e_ref),
                                                float(lambda_e), _ptr(loss), _ptr(grad)))
        return float(loss[0]), grad

    def adam_step(self, which: int, grad, m1: np.ndarray, m2: np.ndarray, t: int, lr: float,
                  beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        """One Adam step on a model's parameters (``dmts_adam_step``); m1, m2
        are the caller's float64 moment arrays, updated in place."""
        n = self.small_n_params if which == SMALL else self.big_n_params
        g = _f64(grad)
        for a, name in ((m1, "m1"), (m2, "m2")):
            if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.size == n and a.flags.c_contiguous):
                raise TypeError(f"{name} must be a contiguous float64 NumPy array of {n} values")
        _check(load_library().dmts_adam_step(self._h, which, _ptr(g), _ptr(m1), _ptr(m2), int(t), float(lr),
                                             float(beta1), float(beta2), float(eps)))

    def get_params(self, which: int = SMALL) -> np.ndarray:
        n = self.small_n_params if which == SMALL else self.big_n_params
        out = np.empty(n)
        _check(load_library().dmts_get_params(self._h, which, _ptr(out), n))
        return out

    def time_stages(self, which: int = BIG, reps: int = 10) -> dict:
        """Per-stage milliseconds of one force evaluation (CUDA events)."""
        out = np.zeros(32)
        n = load_library().dmts_time_stages(self._h, which, reps, _ptr(out), out.size)
        if n < 0:
            _check(n)
        L = (n - 3) // 4
        names = ["neighbors", "embed"] + [f"edge_fwd_l{l}" for l in range(L)] + \
                [f"atom_fwd_l{l}" for l in range(L)] + [f"edge_bwd_l{l}" for l in range(L)] + \
                [f"atom_bwd_l{l}" for l in range(L)] + ["energy_sum"]
        return dict(zip(names, out[:n].tolist()))

    def tuning(self, which: int = BIG) -> dict:
        """Chosen work granularity of one model's kernels."""
        f, b = C.c_int(0), C.c_int(0)
        code = load_library().dmts_get_tuning(self._h, which, C.byref(f), C.byref(b))
        if code < 0:
            _check(code)
        t = load_library().dmts_get_bwd_tiles(self._h, which)
        if t < 0:
            _check(t)
        return {"tuned": bool(code), "atoms_fwd": f.value, "atoms_bwd": b.value, "bwd_tiles": t}

    def set_tuning(self, which: int, fwd: int, bwd: int, bwd_tiles: int = 0):
        """Fix one model's work granularity (``dmts_set_tuning``)."""
        _check(load_library().dmts_set_tuning(self._h, which, int(fwd), int(bwd), int(bwd_tiles)))

    def wait_selftest(self, arrive: bool, max_polls: int = 1000) -> int:
        """Run the bounded-wait self-test (``dmts_wait_selftest``); returns its
        status code (0, or -6 when the wait gave up) without raising."""
        return load_library().dmts_wait_selftest(self._h, 1 if arrive else 0, int(max_polls))

    @property
    def stream(self) -> int:
        return load_library().dmts_stream(self._h) or 0

    @property
    def launch_count(self) -> int:
        return load_library().dmts_launch_count(self._h)

    def monitor(self) -> dict:
        """Force-difference monitor: max |F_big - F_small| (eV/A), outer steps
        redone by the fallback, flagged atoms, log10 histogram (48 bins of 1/8
        decade from 1e-3 eV/A)."""
        mx, nf, na = C.c_double(), C.c_longlong(), C.c_longlong()
        hist = np.zeros(48, dtype=np.int64)
        n = load_library().dmts_monitor(self._h, C.byref(mx), C.byref(nf), C.byref(na), _ptr(hist), hist.size)
        if n < 0:
            _check(n)
        return {"max_df": mx.value, "n_fallback": nf.value, "n_flagged": na.value, "hist": hist[:n]}

    def monitor_reset(self):
        _check(load_library().dmts_monitor_reset(self._h))

    def neighbor_stats(self) -> tuple[int, int]:
        """(displacement checks, candidate-row rebuilds) of the Verlet-skin lists."""
        a, b = C.c_longlong(), C.c_longlong()
        _check(load_library().dmts_neighbor_stats(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def close(self):
        if getattr(self, "_h", None):
            load_library().dmts_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class ForceMatchingLoss:
    """torch.autograd.Function for the distillation loss of the small model:
    ``loss = ForceMatchingLoss.apply(theta, ctx, frames, f_ref)`` with theta
    the flat float64 parameter tensor of the small model; ``loss.backward()``
    fills ``theta.grad`` from the library's adjoint kernels (gradient through
    the forces). The context's small-model parameters are set to theta."""

    _fn = None

    @classmethod
    def apply(cls, theta, context, frames, f_ref):
        if cls._fn is None:
            import torch

            class _Fn(torch.autograd.Function):
                @staticmethod
                def forward(fctx, th, ctx_obj, fr, fref):
                    ctx_obj.set_params(SMALL, th.detach().cpu().numpy())
                    loss, grad = ctx_obj.force_matching_grad(fr, fref)
                    fctx.save_for_backward(torch.as_tensor(grad, dtype=th.dtype, device=th.device))
                    return torch.tensor(loss, dtype=th.dtype, device=th.device)

                @staticmethod
                def backward(fctx, g_out):
                    (grad,) = fctx.saved_tensors
                    return g_out * grad, None, None, None

            cls._fn = _Fn
        return cls._fn.apply(theta, context, frames, f_ref)
