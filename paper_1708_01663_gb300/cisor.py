"""Thin ctypes binding of libcisor (include/cisor.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts arrays to
pointers and structs.  Arrays may be torch tensors (CUDA or CPU) or numpy
arrays; complex arrays must be contiguous complex64.  Outputs are caller
allocated.  Loading fails loudly when libcisor.so has not been built: there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import re
from ctypes import POINTER, Structure, c_char_p, c_double, c_int, c_longlong, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcisor.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "cisor.h")

OK, ERR_INVALID_ARG, ERR_NOT_CONVERGED, ERR_BREAKDOWN, ERR_OOM, ERR_CUDA = range(6)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "NOT_CONVERGED", 3: "BREAKDOWN", 4: "OOM", 5: "CUDA"}


class Geometry(Structure):
    _fields_ = [("dim", c_int), ("n", c_int), ("delta", c_double), ("wavelength", c_double),
                ("eps_b", c_double), ("T", c_int), ("tx_angles", POINTER(c_double)), ("M", c_int),
                ("rx_pos", POINTER(c_double)), ("complex_f", c_int), ("pad", c_int), ("tx_kind", c_int),
                ("vectorial", c_int)]


class SolveOpts(Structure):
    _fields_ = [("tol", c_double), ("max_iter", c_int), ("x0_mode", c_int)]


class SolveInfo(Structure):
    _fields_ = [("iters_max", c_int), ("iters_mean", c_double), ("resid_max", c_double),
                ("n_not_converged", c_int), ("adj_iters_max", c_int), ("adj_iters_mean", c_double),
                ("adj_resid_max", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class FistaState(Structure):
    _fields_ = [("f", c_void_p), ("s", c_void_p), ("t", c_double), ("k", c_int), ("alpha", c_double),
                ("gamma", c_double), ("tau", c_double), ("tv_iters", c_int), ("lo", c_double),
                ("hi", c_double), ("lo_im", c_double), ("hi_im", c_double), ("D", c_double), ("tv_kind", c_int)]


class CisorError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"cisor status {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def declared_functions():
    """Names of the entry points declared in include/cisor.h."""
    with open(HEADER) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:const char\*|cisor_status)\s+(cisor_\w+)\s*\(", text, re.M)))


def load(path: str = LIB_PATH):
    """Load libcisor.so and declare the signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1708_01663_gb300.build.build() "
                           "(the CUDA path has no fallback)")
    lib = ctypes.CDLL(path)
    vp, i, d = c_void_p, c_int, c_double
    sig = {
        "cisor_create": [POINTER(c_void_p), POINTER(Geometry), vp],
        "cisor_destroy": [vp],
        "cisor_sizes": [vp, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_longlong)],
        "cisor_green_spectrum": [vp, vp],
        "cisor_sensing_matrix": [vp, vp],
        "cisor_incident": [vp, vp],
        "cisor_apply_A": [vp, vp, vp, vp, i, i],
        "cisor_forward": [vp, vp, vp, vp, vp, vp, POINTER(SolveOpts), POINTER(SolveInfo)],
        "cisor_sense": [vp, vp, vp, vp],
        "cisor_sense_adjoint": [vp, vp, vp, vp, vp],
        "cisor_grad": [vp, vp, vp, vp, POINTER(c_double), POINTER(SolveOpts), POINTER(SolveInfo)],
        "cisor_tv_prox": [vp, vp, vp, d, i, d, d, d, d],
        "cisor_tv_prox_aniso": [vp, vp, vp, d, i, d, d, d, d],
        "cisor_step": [vp, POINTER(FistaState), vp, POINTER(SolveOpts), POINTER(SolveInfo)],
        "cisor_step_update": [vp, POINTER(FistaState), vp, c_double],
        "cisor_set_cols_cta": [vp, c_int],
        "cisor_set_rx_mask": [vp, vp],
        "cisor_solve_iterations": [vp, c_int, POINTER(c_int), POINTER(c_int)],
        "cisor_launch_count": [vp, POINTER(c_longlong)],
        "cisor_device_info": [i, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int)],
        "cisor_tc_wait_selftest": [i, i, POINTER(c_int)],
        "cisor_time_matvec": [vp, vp, i, i, POINTER(c_double)],
        "cisor_apply_A_static": [vp, vp, vp, vp, i, i, i, i, vp],
        "cisor_data_term": [vp, vp, vp, POINTER(c_double), POINTER(SolveOpts), POINTER(SolveInfo)],
        "cisor_autotune": [vp, i, POINTER(c_int)],
        "cisor_set_tx_chunk": [vp, c_int],
        "cisor_tuning": [vp, POINTER(c_int), POINTER(c_int)],
        "cisor_set_solve_loop": [vp, c_int],
        "cisor_batch_set_solve_loop": [vp, c_int],
        "cisor_fno_create": [POINTER(c_void_p), i, ctypes.c_ulonglong, vp],
        "cisor_fno_destroy": [vp],
        "cisor_fno_num_params": [vp, POINTER(c_longlong)],
        "cisor_fno_get_params": [vp, vp, i],
        "cisor_fno_set_params": [vp, vp],
        "cisor_fno_forward": [vp, vp, i, vp, i, vp],
        "cisor_fno_loss_grad": [vp, vp, i, vp, vp, i, POINTER(c_double), vp],
        "cisor_fno_train_step": [vp, vp, i, vp, vp, i, d, POINTER(c_double)],
        "cisor_fno_warm_start": [vp, vp, vp, vp],
        "cisor_batch_create": [POINTER(c_void_p), POINTER(Geometry), i, vp, i],
        "cisor_batch_destroy": [vp],
        "cisor_batch_context": [vp, i, POINTER(c_void_p)],
        "cisor_batch_forward": [vp, POINTER(c_void_p), POINTER(c_void_p), POINTER(SolveOpts), POINTER(SolveInfo)],
        "cisor_batch_grad": [vp, POINTER(c_void_p), POINTER(c_void_p), POINTER(c_void_p), POINTER(c_double),
                             POINTER(SolveOpts), POINTER(SolveInfo)],
        "cisor_data_backward": [vp, vp, POINTER(SolveOpts), POINTER(SolveInfo)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = c_int
    lib.cisor_last_error.restype = c_char_p
    lib.cisor_last_error.argtypes = []
    lib.cisor_version.restype = c_char_p
    lib.cisor_version.argtypes = []
    _lib = lib
    return lib


def last_error() -> str:
    return load().cisor_last_error().decode()


def _check(status, allow=()):
    if status != OK and status not in allow:
        raise CisorError(status, last_error())
    return status


def ptr(a, count=None, dtype="complex64"):
    """Raw pointer of a contiguous torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch
        if not a.is_contiguous():
            raise ValueError("array must be contiguous")
        if str(a.dtype).replace("torch.", "") != dtype:
            raise TypeError(f"expected {dtype}, got {a.dtype}")
        if count is not None and a.numel() != count:
            raise ValueError(f"expected {count} elements, got {a.numel()}")
        return a.data_ptr()
    arr = a
    if not isinstance(arr, np.ndarray) or not arr.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be a contiguous numpy array or torch tensor")
    if arr.dtype != np.dtype(dtype):
        raise TypeError(f"expected {dtype}, got {arr.dtype}")
    if count is not None and arr.size != count:
        raise ValueError(f"expected {count} elements, got {arr.size}")
    return arr.ctypes.data


def device_info(device=0):
    """SM count, peak SM clock (kHz), FP32 lanes per SM and compute capability x 10 of a CUDA device."""
    lib = load()
    v = [c_int() for _ in range(4)]
    _check(lib.cisor_device_info(int(device), *[ctypes.byref(x) for x in v]))
    return {"sm_count": v[0].value, "max_clock_khz": v[1].value, "fp32_lanes": v[2].value, "cc": v[3].value}


def tc_wait_selftest(arrive, polls):
    """Bounded tensor-core wait on the current device: True if the mbarrier completed within `polls` polls."""
    v = c_int(-1)
    _check(load().cisor_tc_wait_selftest(1 if arrive else 0, int(polls), ctypes.byref(v)))
    return v.value == 1


def apply_A_static(ghat_scaled, f, x, y, n, P, adjoint=False, stream=None):
    """Allocation-free batched matvec (device tensors only): y = A x or A^H x."""
    nvec = x.numel() // (n * n)
    st = load().cisor_apply_A_static(ptr(ghat_scaled, P * P), ptr(f, n * n), ptr(x, nvec * n * n),
                                     ptr(y, nvec * n * n), int(n), int(P), int(nvec), 1 if adjoint else 0,
                                     _current_stream() if stream is None else stream)
    return _check(st)


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


class Cisor:
    """One imaging geometry: tables and workspace on the current CUDA device."""

    def __init__(self, n=None, delta=None, tx_angles=None, rx_pos=None, wavelength=1.0, eps_b=1.0, complex_f=False,
                 pad=0, stream=None, dim=2, tx_kind=0, vectorial=False, _handle=None):
        """2D: tx_angles [T] plane-wave angles, rx_pos [M, 2].  3D (dim=3):
        tx_angles [T, 3] unit propagation directions, rx_pos [M, 3].
        tx_kind=1 (or "point"): tx_angles holds source positions [T, dim].
        vectorial=True (dim=3): the vectorial model of the appendix; tx_angles is
        [T, 6] (unit direction, orthogonal unit polarisation) and fields are [T, 3, N]."""
        lib = load()
        self._lib = lib
        self._owned = _handle is None
        if _handle is not None:  # view of a context owned by a Batch
            self._ctx = _handle
            self.stream = stream
            self.complex_f = bool(complex_f)
            self.dim = int(dim)
            self.ncomp = 3 if vectorial else 1
            self._read_sizes()
            return
        self.dim = int(dim)
        self.ncomp = 3 if vectorial else 1
        kind = 1 if tx_kind in (1, "point") else 0
        per_tx = (6,) if vectorial else ((self.dim,) if kind == 1 else ((3,) if self.dim == 3 else ()))
        self._ang = np.ascontiguousarray(tx_angles, dtype=np.float64).reshape((-1,) + per_tx)
        self._rx = np.ascontiguousarray(rx_pos, dtype=np.float64).reshape(-1, self.dim)
        g = Geometry(self.dim, int(n), float(delta), float(wavelength), float(eps_b), len(self._ang),
                     self._ang.ctypes.data_as(POINTER(c_double)), len(self._rx),
                     self._rx.ctypes.data_as(POINTER(c_double)), 1 if complex_f else 0, int(pad), kind,
                     1 if vectorial else 0)
        self._ctx = c_void_p()
        self.stream = _current_stream() if stream is None else stream
        _check(lib.cisor_create(ctypes.byref(self._ctx), ctypes.byref(g), self.stream))
        self._read_sizes()
        self.complex_f = bool(complex_f)

    def _read_sizes(self):
        n_, P, T, M, N = c_int(), c_int(), c_int(), c_int(), c_longlong()
        _check(self._lib.cisor_sizes(self._ctx, ctypes.byref(n_), ctypes.byref(P), ctypes.byref(T),
                                     ctypes.byref(M), ctypes.byref(N)))
        self.n, self.P, self.T, self.M, self.N = n_.value, P.value, T.value, M.value, N.value
        self.Nf = self.N * getattr(self, "ncomp", 1)  # field length per transmitter

    def autotune(self, reps=5):
        """Time the column-kernel shapes (512, 256; 16 = two-stage, P = 128 / 256 / 2D 512) and keep the fastest."""
        nt = c_int()
        _check(self._lib.cisor_autotune(self._ctx, int(reps), ctypes.byref(nt)))
        return nt.value

    def set_rx_mask(self, mask):
        """Per-transmitter active receivers, [T, M] (non-zero = active); None restores all."""
        if mask is None:
            return _check(self._lib.cisor_set_rx_mask(self._ctx, None))
        m = np.ascontiguousarray(np.asarray(mask) != 0, dtype=np.uint8)
        assert m.shape == (self.T, self.M)
        self._mask = m
        return _check(self._lib.cisor_set_rx_mask(self._ctx, m.ctypes.data_as(c_void_p)))

    def set_tx_chunk(self, chunk):
        """Transforms per FFT-convolution launch (0: all at once); results do not depend on it."""
        return _check(self._lib.cisor_set_tx_chunk(self._ctx, int(chunk)))

    def set_solve_loop(self, device_loop=True):
        """1: whole solve in one graph launch (device-side loop); 0: host-driven chunks."""
        return _check(self._lib.cisor_set_solve_loop(self._ctx, 1 if device_loop else 0))

    def tuning(self):
        """(column shape, transmitter chunk) in use."""
        a, b = c_int(), c_int()
        _check(self._lib.cisor_tuning(self._ctx, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def set_cols_cta(self, nt):
        """Column-kernel shape: 512 or 256 threads of the three-stage kernel, or 16 (two-stage; P = 128, 256, 2D 512)."""
        return _check(self._lib.cisor_set_cols_cta(self._ctx, int(nt)))

    def solve_iterations(self, adjoint=False):
        """Per-transmitter iterations of the last forward (or adjoint) solve, as a numpy array."""
        cnt = c_int()
        _check(self._lib.cisor_solve_iterations(self._ctx, 1 if adjoint else 0, None, ctypes.byref(cnt)))
        out = np.zeros(cnt.value, dtype=np.int32)
        _check(self._lib.cisor_solve_iterations(self._ctx, 1 if adjoint else 0,
                                                out.ctypes.data_as(POINTER(c_int)), ctypes.byref(cnt)))
        return out

    def close(self):
        if getattr(self, "_ctx", None) and getattr(self, "_owned", True):
            self._lib.cisor_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----- tables
    def green_spectrum(self, out):
        return _check(self._lib.cisor_green_spectrum(self._ctx, ptr(out, self.P ** self.dim)))

    def sensing_matrix(self, out):
        return _check(self._lib.cisor_sensing_matrix(self._ctx, ptr(out, self.M * self.Nf)))

    def incident(self, out):
        return _check(self._lib.cisor_incident(self._ctx, ptr(out, self.T * self.Nf)))

    # ----- operators
    def apply_A(self, f, x, y, adjoint=False):
        nvec = (x.numel() if hasattr(x, "numel") else x.size) // self.Nf
        return _check(self._lib.cisor_apply_A(self._ctx, ptr(f, self.N), ptr(x, nvec * self.Nf),
                                              ptr(y, nvec * self.Nf), 1 if adjoint else 0, nvec))

    def sense(self, f, u, Z):
        return _check(self._lib.cisor_sense(self._ctx, ptr(f, self.N), ptr(u, self.T * self.Nf),
                                            ptr(Z, self.T * self.M)))

    def sense_adjoint(self, f, w, z=None, b=None):
        return _check(self._lib.cisor_sense_adjoint(self._ctx, ptr(f, self.N), ptr(w, self.T * self.M),
                                                    ptr(z, self.T * self.Nf), ptr(b, self.T * self.Nf)))

    # ----- solves and gradient
    def forward(self, f, u_in=None, x0=None, u_out=None, y_out=None, tol=1e-4, max_iter=2000, x0_mode=0,
                check=True):
        opts = SolveOpts(tol, max_iter, x0_mode)
        info = SolveInfo()
        st = self._lib.cisor_forward(self._ctx, ptr(f, self.N), ptr(u_in, self.T * self.Nf),
                                     ptr(x0, self.T * self.Nf), ptr(u_out, self.T * self.Nf),
                                     ptr(y_out, self.T * self.M), ctypes.byref(opts), ctypes.byref(info))
        _check(st, () if check else (ERR_NOT_CONVERGED, ERR_BREAKDOWN))
        return st, info

    def grad(self, f, y, grad_out, tol=1e-4, max_iter=2000, x0_mode=0, check=True):
        opts = SolveOpts(tol, max_iter, x0_mode)
        info = SolveInfo()
        D = c_double()
        st = self._lib.cisor_grad(self._ctx, ptr(f, self.N), ptr(y, self.T * self.M), ptr(grad_out, self.N),
                                  ctypes.byref(D), ctypes.byref(opts), ctypes.byref(info))
        _check(st, () if check else (ERR_NOT_CONVERGED, ERR_BREAKDOWN))
        return D.value, st, info

    def data_term(self, f, y, tol=1e-4, max_iter=2000, x0_mode=0, check=True):
        """Forward half of grad: D, with the fields kept in the context for data_backward."""
        opts = SolveOpts(tol, max_iter, x0_mode)
        info = SolveInfo()
        D = c_double()
        st = self._lib.cisor_data_term(self._ctx, ptr(f, self.N), ptr(y, self.T * self.M), ctypes.byref(D),
                                       ctypes.byref(opts), ctypes.byref(info))
        _check(st, () if check else (ERR_NOT_CONVERGED, ERR_BREAKDOWN))
        return D.value, st, info

    def data_backward(self, grad_out, tol=1e-4, max_iter=2000, x0_mode=0, check=True):
        """Backward half of grad: adjoint solve and gradient assembly (after data_term)."""
        opts = SolveOpts(tol, max_iter, x0_mode)
        info = SolveInfo()
        st = self._lib.cisor_data_backward(self._ctx, ptr(grad_out, self.N), ctypes.byref(opts), ctypes.byref(info))
        _check(st, () if check else (ERR_NOT_CONVERGED, ERR_BREAKDOWN))
        return st, info

    def tv_prox(self, z, x, gamma_tau, iters, lo=0.0, hi=2.0, lo_im=0.0, hi_im=0.5, aniso=False):
        fn = self._lib.cisor_tv_prox_aniso if aniso else self._lib.cisor_tv_prox
        return _check(fn(self._ctx, ptr(z, self.N), ptr(x, self.N), float(gamma_tau), int(iters), float(lo),
                         float(hi), float(lo_im), float(hi_im)))

    def new_state(self, f, s, alpha, gamma, tau, tv_iters, lo=0.0, hi=2.0, lo_im=0.0, hi_im=0.5, tv_kind=0):
        """Relaxed-FISTA state over caller-owned f and s arrays (t = 1, k = 1);
        tv_kind 1 selects the anisotropic TV prox."""
        st = FistaState(ptr(f, self.N), ptr(s, self.N), 1.0, 1, alpha, gamma, tau, tv_iters, lo, hi, lo_im, hi_im,
                        0.0, int(tv_kind))
        st._keep = (f, s)
        return st

    def launch_count(self):
        v = c_longlong()
        _check(self._lib.cisor_launch_count(self._ctx, ctypes.byref(v)))
        return v.value

    def time_matvec(self, f, adjoint=False, reps=20):
        ms = c_double()
        _check(self._lib.cisor_time_matvec(self._ctx, ptr(f, self.N), 1 if adjoint else 0, int(reps),
                                           ctypes.byref(ms)))
        return ms.value

    def step(self, state, y, tol=1e-4, max_iter=2000, x0_mode=2, check=True):
        opts = SolveOpts(tol, max_iter, x0_mode)
        info = SolveInfo()
        st = self._lib.cisor_step(self._ctx, ctypes.byref(state), ptr(y, self.T * self.M), ctypes.byref(opts),
                                  ctypes.byref(info))
        _check(st, () if check else (ERR_NOT_CONVERGED, ERR_BREAKDOWN))
        return st, info


    def step_update(self, state, grad, D):
        """The prox and momentum half of step() from a gradient summed over all transmitters
        (e.g. over the contexts of a transmitter split)."""
        return _check(self._lib.cisor_step_update(self._ctx, ctypes.byref(state), ptr(grad, self.N), float(D)))


def _geometry(g, keep):
    dim = int(g.get("dim", 2))
    kind = 1 if g.get("tx_kind", 0) in (1, "point") else 0
    vec = 1 if g.get("vectorial") else 0
    per_tx = (6,) if vec else ((dim,) if kind == 1 else ((3,) if dim == 3 else ()))
    ang = np.ascontiguousarray(g["tx_angles"], dtype=np.float64).reshape((-1,) + per_tx)
    rx = np.ascontiguousarray(g["rx_pos"], dtype=np.float64).reshape(-1, dim)
    keep += [ang, rx]
    return Geometry(dim, int(g["n"]), float(g["delta"]), float(g.get("wavelength", 1.0)), float(g.get("eps_b", 1.0)),
                    len(ang), ang.ctypes.data_as(POINTER(c_double)), len(rx), rx.ctypes.data_as(POINTER(c_double)),
                    1 if g.get("complex_f") else 0, int(g.get("pad", 0)), kind, vec)


class Batch:
    """Problems of uneven size solved together (cisor_batch_*): geoms is a list of dicts
    with n, delta, tx_angles, rx_pos and optionally wavelength, eps_b, complex_f, pad."""

    def __init__(self, geoms, autotune=True, stream=None):
        lib = load()
        self._lib = lib
        self._keep = []
        arr = (Geometry * len(geoms))(*[_geometry(g, self._keep) for g in geoms])
        self._b = c_void_p()
        self.stream = _current_stream() if stream is None else stream
        _check(lib.cisor_batch_create(ctypes.byref(self._b), arr, len(geoms), self.stream, 1 if autotune else 0))
        self.problems = []
        for i, g in enumerate(geoms):
            h = c_void_p()
            _check(lib.cisor_batch_context(self._b, i, ctypes.byref(h)))
            self.problems.append(Cisor(_handle=h, stream=self.stream, complex_f=g.get("complex_f", False),
                                       dim=g.get("dim", 2), vectorial=bool(g.get("vectorial", False))))

    def close(self):
        if getattr(self, "_b", None):
            self._lib.cisor_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_solve_loop(self, device_loop=True):
        """1: each solve of all problems in one graph launch (device-side loop); 0: host-driven chunks."""
        return _check(self._lib.cisor_batch_set_solve_loop(self._b, 1 if device_loop else 0))

    def _ptrs(self, arrs, counts):
        return (c_void_p * len(arrs))(*[ptr(a, c) if a is not None else None for a, c in zip(arrs, counts)])

    def forward(self, f, u_out=None, tol=1e-4, max_iter=2000, x0_mode=0, check=True):
        ps = self.problems
        opts = SolveOpts(tol, max_iter, x0_mode)
        infos = (SolveInfo * len(ps))()
        fp = self._ptrs(f, [p.N for p in ps])
        up = self._ptrs(u_out, [p.T * p.Nf for p in ps]) if u_out is not None else None
        st = self._lib.cisor_batch_forward(self._b, fp, up, ctypes.byref(opts), infos)
        _check(st, () if check else (ERR_NOT_CONVERGED, ERR_BREAKDOWN))
        return st, list(infos)

    def grad(self, f, y, grad_out, tol=1e-4, max_iter=2000, x0_mode=0, check=True):
        ps = self.problems
        opts = SolveOpts(tol, max_iter, x0_mode)
        infos = (SolveInfo * len(ps))()
        D = (c_double * len(ps))()
        st = self._lib.cisor_batch_grad(self._b, self._ptrs(f, [p.N for p in ps]),
                                        self._ptrs(y, [p.T * p.M for p in ps]),
                                        self._ptrs(grad_out, [p.N for p in ps]), D, ctypes.byref(opts), infos)
        _check(st, () if check else (ERR_NOT_CONVERGED, ERR_BREAKDOWN))
        return list(D), st, list(infos)


FNO_N = 128


class FNO:
    """Learned warm start (cisor_fno_*): a 128 x 128 Fourier neural operator."""

    def __init__(self, max_batch=32, seed=0, stream=None):
        lib = load()
        self._lib = lib
        self._h = c_void_p()
        self.stream = _current_stream() if stream is None else stream
        _check(lib.cisor_fno_create(ctypes.byref(self._h), int(max_batch), int(seed), self.stream))
        cnt = c_longlong()
        _check(lib.cisor_fno_num_params(self._h, ctypes.byref(cnt)))
        self.num_params = cnt.value
        self.max_batch = max_batch

    def close(self):
        if getattr(self, "_h", None):
            self._lib.cisor_fno_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self, out, as_used=True):
        return _check(self._lib.cisor_fno_get_params(self._h, ptr(out, self.num_params, "float32"), int(as_used)))

    def set_params(self, arr):
        return _check(self._lib.cisor_fno_set_params(self._h, ptr(arr, self.num_params, "float32")))

    def forward(self, f, u_in, out, f_per_sample=True):
        B = (u_in.numel() if hasattr(u_in, "numel") else u_in.size) // (FNO_N * FNO_N)
        nf = B if f_per_sample else 1
        return _check(self._lib.cisor_fno_forward(self._h, ptr(f, nf * FNO_N * FNO_N), int(f_per_sample),
                                                  ptr(u_in, B * FNO_N * FNO_N), B, ptr(out, B * FNO_N * FNO_N)))

    def loss_grad(self, f, u_in, target, grad_out=None, f_per_sample=True):
        B = (u_in.numel() if hasattr(u_in, "numel") else u_in.size) // (FNO_N * FNO_N)
        nf = B if f_per_sample else 1
        loss = c_double()
        _check(self._lib.cisor_fno_loss_grad(self._h, ptr(f, nf * FNO_N * FNO_N), int(f_per_sample),
                                             ptr(u_in, B * FNO_N * FNO_N), ptr(target, B * FNO_N * FNO_N), B,
                                             ctypes.byref(loss),
                                             ptr(grad_out, self.num_params, "float32") if grad_out is not None
                                             else None))
        return loss.value

    def train_step(self, f, u_in, target, lr, f_per_sample=True):
        B = (u_in.numel() if hasattr(u_in, "numel") else u_in.size) // (FNO_N * FNO_N)
        nf = B if f_per_sample else 1
        loss = c_double()
        _check(self._lib.cisor_fno_train_step(self._h, ptr(f, nf * FNO_N * FNO_N), int(f_per_sample),
                                              ptr(u_in, B * FNO_N * FNO_N), ptr(target, B * FNO_N * FNO_N), B,
                                              float(lr), ctypes.byref(loss)))
        return loss.value

    def warm_start(self, ctx, f, x0_out):
        return _check(self._lib.cisor_fno_warm_start(self._h, ctx._ctx, ptr(f, ctx.N), ptr(x0_out, ctx.T * ctx.N)))


def fno_param_dict(flat, C=32, m=16, L=4, H=128):
    """Split a flat parameter array into named arrays (FP64, complex spectral weights)."""
    flat = np.asarray(flat, dtype=np.float64)
    out, o = {}, 0

    def take(name, shape, cplx=False):
        nonlocal o
        cnt = int(np.prod(shape)) * (2 if cplx else 1)
        a = flat[o:o + cnt]
        o += cnt
        out[name] = (a[0::2] + 1j * a[1::2]).reshape(shape) if cplx else a.reshape(shape)

    take("W0", (C, 8))
    take("b0", (C,))
    for l in range(L):
        take(f"R{l}", (2 * m, m, C, C), True)
        take(f"W{l + 1}", (C, C))
        take(f"b{l + 1}", (C,))
    take("P1", (H, C))
    take("c1", (H,))
    take("P2", (2, H))
    take("c2", (2,))
    assert o == flat.size
    return out
