"""FP64 CPU oracle of the parareal + splitting method (arXiv 2502.08370).

TEST INFRASTRUCTURE ONLY: the slow, plain reference that the CUDA library is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It
shares no code with the CUDA path and never imports the package.

The arithmetic lives in ``ps_oracle.c`` (plain C, FP64, OpenMP over lines),
built by :func:`build` with gcc; this module only marshals numpy arrays.  The
closed forms of the paper's analysis (stability functions, convergence factor)
are in :mod:`oracle.analysis`.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ps_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libps_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ps_oracle.c into oracle/_build/libps_oracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("a", C.POINTER(C.c_double)), ("c", C.c_double),
        ("src", C.POINTER(C.c_double)), ("src_t", C.POINTER(C.c_double)),
        ("src_t_len", C.c_int), ("split", C.c_int),
        ("boxes_x", C.c_int), ("boxes_y", C.c_int), ("overlap", C.c_double),
        ("d12", C.POINTER(C.c_double)), ("src2", C.POINTER(C.c_double)), ("src2_t", C.POINTER(C.c_double)),
        ("src2_t_len", C.c_int),
    ]


_D = C.POINTER(C.c_double)


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER(_Problem)
            sig = {
                "or_num_substeps": (C.c_int, [P]),
                "or_phi1d": (C.c_double, [C.c_int, C.c_int, C.c_double, C.c_double]),
                "or_rho": (C.c_double, [P, C.c_int, C.c_double, C.c_double]),
                "or_box_range": (C.c_int, [P, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
                "or_apply_A": (None, [P, C.c_int, _D, _D]),
                "or_substep_solve": (C.c_int, [P, C.c_int, C.c_double, _D]),
                "or_fie_step": (C.c_int, [P, C.c_double, C.c_int, C.c_int, _D]),
                "or_propagate": (C.c_int, [P, C.c_double, C.c_int, C.c_int, C.c_int, _D]),
                "or_fine_sequential": (C.c_int, [P, C.c_double, C.c_int, C.c_int, _D, _D]),
                "or_coarse_sequential": (C.c_int, [P, C.c_double, C.c_int, C.c_int, C.c_int, _D, _D]),
                "or_parareal": (C.c_int, [P, C.c_double, C.c_int, C.c_int, C.c_int, _D, C.c_double,
                                          C.c_int, _D, _D, C.POINTER(C.c_int)]),
                "or_parareal2": (C.c_int, [P, P, C.c_double, C.c_int, C.c_int, C.c_int, _D, C.c_double,
                                           C.c_int, _D, _D, C.POINTER(C.c_int)]),
                "or_parareal_fine": (C.c_int, [P, P, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, _D,
                                               C.c_double, C.c_int, _D, _D, C.POINTER(C.c_int)]),
                "or_dr_step": (C.c_int, [P, C.c_double, C.c_int, _D]),
                "or_propagate_dr": (C.c_int, [P, C.c_double, C.c_int, C.c_int, C.c_int, _D]),
                "or_fine_sequential_dr": (C.c_int, [P, C.c_double, C.c_int, C.c_int, _D, _D]),
                "or_adjoint": (C.c_int, [P, C.c_double, C.c_int, C.c_int, _D, _D, _D, _D, _D]),
                "or_num_threads": (C.c_int, []),
                "or_set_num_threads": (None, [C.c_int]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _ptr(x):
    return None if x is None else x.ctypes.data_as(_D)


def _f64(x):
    return None if x is None else np.ascontiguousarray(x, dtype=np.float64)


class Problem:
    """Model problem of Sec. 2.1 with D = a(x) I, or in 2-D the full tensor
    D = [[a, d12], [d12, a]] of Sec. 5.2; homogeneous Dirichlet data.

    n      : interior nodes per direction, (nx, ny) or (nx, ny, nz); h_i = 1/(n_i+1)
    a      : nodal diffusion on the (n+2)^d grid incl. boundary (x fastest), or None (a = 1)
    c      : reaction coefficient, split as c/M (dimensional) or rho_j c (DD)
    src    : spatial source on interior nodes, or None (f = 0)
    src_t  : time factor of the source at fine times t_j = j*dt (f = src(x) src_t(t)), or None
    split  : "dim" (x/y/z splitting) or "dd" (partition-of-unity splitting, 2-D)
    boxes  : DD boxes per direction (bx, by); overlap: DD overlap width beta
    d12    : off-diagonal diffusion, nodal on the (n+2)^2 grid or a scalar; 2-D DD only
             (dimensional splitting cannot take the mixed derivatives, Sec. 2.1)
    src2, src2_t : a second separable source term, f = src src_t + src2 src2_t
    """

    def __init__(self, n, a=None, c=0.0, src=None, src_t=None, split="dim", boxes=(1, 1), overlap=0.0,
                 d12=None, src2=None, src2_t=None):
        n = tuple(int(v) for v in n)
        assert len(n) in (2, 3)
        self.n = n
        self.dim = len(n)
        self.shape = tuple(reversed(n))  # numpy shape, x fastest
        self.a = _f64(a)
        if self.a is not None:
            assert self.a.size == int(np.prod([v + 2 for v in n]))
        self.c = float(c)
        self.src = _f64(src)
        self.src_t = _f64(src_t)
        self.split = split
        self.boxes = tuple(boxes)
        self.overlap = float(overlap)
        s = _Problem()
        s.dim = self.dim
        s.nx, s.ny = n[0], n[1]
        s.nz = n[2] if self.dim == 3 else 1
        s.a = _ptr(self.a)
        s.c = self.c
        s.src = _ptr(self.src)
        s.src_t = _ptr(self.src_t)
        s.src_t_len = 0 if self.src_t is None else int(self.src_t.size)
        s.split = 0 if split == "dim" else 1
        s.boxes_x, s.boxes_y = int(boxes[0]), int(boxes[1])
        s.overlap = self.overlap
        if d12 is not None:
            if self.dim != 2 or split != "dd":
                raise ValueError("the off-diagonal diffusion d12 needs the 2-D DD splitting")
            d12 = np.broadcast_to(np.asarray(d12, dtype=np.float64), (n[1] + 2, n[0] + 2))
        self.d12 = _f64(d12)
        self.src2 = _f64(src2)
        self.src2_t = _f64(src2_t)
        s.d12 = _ptr(self.d12)
        s.src2 = _ptr(self.src2)
        s.src2_t = _ptr(self.src2_t)
        s.src2_t_len = 0 if self.src2_t is None else int(self.src2_t.size)
        self._s = s

    @property
    def size(self):
        return int(np.prod(self.n))

    @property
    def M(self):
        return _lib_handle().or_num_substeps(C.byref(self._s))

    def _state(self, u):
        u = np.array(u, dtype=np.float64, copy=True).reshape(-1)
        assert u.size == self.size
        return u


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def phi1d(b, B, w, x):
    return _lib_handle().or_phi1d(b, B, w, x)


def rho(p: Problem, colour, x, y):
    return _lib_handle().or_rho(C.byref(p._s), colour, x, y)


def box_range(p: Problem, d, b):
    lo, hi = C.c_int(), C.c_int()
    ok = _lib_handle().or_box_range(C.byref(p._s), d, b, C.byref(lo), C.byref(hi))
    return (lo.value, hi.value) if ok else None


def apply_A(p: Problem, m, u):
    """(A_m u) of the semidiscrete problem (eq. semidisc_prob), substep m."""
    u = p._state(u)
    out = np.empty_like(u)
    _lib_handle().or_apply_A(C.byref(p._s), m, _ptr(u), _ptr(out))
    return out.reshape(p.shape)


def substep_solve(p: Problem, m, tau, b):
    """x with (I - tau A_m) x = b (one internal stage of eq. FIE_method)."""
    x = p._state(b)
    _check(_lib_handle().or_substep_solve(C.byref(p._s), m, tau, _ptr(x)), "substep_solve")
    return x.reshape(p.shape)


def fie_step(p: Problem, tau, u, t_end=0, reversed_order=False):
    """One FIE step (eq. FIE_method) with the source at fine time index t_end."""
    x = p._state(u)
    _check(_lib_handle().or_fie_step(C.byref(p._s), tau, t_end, int(reversed_order), _ptr(x)), "fie_step")
    return x.reshape(p.shape)


def propagate(p: Problem, tau, nsteps, u, t0=0, tstride=1):
    x = p._state(u)
    _check(_lib_handle().or_propagate(C.byref(p._s), tau, nsteps, t0, tstride, _ptr(x)), "propagate")
    return x.reshape(p.shape)


def fine_sequential(p: Problem, T, N, s, u0):
    """Sequential fine solution at the coarse times T_n, n = 0..N (shape (N+1,)+grid)."""
    u0 = p._state(u0)
    U = np.empty((N + 1) * p.size)
    _check(_lib_handle().or_fine_sequential(C.byref(p._s), T, N, s, _ptr(u0), _ptr(U)), "fine_sequential")
    return U.reshape((N + 1,) + p.shape)


def coarse_sequential(p: Problem, T, N, g, s, u0):
    u0 = p._state(u0)
    U = np.empty((N + 1) * p.size)
    _check(_lib_handle().or_coarse_sequential(C.byref(p._s), T, N, g, s, _ptr(u0), _ptr(U)), "coarse_sequential")
    return U.reshape((N + 1,) + p.shape)


def dr_step(p: Problem, tau, u, t_end=0):
    """One Douglas-Rachford step (eq. DR_method) with the source at fine time index t_end."""
    x = p._state(u)
    _check(_lib_handle().or_dr_step(C.byref(p._s), tau, t_end, _ptr(x)), "dr_step")
    return x.reshape(p.shape)


def propagate_dr(p: Problem, tau, nsteps, u, t0=0, tstride=1):
    x = p._state(u)
    _check(_lib_handle().or_propagate_dr(C.byref(p._s), tau, nsteps, t0, tstride, _ptr(x)), "propagate_dr")
    return x.reshape(p.shape)


def fine_sequential_dr(p: Problem, T, N, s, u0):
    """Sequential solution by s DR steps per slice, at the coarse times T_n, n = 0..N."""
    u0 = p._state(u0)
    U = np.empty((N + 1) * p.size)
    _check(_lib_handle().or_fine_sequential_dr(C.byref(p._s), T, N, s, _ptr(u0), _ptr(U)), "fine_sequential_dr")
    return U.reshape((N + 1,) + p.shape)


def parareal(p: Problem, T, N, g, s, u0, tol, max_iter=None, pG: Problem = None, fine="fie"):
    """Parareal/FIE-FIE (Sec. 3, Sec. 4.1), or Parareal/FIE-DR with fine="dr" (Sec. 4.2: the
    fine propagator takes s DR steps).  Returns (U, history, iters):
    U[n] = U_n^k at the final k, history[k-1] = max_n ||U_n^k - U_n^{k-1}||_inf.
    pG, when given, is the problem whose splitting the coarse propagator uses
    (Sec. 5.1 uses different DD decompositions for G and F)."""
    if fine not in ("fie", "dr"):
        raise ValueError("fine must be 'fie' or 'dr'")
    u0 = p._state(u0)
    if max_iter is None:
        max_iter = N
    U = np.empty((N + 1) * p.size)
    hist = np.zeros(max(N, 1))
    it = C.c_int(0)
    pg = p if pG is None else pG
    _check(_lib_handle().or_parareal_fine(C.byref(pg._s), C.byref(p._s), 0 if fine == "fie" else 1, T, N, g, s,
                                          _ptr(u0), tol, max_iter, _ptr(U), _ptr(hist), C.byref(it)), "parareal")
    k = it.value
    return U.reshape((N + 1,) + p.shape), hist[:k].copy(), k


def adjoint(p: Problem, T, N, s, u0, target):
    """J = 1/2 ||U_N - target||^2 of the sequential fine solution, dJ/du0, dJ/da (nodal)."""
    u0 = p._state(u0)
    tg = p._state(target)
    gu = np.empty(p.size)
    ga = np.empty(int(np.prod([v + 2 for v in p.n])))
    J = np.zeros(1)
    _check(_lib_handle().or_adjoint(C.byref(p._s), T, N, s, _ptr(u0), _ptr(tg), _ptr(J), _ptr(gu), _ptr(ga)),
           "adjoint")
    return float(J[0]), gu.reshape(p.shape), ga.reshape(tuple(v + 2 for v in reversed(p.n)))


def num_threads():
    return _lib_handle().or_num_threads()


def set_num_threads(n):
    _lib_handle().or_set_num_threads(int(n))
