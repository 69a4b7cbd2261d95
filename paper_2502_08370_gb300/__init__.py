"""GB300 parareal + splitting solver (arXiv 2502.08370) -- Python binding.

The numerical work runs in the CUDA library ``_lib/libps.so`` (C ABI declared
in ``include/ps.h``); this module only loads it and marshals arguments.  Device
arrays are torch tensors (float64, CUDA, contiguous); torch provides the
memory and the streams.  There is no CPU fallback: every call fails loudly
when the library or a CUDA device is missing.

Function names follow the C ABI: ``ps_grid_create`` etc. are exposed as raw
calls on :func:`lib`, and :class:`Grid`, :class:`Operator`, :class:`Splitting`
and :class:`Problem` own the corresponding handles.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libps.so")

PS_OK = 0
ERRORS = {1: "PS_ERR_INVALID", 2: "PS_ERR_CUDA", 3: "PS_ERR_OOM", 4: "PS_ERR_NONFINITE",
          5: "PS_ERR_DEVICE_TIMEOUT", 6: "PS_ERR_UNSUPPORTED"}
PS_SPLIT_DIM, PS_SPLIT_DD = 0, 1
PS_PREC_FP64, PS_PREC_MIXED = 0, 1
PS_VERSION = 103  # the header's PS_VERSION this binding marshals for
PS_SCHED_AUTO, PS_SCHED_THOMAS, PS_SCHED_PCR, PS_SCHED_HYBRID = 0, 1, 2, 3
PS_COARSE_FP64, PS_COARSE_DELTA32 = 0, 1
PS_FINE_FIE, PS_FINE_DR = 0, 1
PS_COARSE_SWEEP_AUTO, PS_COARSE_SWEEP_STAGED, PS_COARSE_SWEEP_STREAMED = 0, 1, 2
PS_NOALLOC_MAX_UNKNOWNS = 1 << 20

_lock = threading.Lock()
_lib = None


class PsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class _DD(C.Structure):
    _fields_ = [("boxes", C.c_int * 2), ("overlap", C.c_double)]


class _OpDesc(C.Structure):
    _fields_ = [("a_nodal_dev", C.c_void_p), ("d12_nodal_dev", C.c_void_p), ("c", C.c_double),
                ("src_dev", C.c_void_p), ("src_t_host", C.c_void_p), ("src_t_len", C.c_int),
                ("src2_dev", C.c_void_p), ("src2_t_host", C.c_void_p), ("src2_t_len", C.c_int)]


class _Params(C.Structure):
    _fields_ = [("precision", C.c_int), ("schedule", C.c_int), ("timing", C.c_int), ("dd_slices_per_block", C.c_int),
                ("tile_positions", C.c_int), ("tile_pipeline", C.c_int), ("tile_slots", C.c_int),
                ("tol_mode", C.c_int), ("coarse", C.c_int), ("tile_lines_per_thread", C.c_int),
                ("fine_method", C.c_int), ("overlap_phases", C.c_int), ("coarse_sweep", C.c_int)]


class _Stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("unknown_updates", C.c_double), ("ms_total", C.c_double),
                ("ms_fine", C.c_double), ("ms_coarse", C.c_double), ("kernel_launches", C.c_int)]


class _TuneEntry(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("ms", C.c_double), ("chosen", C.c_int)]


class _KTime(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int), ("ms", C.c_double), ("bytes", C.c_double),
                ("flops", C.c_double)]


_VP = C.c_void_p
_I = C.c_int
_D = C.c_double
_U = C.c_uint64
_IP = C.POINTER(C.c_int)

# name -> argtypes (every entry point returns int status unless listed in _RESTYPE)
SIGNATURES = {
    "ps_last_error": [],
    "ps_version": [],
    "ps_grid_create": [_I, C.POINTER(C.c_int * 3), C.POINTER(_VP)],
    "ps_grid_destroy": [_VP],
    "ps_operator_create": [_VP, _VP, _D, _VP, _VP, _I, _U, C.POINTER(_VP)],
    "ps_operator_destroy": [_VP],
    "ps_operator_create_ex": [_VP, C.POINTER(_OpDesc), _U, C.POINTER(_VP)],
    "ps_splitting_create": [_VP, _I, C.POINTER(_DD), C.POINTER(_VP)],
    "ps_splitting_destroy": [_VP],
    "ps_problem_create": [_VP, _VP, _D, _I, _I, _I, C.POINTER(_Params), _U, C.POINTER(_VP)],
    "ps_problem_destroy": [_VP],
    "ps_run_parareal": [_VP, _VP, _D, _I, _U, _IP],
    "ps_run_parareal_host": [_VP, _VP, _VP, _D, _I, _U, _IP],
    "ps_get_state": [_VP, _I, _VP, _U],
    "ps_get_history": [_VP, _VP, _I, _IP],
    "ps_set_state": [_VP, _I, _VP, _U],
    "ps_checkpoint_bytes": [_VP, C.POINTER(C.c_size_t)],
    "ps_checkpoint_save": [_VP, _VP, C.c_size_t, _U],
    "ps_checkpoint_load": [_VP, _VP, C.c_size_t, _U],
    "ps_resume_parareal": [_VP, _D, _I, _U, _IP],
    "ps_run_fine_sequential": [_VP, _VP, _VP, _U],
    "ps_run_coarse_sequential": [_VP, _VP, _VP, _U],
    "ps_run_coarse_sequential_noalloc": [_VP, _VP, _VP, _U],
    "ps_substep_solve": [_VP, _I, _I, _VP, _U],
    "ps_propagate": [_VP, _I, _I, _I, _I, _VP, _U],
    "ps_problem_stats": [_VP, C.POINTER(_Stats)],
    "ps_problem_update_coefficients": [_VP, _VP, _U],
    "ps_batch_create": [C.POINTER(_VP), _I, _U, C.POINTER(_VP)],
    "ps_batch_run": [_VP, C.POINTER(_VP), _D, _I, _U, _IP],
    "ps_batch_stats": [_VP, C.POINTER(_Stats)],
    "ps_batch_last_error": [],
    "ps_batch_destroy": [_VP],
    "ps_autotune": [_VP, _I, _U, _IP],
    "ps_copy_schedule": [_VP, _VP],
    "ps_autotune_record": [_VP, C.POINTER(_TuneEntry), _I, _IP],
    "ps_adjoint_vjp": [_VP, _VP, _D, _I, _VP, _VP, _U, _IP],
    "ps_adjoint": [_VP, _VP, _D, _I, _VP, _VP, _U, C.POINTER(C.c_double), _IP],
    "ps_problem_set_slices": [_VP, _I, _I, _I, _U],
    "ps_batch_add": [_VP, _VP, _U],
    "ps_batch_get_state": [_VP, _I, _I, _VP, _U],
    "ps_problem_kernel_times": [_VP, C.POINTER(_KTime), _I, _IP],
    "ps_selftest_wait_timeout": [_I, _U],
}
_RESTYPE = {"ps_last_error": C.c_char_p, "ps_batch_last_error": C.c_char_p}


def lib():
    """Load libps.so (built by ``build.build()``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run paper_2502_08370_gb300.build.build())")
            h = C.CDLL(LIB_PATH)
            for name, args in SIGNATURES.items():
                f = getattr(h, name)
                f.argtypes = args
                f.restype = _RESTYPE.get(name, C.c_int)
            if h.ps_version() != PS_VERSION:
                raise RuntimeError(f"{LIB_PATH} has ABI version {h.ps_version()}, this binding expects "
                                   f"{PS_VERSION}: rebuild it (paper_2502_08370_gb300.build.build())")
            _lib = h
    return _lib


def check(rc):
    if rc != PS_OK:
        raise PsError(rc, lib().ps_last_error().decode())


def _dev_ptr(t, n=None):
    """Pointer of a contiguous float64 CUDA tensor (optionally checking its element count)."""
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"expected {n} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def selftest_wait_timeout(limit_us=20000, stream=None):
    """Run the device-side bounded wait against a barrier nothing arrives at; returns the
    status code (PS_ERR_DEVICE_TIMEOUT = 5 is the expected outcome)."""
    return lib().ps_selftest_wait_timeout(int(limit_us), _stream(stream))


class Grid:
    def __init__(self, n):
        n = tuple(int(v) for v in n)
        self.dim = len(n)
        self.n = n
        self.nt = 1
        for v in n:
            self.nt *= v
        arr = (C.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
        h = _VP()
        check(lib().ps_grid_create(self.dim, C.byref(arr), C.byref(h)))
        self._h = h

    @property
    def shape(self):
        return tuple(reversed(self.n))

    @property
    def nodal_size(self):
        s = 1
        for v in self.n:
            s *= v + 2
        return s

    def __del__(self):
        if getattr(self, "_h", None):
            lib().ps_grid_destroy(self._h)
            self._h = None


class Operator:
    """u_t = div(D grad u) - c u + src(x) src_t(t) + src2(x) src2_t(t); D = a I with a nodal incl.
    boundary (None: a = 1), or the full 2-D tensor [[a, d12], [d12, a]] when d12 (nodal) is given
    (DD splitting only, Sec. 5.2)."""

    def __init__(self, grid: Grid, a=None, c=0.0, src=None, src_t=None, d12=None, src2=None, src2_t=None,
                 stream=None):
        import numpy as np
        self.grid = grid
        st = None if src_t is None else np.ascontiguousarray(src_t, dtype=np.float64)
        st2 = None if src2_t is None else np.ascontiguousarray(src2_t, dtype=np.float64)
        self._host = (st, st2)  # the library copies them during the call
        h = _VP()
        if d12 is None and src2 is None:
            check(lib().ps_operator_create(grid._h, _dev_ptr(a, grid.nodal_size), float(c), _dev_ptr(src, grid.nt),
                                           None if st is None else st.ctypes.data_as(_VP),
                                           0 if st is None else st.size, _stream(stream), C.byref(h)))
        else:
            d = _OpDesc(_dev_ptr(a, grid.nodal_size), _dev_ptr(d12, grid.nodal_size), float(c), _dev_ptr(src, grid.nt),
                        None if st is None else st.ctypes.data_as(_VP), 0 if st is None else st.size,
                        _dev_ptr(src2, grid.nt), None if st2 is None else st2.ctypes.data_as(_VP),
                        0 if st2 is None else st2.size)
            check(lib().ps_operator_create_ex(grid._h, C.byref(d), _stream(stream), C.byref(h)))
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            lib().ps_operator_destroy(self._h)
            self._h = None


class Splitting:
    def __init__(self, op: Operator, kind="dim", boxes=(1, 1), overlap=0.0):
        self.op = op
        dd = _DD((C.c_int * 2)(*boxes), float(overlap))
        h = _VP()
        check(lib().ps_splitting_create(op._h, PS_SPLIT_DIM if kind == "dim" else PS_SPLIT_DD, C.byref(dd),
                                        C.byref(h)))
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            lib().ps_splitting_destroy(self._h)
            self._h = None


class Problem:
    """Parareal problem: G = g FIE steps of T/(N g), F = s FIE steps of T/(N s) (Sec. 3)."""

    def __init__(self, fine: Splitting, T, N, g, s, coarse: Splitting = None, precision="fp64",
                 schedule=PS_SCHED_AUTO, timing=False, dd_slices_per_block=0, tile_positions=0, tile_pipeline=0,
                 tile_slots=0, tol_mode=0, coarse_mode="fp64", tile_lines_per_thread=0, fine_method="fie",
                 coarse_sweep="auto", overlap_phases=False, stream=None):
        self.fine, self.coarse = fine, coarse
        self.grid = fine.op.grid
        self.N = int(N)
        if coarse_mode not in ("fp64", "delta32"):
            raise ValueError("coarse_mode must be 'fp64' or 'delta32'")
        if fine_method not in ("fie", "dr"):
            raise ValueError("fine_method must be 'fie' or 'dr'")
        prm = _Params(PS_PREC_FP64 if precision == "fp64" else PS_PREC_MIXED, int(schedule), int(timing),
                      int(dd_slices_per_block), int(tile_positions), int(tile_pipeline), int(tile_slots),
                      int(tol_mode), PS_COARSE_FP64 if coarse_mode == "fp64" else PS_COARSE_DELTA32,
                      int(tile_lines_per_thread), PS_FINE_FIE if fine_method == "fie" else PS_FINE_DR,
                      int(bool(overlap_phases)), {"auto": 0, "staged": 1, "streamed": 2}[coarse_sweep])
        h = _VP()
        check(lib().ps_problem_create(fine._h, None if coarse is None else coarse._h, float(T), int(N), int(g),
                                      int(s), C.byref(prm), _stream(stream), C.byref(h)))
        self._h = h

    def run(self, u0, tol, max_iter=0, stream=None):
        it = C.c_int(0)
        check(lib().ps_run_parareal(self._h, _dev_ptr(u0, self.grid.nt), float(tol), int(max_iter), _stream(stream),
                                    C.byref(it)))
        return it.value

    def run_host(self, u0_host, uN_host, tol, max_iter=0, stream=None):
        """u0_host/uN_host: contiguous float64 CPU tensors (pinned for async copies)."""
        it = C.c_int(0)
        check(lib().ps_run_parareal_host(self._h, C.c_void_p(u0_host.data_ptr()), C.c_void_p(uN_host.data_ptr()),
                                         float(tol), int(max_iter), _stream(stream), C.byref(it)))
        return it.value

    def state(self, n, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.grid.shape, dtype=torch.float64, device="cuda")
        check(lib().ps_get_state(self._h, int(n), _dev_ptr(out, self.grid.nt), _stream(stream)))
        return out

    def set_state(self, n, x, stream=None):
        check(lib().ps_set_state(self._h, int(n), _dev_ptr(x, self.grid.nt), _stream(stream)))

    def checkpoint(self, stream=None):
        """The current parareal iterate as bytes (k, history, U^k, coarse values)."""
        nb = C.c_size_t(0)
        check(lib().ps_checkpoint_bytes(self._h, C.byref(nb)))
        buf = C.create_string_buffer(nb.value)
        check(lib().ps_checkpoint_save(self._h, buf, nb, _stream(stream)))
        return buf.raw

    def load_checkpoint(self, data, stream=None):
        buf = C.create_string_buffer(bytes(data), len(data))
        check(lib().ps_checkpoint_load(self._h, buf, len(data), _stream(stream)))

    def resume(self, tol, max_iter=0, stream=None):
        it = C.c_int(0)
        check(lib().ps_resume_parareal(self._h, float(tol), int(max_iter), _stream(stream), C.byref(it)))
        return it.value

    def history(self):
        import numpy as np
        buf = np.zeros(max(self.N, 1))
        ln = C.c_int(0)
        check(lib().ps_get_history(self._h, buf.ctypes.data_as(_VP), buf.size, C.byref(ln)))
        return buf[:ln.value].copy()

    def fine_sequential(self, u0, stream=None):
        import torch
        out = torch.empty((self.N + 1,) + self.grid.shape, dtype=torch.float64, device="cuda")
        check(lib().ps_run_fine_sequential(self._h, _dev_ptr(u0, self.grid.nt), _dev_ptr(out), _stream(stream)))
        return out

    def coarse_sequential(self, u0, stream=None):
        import torch
        out = torch.empty((self.N + 1,) + self.grid.shape, dtype=torch.float64, device="cuda")
        check(lib().ps_run_coarse_sequential(self._h, _dev_ptr(u0, self.grid.nt), _dev_ptr(out), _stream(stream)))
        return out

    def coarse_sequential_noalloc(self, u0, out, stream=None):
        """Same result as coarse_sequential, computed without any device allocation inside the
        library (the working state lives in a fixed per-device array of
        PS_NOALLOC_MAX_UNKNOWNS doubles); the caller provides `out` ((N+1) states)."""
        check(lib().ps_run_coarse_sequential_noalloc(self._h, _dev_ptr(u0, self.grid.nt),
                                                     _dev_ptr(out, (self.N + 1) * self.grid.nt), _stream(stream)))
        return out

    def substep_solve(self, which, m, x, stream=None):
        check(lib().ps_substep_solve(self._h, int(which), int(m), _dev_ptr(x, self.grid.nt), _stream(stream)))
        return x

    def propagate(self, which, nsteps, x, t0=0, tstride=1, stream=None):
        check(lib().ps_propagate(self._h, int(which), int(nsteps), int(t0), int(tstride), _dev_ptr(x, self.grid.nt),
                                 _stream(stream)))
        return x

    def stats(self):
        s = _Stats()
        check(lib().ps_problem_stats(self._h, C.byref(s)))
        return dict(iterations=s.iterations, unknown_updates=s.unknown_updates, ms_total=s.ms_total,
                    ms_fine=s.ms_fine, ms_coarse=s.ms_coarse, kernel_launches=s.kernel_launches)

    def update_coefficients(self, a, stream=None):
        """Replace the nodal coefficient and rebuild the substep factors."""
        check(lib().ps_problem_update_coefficients(self._h, _dev_ptr(a, self.grid.nodal_size), _stream(stream)))

    def vjp(self, gN, tol, max_iter=0, want_a=True, stream=None):
        """(dL/du0, dL/da) for the upstream gradient gN = dL/dU_N of the last run."""
        import torch
        gu = torch.empty(self.grid.shape, dtype=torch.float64, device="cuda")
        ga = torch.empty(tuple(v + 2 for v in reversed(self.grid.n)), dtype=torch.float64, device="cuda") \
            if want_a else None
        it = C.c_int(0)
        check(lib().ps_adjoint_vjp(self._h, _dev_ptr(gN, self.grid.nt), float(tol), int(max_iter), _dev_ptr(gu),
                                   _dev_ptr(ga), _stream(stream), C.byref(it)))
        self.last_adjoint_iters = it.value
        return gu, ga

    def adjoint(self, u_target, tol, max_iter=0, want_a=True, stream=None):
        """(J, dJ/du0, dJ/da) for J = 1/2 ||U_N - u_target||^2 of the last run."""
        import torch
        gu = torch.empty(self.grid.shape, dtype=torch.float64, device="cuda")
        ga = torch.empty(tuple(v + 2 for v in reversed(self.grid.n)), dtype=torch.float64, device="cuda") \
            if want_a else None
        J = C.c_double(0.0)
        it = C.c_int(0)
        check(lib().ps_adjoint(self._h, _dev_ptr(u_target, self.grid.nt), float(tol), int(max_iter), _dev_ptr(gu),
                               _dev_ptr(ga), _stream(stream), C.byref(J), C.byref(it)))
        self.last_adjoint_iters = it.value
        return J.value, gu, ga

    def set_slices(self, N, g, s, stream=None):
        """New slice count and propagator step counts (rebuilds factors and slice states)."""
        check(lib().ps_problem_set_slices(self._h, int(N), int(g), int(s), _stream(stream)))
        self.N = int(N)

    def autotune(self, budget_ms=200, stream=None):
        """Time the fine-sweep schedules on this problem and keep the fastest (returns its code)."""
        ch = C.c_int(0)
        check(lib().ps_autotune(self._h, int(budget_ms), _stream(stream), C.byref(ch)))
        return ch.value

    def autotune_record(self):
        """Timings of the last autotune: list of (name, ms, chosen)."""
        buf = (_TuneEntry * 64)()
        ln = C.c_int(0)
        check(lib().ps_autotune_record(self._h, buf, 64, C.byref(ln)))
        return [(buf[i].name.decode(), buf[i].ms, bool(buf[i].chosen)) for i in range(ln.value)]

    def copy_schedule_from(self, other: "Problem"):
        check(lib().ps_copy_schedule(other._h, self._h))

    def kernel_times(self):
        """Per-kernel-kind times of the last run (needs timing=2): name -> dict."""
        buf = (_KTime * 64)()
        ln = C.c_int(0)
        check(lib().ps_problem_kernel_times(self._h, buf, 64, C.byref(ln)))
        return {buf[i].name.decode(): dict(launches=buf[i].launches, ms=buf[i].ms, bytes=buf[i].bytes,
                                           flops=buf[i].flops) for i in range(ln.value)}

    def __del__(self):
        if getattr(self, "_h", None):
            lib().ps_problem_destroy(self._h)
            self._h = None


def parareal_solve(problem: "Problem", u0, a, tol, adjoint_tol=None):
    """U_N of the parareal solve as a differentiable function of u0 and the nodal
    coefficient a (torch.autograd.Function backed by ps_run_parareal and ps_adjoint_vjp)."""
    import torch

    class _Solve(torch.autograd.Function):
        @staticmethod
        def forward(ctx, u0_, a_):
            problem.update_coefficients(a_.detach().contiguous())
            problem.run(u0_.detach().contiguous(), tol)
            return problem.state(problem.N).clone()

        @staticmethod
        def backward(ctx, gN):
            gu, ga = problem.vjp(gN.detach().contiguous(), adjoint_tol if adjoint_tol is not None else tol,
                                 want_a=ctx.needs_input_grad[1])
            return gu, ga

    return _Solve.apply(u0, a)


class Batch:
    """Independent problems advanced together (grouped launches, one CUDA graph per parareal
    iteration).  Keeps references to its problems."""

    def __init__(self, problems, stream=None):
        self.problems = list(problems)
        arr = (_VP * max(len(self.problems), 1))(*[p._h for p in self.problems])
        h = _VP()
        rc = lib().ps_batch_create(arr, len(self.problems), _stream(stream), C.byref(h))
        if rc != PS_OK:
            raise PsError(rc, lib().ps_batch_last_error().decode())
        self._h = h

    def add(self, problem, stream=None):
        """Append a problem (its index is the previous problem count)."""
        rc = lib().ps_batch_add(self._h, problem._h, _stream(stream))
        if rc != PS_OK:
            raise PsError(rc, lib().ps_batch_last_error().decode())
        self.problems.append(problem)

    def state(self, index, n, out=None, stream=None):
        """U_n of problem `index` after the last run (through ps_batch_get_state)."""
        import torch
        p = self.problems[index] if 0 <= index < len(self.problems) else None
        if out is None:
            out = torch.empty(p.grid.shape if p else (1,), dtype=torch.float64, device="cuda")
        # the library checks the index and slice (a bad one raises PsError below)
        rc = lib().ps_batch_get_state(self._h, int(index), int(n), _dev_ptr(out, p.grid.nt if p else None),
                                      _stream(stream))
        if rc != PS_OK:
            raise PsError(rc, lib().ps_batch_last_error().decode())
        return out

    def run(self, u0s, tol, max_iter=0, stream=None):
        ptrs = (_VP * len(u0s))(*[_dev_ptr(u, p.grid.nt) for u, p in zip(u0s, self.problems)])
        its = (C.c_int * len(u0s))()
        rc = lib().ps_batch_run(self._h, ptrs, float(tol), int(max_iter), _stream(stream), its)
        if rc != PS_OK:
            raise PsError(rc, lib().ps_batch_last_error().decode())
        return list(its)

    def stats(self):
        s = _Stats()
        rc = lib().ps_batch_stats(self._h, C.byref(s))
        if rc != PS_OK:
            raise PsError(rc, lib().ps_batch_last_error().decode())
        return dict(iterations=s.iterations, unknown_updates=s.unknown_updates, kernel_launches=s.kernel_launches)

    def autotune(self, budget_ms=100, stream=None):
        """Autotune one problem per grid size and slice count, copy its schedule to the rest."""
        chosen = {}
        for p in self.problems:
            key = (p.grid.n, p.N)
            if key not in chosen:
                chosen[key] = (p, p.autotune(budget_ms, stream))
            else:
                p.copy_schedule_from(chosen[key][0])
        return {k: v[1] for k, v in chosen.items()}

    def __del__(self):
        if getattr(self, "_h", None):
            lib().ps_batch_destroy(self._h)
            self._h = None
