"""Python binding of liblpop.so: PDHG with online preconditioning for LP on GB300.

Argument marshalling only.  Every step of the method runs in the library's
CUDA kernels; there is no Python or CPU fallback, and every function raises
if the shared library has not been built (``python -m
paper_2506_17650_gb300.build``).  The function names are those of the C ABI
in ``include/lpop.h``.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblpop.so")

LP_OK = 0
LP_ERR_INVALID_ARG = -1
LP_ERR_INVALID_INPUT = -2
LP_ERR_CUDA = -3
LP_ERR_OOM = -4
LP_ERR_NOT_SOLVED = -5

LP_STATUS_NONE = 0
LP_OPTIMAL = 1
LP_ITERATION_LIMIT = 2
LP_TIME_LIMIT = 3
LP_NUMERICAL_ERROR = 4

LP_MODE_PLAIN = 0
LP_MODE_PDLP = 1

LP_PREC_FP64 = 0
LP_PREC_MIXED = 1

LP_SCHED_ADAGRAD = 0
LP_SCHED_ADAGRAD_NORM = 1
LP_SCHED_CONST = 2


class LpOptions(ctypes.Structure):
    _fields_ = [
        ("mode", c_int32),
        ("scheduler", c_int32),
        ("alpha", c_double),
        ("phi", c_int32),
        ("normalize", c_int32),
        ("precond_floor", c_double),
        ("ruiz_iters", c_int32),
        ("pc_beta", c_double),
        ("check_every", c_int32),
        ("restart", c_int32),
        ("power_iters", c_int32),
        ("plain_step_factor", c_double),
        ("time_limit", c_double),
        ("use_graph", c_int32),
        ("kernel_timing", c_int32),
        ("device", c_int32),
        ("stream", c_void_p),
        ("precision", c_int32),
        ("refine_tol", c_double),
        ("device_alloc", c_void_p),
        ("device_free", c_void_p),
        ("alloc_ctx", c_void_p),
        ("refine_stall", c_int32),
        ("log_every", c_int32),
    ]


class LpStats(ctypes.Structure):
    _fields_ = [
        ("pobj", c_double),
        ("dobj", c_double),
        ("rel_pres", c_double),
        ("rel_dres", c_double),
        ("rel_gap", c_double),
        ("iterations", c_int64),
        ("accepted", c_int64),
        ("restarts", c_int64),
        ("eta", c_double),
        ("omega", c_double),
        ("solve_ms", c_double),
        ("status", c_int32),
        ("reserved", c_int32),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


class LpError(RuntimeError):
    def __init__(self, code, message):
        super().__init__(f"lpop error {code}: {message}")
        self.code = code


_lib = None
_DP = POINTER(c_double)


def load_library(path: str | None = None):
    """Load liblpop.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing; build it with `python -m paper_2506_17650_gb300.build` "
            "(the solver has no CPU fallback)")
    lib = ctypes.CDLL(path)
    lib.lp_options_default.argtypes = [POINTER(LpOptions)]
    lib.lp_options_default.restype = None
    lib.lp_create.argtypes = [c_int32, c_int32, c_int64, POINTER(c_int64), POINTER(c_int32), _DP, _DP, _DP, _DP,
                              _DP, c_char_p, POINTER(LpOptions), POINTER(c_void_p)]
    lib.lp_create.restype = c_int32
    lib.lp_solve.argtypes = [c_void_p, c_double, c_int64, POINTER(c_int32)]
    lib.lp_solve.restype = c_int32
    lib.lp_result.argtypes = [c_void_p, _DP, _DP, POINTER(LpStats)]
    lib.lp_result.restype = c_int32
    lib.lp_get_iterate.argtypes = [c_void_p, _DP, _DP, _DP, _DP, _DP]
    lib.lp_get_iterate.restype = c_int32
    lib.lp_get_scaling.argtypes = [c_void_p, _DP, _DP, _DP]
    lib.lp_get_scaling.restype = c_int32
    lib.lp_get_state.argtypes = [c_void_p, _DP, _DP, _DP]
    lib.lp_get_state.restype = c_int32
    lib.lp_set_state.argtypes = [c_void_p, _DP, _DP, _DP]
    lib.lp_set_state.restype = c_int32
    lib.lp_reset.argtypes = [c_void_p]
    lib.lp_reset.restype = c_int32
    lib.lp_kernel_times.argtypes = [c_void_p, _DP, POINTER(c_int64), c_int32, POINTER(c_int64)]
    lib.lp_kernel_times.restype = c_int32
    lib.lp_power_norm_noalloc.argtypes = [c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                          c_void_p, c_int32, c_void_p, POINTER(c_double)]
    lib.lp_power_norm_noalloc.restype = c_int32
    lib.lp_batch_create.argtypes = [c_int32, POINTER(c_void_p), POINTER(c_void_p)]
    lib.lp_batch_create.restype = c_int32
    lib.lp_batch_set_members.argtypes = [c_void_p, c_int32, POINTER(c_void_p)]
    lib.lp_batch_set_members.restype = c_int32
    lib.lp_batch_set_schedule.argtypes = [c_void_p, c_int32, c_int64]
    lib.lp_batch_set_schedule.restype = c_int32
    lib.lp_batch_set_handoff.argtypes = [c_void_p, c_int64]
    lib.lp_batch_set_handoff.restype = c_int32
    lib.lp_batch_round.argtypes = [c_void_p, c_double, c_int32, c_int64, POINTER(c_int32)]
    lib.lp_batch_round.restype = c_int32
    lib.lp_batch_solve.argtypes = [c_void_p, c_double, c_int64, c_int32, POINTER(c_int32)]
    lib.lp_batch_solve.restype = c_int32
    lib.lp_batch_autotune.argtypes = [c_void_p, c_double, c_int32, POINTER(c_int32), POINTER(c_int64),
                                      POINTER(c_double)]
    lib.lp_batch_autotune.restype = c_int32
    lib.lp_batch_status.argtypes = [c_void_p, POINTER(c_int32), POINTER(c_int64)]
    lib.lp_batch_status.restype = c_int32
    lib.lp_batch_launches.argtypes = [c_void_p, POINTER(c_int64)]
    lib.lp_batch_launches.restype = c_int32
    lib.lp_batch_destroy.argtypes = [c_void_p]
    lib.lp_batch_destroy.restype = None
    lib.lp_memory_bytes.argtypes = [c_int32, c_int32, c_int64, POINTER(LpOptions), POINTER(c_int64)]
    lib.lp_memory_bytes.restype = c_int32
    lib.lp_destroy.argtypes = [c_void_p]
    lib.lp_destroy.restype = None
    lib.lp_last_error.argtypes = [c_void_p]
    lib.lp_last_error.restype = c_char_p
    _lib = lib
    return lib


def _check(rc, handle=None):
    if rc != LP_OK:
        msg = load_library().lp_last_error(handle)
        raise LpError(rc, msg.decode() if msg else "")


def _ptr(a, ctype):
    return a.ctypes.data_as(POINTER(ctype)) if a is not None else None


def _out(n):
    return np.empty(n, dtype=np.float64)


def lp_options_default(**overrides) -> LpOptions:
    """Default options, with keyword overrides (e.g. ``alpha=1e-3, phi=20``)."""
    o = LpOptions()
    load_library().lp_options_default(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "stream" and v is not None:
            v = int(v)
        setattr(o, k, v)
    return o


def lp_create(m, n, row_ptr, col_idx, val, b, c, lb, ub, sense, opts: LpOptions | None = None):
    """Create a problem from host arrays (CSR of A, b, c, bounds, senses 'E'/'L'/'G')."""
    lib = load_library()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    lb = np.ascontiguousarray(lb, dtype=np.float64)
    ub = np.ascontiguousarray(ub, dtype=np.float64)
    if isinstance(sense, str):
        sense = sense.encode()
    sense = np.ascontiguousarray(np.frombuffer(bytes(sense), dtype=np.uint8) if isinstance(sense, bytes) else sense,
                                 dtype=np.uint8)
    if row_ptr.size != m + 1 or b.size != m or sense.size != m or c.size != n or lb.size != n or ub.size != n:
        raise LpError(LP_ERR_INVALID_ARG, "array sizes do not match m and n")
    handle = c_void_p()
    rc = lib.lp_create(int(m), int(n), int(row_ptr[-1]) if row_ptr.size else 0, _ptr(row_ptr, c_int64),
                       _ptr(col_idx, c_int32), _ptr(val, c_double), _ptr(b, c_double), _ptr(c, c_double),
                       _ptr(lb, c_double), _ptr(ub, c_double), sense.ctypes.data_as(c_char_p),
                       ctypes.byref(opts) if opts is not None else None, ctypes.byref(handle))
    _check(rc)
    return handle


def lp_solve(handle, rel_kkt_tol=1e-4, iter_limit=1_000_000) -> int:
    """Run until the relative KKT tolerance or the (cumulative) iteration limit; returns an LP_* status."""
    st = c_int32(0)
    _check(load_library().lp_solve(handle, float(rel_kkt_tol), int(iter_limit), ctypes.byref(st)), handle)
    return st.value


def lp_result(handle, m, n, want_x=True, want_y=True):
    """(x, y, stats) in user units and the caller's order."""
    x = _out(n) if want_x else None
    y = _out(m) if want_y else None
    st = LpStats()
    _check(load_library().lp_result(handle, _ptr(x, c_double), _ptr(y, c_double), ctypes.byref(st)), handle)
    return x, y, st.as_dict()


def lp_get_iterate(handle, m, n):
    """Scaled-space iterate: dict(x, y, T, Sigma, eta, omega, k, attempts, wsum, restarts, eta_max, accepted)."""
    x, y, T, S, scal = _out(n), _out(m), _out(n), _out(m), _out(8)
    _check(load_library().lp_get_iterate(handle, _ptr(x, c_double), _ptr(y, c_double), _ptr(T, c_double),
                                         _ptr(S, c_double), _ptr(scal, c_double)), handle)
    return dict(x=x, y=y, T=T, Sigma=S, eta=scal[0], omega=scal[1], k=int(scal[2]), attempts=int(scal[3]),
                wsum=scal[4], restarts=int(scal[5]), eta_max=scal[6], accepted=bool(scal[7]))


def lp_get_scaling(handle, m, n):
    """(dr, dc, dict(eta0, omega0, norm_est, amax, grid sizes, work units)) with A~ = diag(dr) A diag(dc)."""
    dr, dc, scal = _out(m), _out(n), _out(8)
    _check(load_library().lp_get_scaling(handle, _ptr(dr, c_double), _ptr(dc, c_double), _ptr(scal, c_double)),
           handle)
    return dr, dc, dict(eta0=scal[0], omega0=scal[1], norm_est=scal[2], amax=scal[3], grid_a=int(scal[4]),
                        grid_at=int(scal[5]), units_a=int(scal[6]), units_at=int(scal[7]))


STATE_N = ("x", "xbar", "T", "GT", "x_last")
STATE_M = ("y", "ybar", "ax", "Sigma", "GS", "y_last")
STATE_SCAL = ("eta", "omega", "wsum", "gp_norm", "gd_norm", "klast_p2", "klast_d2", "klast_g2", "k_prev", "k",
              "attempts", "last_restart_attempt", "restarts", "refs_set", "initial_check_done")
_STATE_INT = {"k", "attempts", "last_restart_attempt", "restarts", "refs_set", "initial_check_done"}


def lp_get_state(handle, m, n):
    """Complete scaled-space state (checkpoint): dict of the STATE_N / STATE_M vectors and STATE_SCAL scalars."""
    vn, vm, scal = _out(5 * n), _out(6 * m), _out(16)
    _check(load_library().lp_get_state(handle, _ptr(vn, c_double), _ptr(vm, c_double), _ptr(scal, c_double)), handle)
    out = {k: vn[i * n:(i + 1) * n].copy() for i, k in enumerate(STATE_N)}
    out.update({k: vm[i * m:(i + 1) * m].copy() for i, k in enumerate(STATE_M)})
    out.update({k: (int(scal[i]) if k in _STATE_INT else float(scal[i])) for i, k in enumerate(STATE_SCAL)})
    return out


def lp_set_state(handle, m, n, state):
    """Resume from a state dict with the keys of lp_get_state."""
    vn = np.ascontiguousarray(np.concatenate([np.asarray(state[k], dtype=np.float64).reshape(n) for k in STATE_N]))
    vm = np.ascontiguousarray(np.concatenate([np.asarray(state[k], dtype=np.float64).reshape(m) for k in STATE_M])) \
        if m > 0 else np.zeros(1)
    scal = np.zeros(16)
    for i, k in enumerate(STATE_SCAL):
        scal[i] = float(state[k])
    _check(load_library().lp_set_state(handle, _ptr(vn, c_double), _ptr(vm, c_double), _ptr(scal, c_double)), handle)


def lp_reset(handle):
    _check(load_library().lp_reset(handle), handle)


def lp_kernel_times(handle):
    """(ms[2], samples[2], launches): event-timed primal / dual step kernels and the launch count."""
    ms = _out(2)
    ns = np.zeros(2, dtype=np.int64)
    launches = c_int64(0)
    _check(load_library().lp_kernel_times(handle, _ptr(ms, c_double), _ptr(ns, c_int64), 2, ctypes.byref(launches)),
           handle)
    return ms, ns, launches.value


def lp_power_norm_noalloc(m, n, a_row_ptr, a_col_idx, a_val, at_row_ptr, at_col_idx, at_val, iters=200,
                          stream=None) -> float:
    """||A||_2 power-iteration estimate without any device allocation.

    For callers that cannot allocate device memory; the six matrix arguments
    are DEVICE addresses (ints, e.g. ``tensor.data_ptr()``) of the CSR of A and
    of A^T.  Uses the library's fixed 8 MiB scratch (2 n + m + 1025 doubles at
    most)."""
    out = c_double(0.0)
    rc = load_library().lp_power_norm_noalloc(int(m), int(n), a_row_ptr, a_col_idx, a_val, at_row_ptr, at_col_idx,
                                              at_val, int(iters), stream, ctypes.byref(out))
    _check(rc)
    return out.value


def lp_memory_bytes(m, n, nnz, opts: LpOptions | None = None) -> int:
    """Device bytes lp_create allocates for a problem of this size (admission by free memory)."""
    v = c_int64(0)
    _check(load_library().lp_memory_bytes(int(m), int(n), int(nnz), ctypes.byref(opts) if opts is not None else None,
                                          ctypes.byref(v)))
    return v.value


def lp_destroy(handle):
    if handle:
        load_library().lp_destroy(handle)


def lp_last_error(handle=None) -> str:
    msg = load_library().lp_last_error(handle)
    return msg.decode() if msg else ""


_DEVICE_ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, ctypes.c_size_t, c_void_p)
_DEVICE_FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, ctypes.c_size_t, c_void_p)


class TorchDeviceAllocator:
    """lp_options.device_alloc / device_free backed by PyTorch's caching
    allocator: a problem's device buffers then count against (and come back
    to) torch's memory pool.  Keep the object alive as long as the problems
    that use it (Problem does)."""

    def __init__(self, device=None):
        import torch

        self._torch = torch
        self.device = torch.cuda.current_device() if device is None else int(device)
        self._alloc = _DEVICE_ALLOC_FN(self._do_alloc)
        self._free = _DEVICE_FREE_FN(self._do_free)

    def _do_alloc(self, nbytes, ctx):
        try:
            return self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device)
        except RuntimeError:
            return None  # the library reports LP_ERR_OOM

    def _do_free(self, ptr, nbytes, ctx):
        self._torch.cuda.caching_allocator_delete(ptr)

    def options(self):
        return dict(device_alloc=ctypes.cast(self._alloc, c_void_p).value,
                    device_free=ctypes.cast(self._free, c_void_p).value)


class Problem:
    """Owning wrapper: ``with Problem(lp, alpha=1e-3) as p: p.solve(1e-4)``.

    ``lp`` is any object with the attributes m, n, row_ptr, col_idx, val, b,
    c, lb, ub, sense (the caller's host arrays).  ``allocator``: an object with
    ``options()`` giving device_alloc / device_free (e.g. TorchDeviceAllocator)."""

    def __init__(self, lp, allocator=None, **options):
        self.m, self.n = int(lp.m), int(lp.n)
        self.allocator = allocator  # its callbacks must outlive the problem
        if allocator is not None:
            options = dict(options, **allocator.options())
        self.options = lp_options_default(**options)
        self.handle = lp_create(self.m, self.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, lp.lb, lp.ub,
                                lp.sense, self.options)

    def solve(self, rel_kkt_tol=1e-4, iter_limit=1_000_000):
        return lp_solve(self.handle, rel_kkt_tol, iter_limit)

    def result(self, want_x=True, want_y=True):
        return lp_result(self.handle, self.m, self.n, want_x, want_y)

    def iterate(self):
        return lp_get_iterate(self.handle, self.m, self.n)

    def scaling(self):
        return lp_get_scaling(self.handle, self.m, self.n)

    def reset(self):
        lp_reset(self.handle)

    def get_state(self):
        return lp_get_state(self.handle, self.m, self.n)

    def set_state(self, state):
        lp_set_state(self.handle, self.m, self.n, state)

    def kernel_times(self):
        return lp_kernel_times(self.handle)

    def close(self):
        if self.handle:
            lp_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _handles(problems):
    arr = (c_void_p * max(len(problems), 1))()
    for i, p in enumerate(problems):
        arr[i] = p.handle if isinstance(p, Problem) else p
    return arr


def lp_batch_create(problems):
    h = c_void_p()
    _check(load_library().lp_batch_create(len(problems), _handles(problems), ctypes.byref(h)))
    return h


def lp_batch_set_members(batch, problems):
    _check(load_library().lp_batch_set_members(batch, len(problems), _handles(problems)))


def lp_batch_set_schedule(batch, cluster_size=1, wide_nnz=1 << 62):
    _check(load_library().lp_batch_set_schedule(batch, int(cluster_size), int(wide_nnz)))


def lp_batch_set_handoff(batch, attempts=0):
    _check(load_library().lp_batch_set_handoff(batch, int(attempts)))


def lp_batch_round(batch, rel_kkt_tol=1e-4, attempts=64, iter_limit=1_000_000) -> int:
    act = c_int32(0)
    _check(load_library().lp_batch_round(batch, float(rel_kkt_tol), int(attempts), int(iter_limit), ctypes.byref(act)))
    return act.value


def lp_batch_solve(batch, rel_kkt_tol=1e-4, iter_limit=1_000_000, round_attempts=256) -> int:
    n = c_int32(0)
    _check(load_library().lp_batch_solve(batch, float(rel_kkt_tol), int(iter_limit), int(round_attempts),
                                         ctypes.byref(n)))
    return n.value


def lp_batch_autotune(batch, rel_kkt_tol=1e-4, trial_attempts=128):
    """Pick the fastest team schedule on whole trial solves (attempt limit trial_attempts, the batch's
    handoff); resets every member before and after.  Returns (cluster, wide_nnz, ms)."""
    c = c_int32(0)
    w = c_int64(0)
    ms = c_double(0.0)
    _check(load_library().lp_batch_autotune(batch, float(rel_kkt_tol), int(trial_attempts), ctypes.byref(c),
                                            ctypes.byref(w), ctypes.byref(ms)))
    return c.value, w.value, ms.value


def lp_batch_status(batch, count):
    st = np.zeros(count, dtype=np.int32)
    it = np.zeros(count, dtype=np.int64)
    _check(load_library().lp_batch_status(batch, st.ctypes.data_as(POINTER(c_int32)),
                                          it.ctypes.data_as(POINTER(c_int64))))
    return st, it


def lp_batch_launches(batch) -> int:
    v = c_int64(0)
    _check(load_library().lp_batch_launches(batch, ctypes.byref(v)))
    return v.value


def lp_batch_destroy(batch):
    if batch:
        load_library().lp_batch_destroy(batch)


class Batch:
    """Owning wrapper of a batch over Problem objects (which stay owned by the caller)."""

    def __init__(self, problems, cluster_size=1, wide_nnz=1 << 62):
        self.problems = list(problems)
        self.handle = lp_batch_create(self.problems)
        lp_batch_set_schedule(self.handle, cluster_size, wide_nnz)

    def set_members(self, problems):
        self.problems = list(problems)
        lp_batch_set_members(self.handle, self.problems)

    def set_schedule(self, cluster_size, wide_nnz):
        lp_batch_set_schedule(self.handle, cluster_size, wide_nnz)

    def set_handoff(self, attempts):
        lp_batch_set_handoff(self.handle, attempts)

    def round(self, rel_kkt_tol=1e-4, attempts=64, iter_limit=1_000_000):
        return lp_batch_round(self.handle, rel_kkt_tol, attempts, iter_limit)

    def solve(self, rel_kkt_tol=1e-4, iter_limit=1_000_000, round_attempts=256):
        return lp_batch_solve(self.handle, rel_kkt_tol, iter_limit, round_attempts)

    def autotune(self, rel_kkt_tol=1e-4, trial_attempts=128):
        return lp_batch_autotune(self.handle, rel_kkt_tol, trial_attempts)

    def status(self):
        return lp_batch_status(self.handle, len(self.problems))

    def launches(self):
        return lp_batch_launches(self.handle)

    def close(self):
        if self.handle:
            lp_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
