"""ctypes binding of librve.so (names and arguments as in include/rve.h)."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

lib_path = os.environ.get("RVE_LIB") or os.path.join(os.path.dirname(os.path.abspath(__file__)), "librve.so")
if not os.path.exists(lib_path):
    raise ImportError(f"{lib_path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
                      "(the solver has no CPU fallback)")
lib = C.CDLL(lib_path)

RVE_OK, RVE_EINVAL, RVE_ENOMEM, RVE_ECUDA, RVE_EADMIT = 0, -1, -2, -3, -4
RVE_STATUS_CONVERGED, RVE_STATUS_MAX_ITER, RVE_STATUS_NONFINITE, RVE_STATUS_EMPTY = 0, 1, 2, 3
RVE_STATUS_RUNNING = 4
RVE_PREC_PLAIN_F64, RVE_PREC_MIXED, RVE_PREC_BATCHED_F64 = 0, 1, 2
RVE_DAMP_VISCOUS, RVE_DAMP_KINETIC = 0, 1
RVE_KERNEL_AUTO, RVE_KERNEL_TWO_PHASE, RVE_KERNEL_NODE = 0, 1, 2


class rve_options(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("check_every", C.c_int32),
                ("precision", C.c_int32), ("warm_start", C.c_int32), ("damping", C.c_double),
                ("threads", C.c_int32), ("graphs", C.c_int32), ("sigma_tol", C.c_double),
                ("damping_mode", C.c_int32), ("energy_check", C.c_int32), ("damping_scale", C.c_double),
                ("kernel", C.c_int32), ("reserved_", C.c_int32)]


class rve_batch_info(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("n_rve", "free_nodes", "active_fibers", "fixed_fibers",
                                         "pruned_fibers", "n_bins", "device_bytes")]


_P = C.c_void_p
_I64 = C.c_int64
_I32 = C.c_int32
_D = C.c_double


def _sig(name, res, args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = args
    return f


rve_options_default = _sig("rve_options_default", None, [C.POINTER(rve_options)])
rve_batch_create = _sig("rve_batch_create", C.c_int, [C.POINTER(_P), C.c_int, _I64, _P, _P, _P, _P, _P, _P, _P, _P,
                                                      _P, C.POINTER(rve_options)])
rve_set_options = _sig("rve_set_options", C.c_int, [_P, C.POINTER(rve_options)])
rve_solve = _sig("rve_solve", C.c_int, [_P, _P, _D, _I32, _P, _P, _P, _P])
rve_solve_subset = _sig("rve_solve_subset", C.c_int, [_P, _P, _I64, _P, _D, _I32, _P, _P, _P, _P])
rve_solve_host = _sig("rve_solve_host", C.c_int, [_P, _P, _D, _I32, _P, _P, _P])
rve_solve_plain_noalloc = _sig("rve_solve_plain_noalloc", C.c_int, [_P, _I64, _P, _D, _I32, _P, _P, _P, _P])
RVE_NOALLOC_MAX_ACTIVE_FIBERS, RVE_NOALLOC_MAX_FREE_NODES = 16384, 8192
rve_tangent = _sig("rve_tangent", C.c_int, [_P, _P, _D, _D, _I32, _P, _P, _P, _P])
rve_tangent_mandel = _sig("rve_tangent_mandel", C.c_int, [_P, _P, _D, _D, _I32, _P, _P, _P, _P])
rve_orientation = _sig("rve_orientation", C.c_int, [_P, _P, _I32, _P, _P])
rve_energy = _sig("rve_energy", C.c_int, [_P, _I32, _P, _P])
rve_reset_state = _sig("rve_reset_state", C.c_int, [_P, _P, _I64])
rve_batch_get_info = _sig("rve_batch_get_info", C.c_int, [_P, C.POINTER(rve_batch_info)])
rve_batch_get_sizes = _sig("rve_batch_get_sizes", C.c_int, [_P, _P, _P, _P])
rve_get_positions = _sig("rve_get_positions", C.c_int, [_P, _I64, _P, _I32, _P])
rve_set_positions = _sig("rve_set_positions", C.c_int, [_P, _I64, _P, _I32, _P])


class rve_bin_info(C.Structure):
    _fields_ = [("n_rve", C.c_int32), ("mode", C.c_int32), ("threads", C.c_int32), ("nodes_per_thread", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("check_every", C.c_int32), ("smem_bytes", C.c_int64),
                ("kernel", C.c_int32), ("cluster", C.c_int32), ("exclusive", C.c_int32), ("sorted", C.c_int32)]


rve_batch_get_bins = _sig("rve_batch_get_bins", C.c_int, [_P, _I32, _I32, C.POINTER(rve_bin_info)])
rve_autotune = _sig("rve_autotune", C.c_int, [_P, _P, _I32, _P, C.POINTER(_D), C.POINTER(_D)])
rve_set_kernel_timing = _sig("rve_set_kernel_timing", C.c_int, [_P, _I32])
rve_last_kernel_ms = _sig("rve_last_kernel_ms", C.c_int, [_P, _I32, _P])
rve_batch_destroy = _sig("rve_batch_destroy", None, [_P])


class rve_server_stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("queued", "in_flight", "ready", "completed", "waves", "device_bytes",
                                         "pool_rves", "pool_device_bytes", "wave_iters")]


rve_server_create = _sig("rve_server_create", C.c_int, [C.POINTER(_P), _P, _I32, _I32, _D])
rve_server_submit = _sig("rve_server_submit", C.c_int, [_P, _I64, _P, _I64])
rve_server_set_wave_iters = _sig("rve_server_set_wave_iters", C.c_int, [_P, _I32])
rve_server_add_rves = _sig("rve_server_add_rves", C.c_int, [_P, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                                            C.POINTER(_I64)])
rve_server_remove_rves = _sig("rve_server_remove_rves", C.c_int, [_P, _I64])
rve_server_step = _sig("rve_server_step", C.c_int, [_P])
rve_server_drain = _sig("rve_server_drain", C.c_int, [_P])
rve_server_poll = _sig("rve_server_poll", C.c_int64, [_P, _I64, _P, _P, _P, _P, _P])
rve_server_get_stats = _sig("rve_server_get_stats", C.c_int, [_P, C.POINTER(rve_server_stats)])
rve_server_destroy = _sig("rve_server_destroy", None, [_P])
rve_last_error = _sig("rve_last_error", C.c_char_p, [])


class RveError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where} failed ({code}): {rve_last_error().decode()}")


def _check(rc: int, where: str) -> None:
    if rc != RVE_OK:
        raise RveError(rc, where)


def _ptr(a) -> int | None:
    """Address of a numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "arrays must be C-contiguous"
        return a.ctypes.data
    assert a.is_contiguous(), "tensors must be contiguous"
    return a.data_ptr()


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


_OPTION_NAMES = frozenset(n for n, _ in rve_options._fields_ if not n.startswith("reserved"))


def _set_fields(o: rve_options, kw: dict) -> None:
    for k, v in kw.items():
        if k not in _OPTION_NAMES:  # a ctypes structure would silently take a new attribute
            raise TypeError(f"unknown option {k!r}; options are {sorted(_OPTION_NAMES)}")
        setattr(o, k, v)


def options(**kw) -> rve_options:
    o = rve_options()
    rve_options_default(C.byref(o))
    _set_fields(o, kw)
    return o


class RveBatch:
    """Owner of an ``rve_batch`` handle; methods map one to one on the C calls."""

    def __init__(self, packed, device: int = 0, **opts):
        p = packed
        self._keep = [np.ascontiguousarray(p.node_off, np.int64), np.ascontiguousarray(p.X, np.float64),
                      np.ascontiguousarray(p.fiber_off, np.int64), np.ascontiguousarray(p.conn, np.int32),
                      np.ascontiguousarray(p.L0, np.float64), np.ascontiguousarray(p.EA, np.float64),
                      np.ascontiguousarray(p.B, np.float64), np.ascontiguousarray(p.is_boundary, np.uint8),
                      None if p.V0 is None else np.ascontiguousarray(p.V0, np.float64)]
        self.n_rve = int(self._keep[0].shape[0] - 1)
        self.device = device
        self.opt = options(**opts)
        h = _P()
        rc = rve_batch_create(C.byref(h), device, self.n_rve, *[_ptr(a) for a in self._keep], C.byref(self.opt))
        _check(rc, "rve_batch_create")
        self.h = h
        self._keep = None

    def close(self) -> None:
        if getattr(self, "h", None):
            rve_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, **kw) -> None:
        _set_fields(self.opt, kw)
        _check(rve_set_options(self.h, C.byref(self.opt)), "rve_set_options")

    def info(self) -> dict:
        i = rve_batch_info()
        _check(rve_batch_get_info(self.h, C.byref(i)), "rve_batch_get_info")
        return {n: getattr(i, n) for n, _ in rve_batch_info._fields_}

    def sizes(self):
        nf, na, nb = (np.zeros(self.n_rve, np.int32) for _ in range(3))
        _check(rve_batch_get_sizes(self.h, _ptr(nf), _ptr(na), _ptr(nb)), "rve_batch_get_sizes")
        return nf, na, nb

    def solve(self, F, tol: float = 0.0, max_iter: int = 0, sigma=None, iters=None, status=None, stream=None):
        """F: CUDA float64 tensor (n, 9) or (n, 3, 3).  Returns (sigma, iters, status) tensors."""
        import torch
        n = self.n_rve
        if sigma is None:
            sigma = torch.empty((n, 9), dtype=torch.float64, device=F.device)
        if iters is None:
            iters = torch.empty(n, dtype=torch.int32, device=F.device)
        if status is None:
            status = torch.empty(n, dtype=torch.int32, device=F.device)
        _check(rve_solve(self.h, _ptr(F), tol, max_iter, _ptr(sigma), _ptr(iters), _ptr(status),
                         _stream_handle(stream)), "rve_solve")
        return sigma, iters, status

    def solve_subset(self, ids, F, tol: float = 0.0, max_iter: int = 0, sigma=None, iters=None, status=None,
                     stream=None):
        import torch
        ids = np.ascontiguousarray(ids, np.int64)
        m = ids.shape[0]
        if sigma is None:
            sigma = torch.empty((m, 9), dtype=torch.float64, device=F.device)
        if iters is None:
            iters = torch.empty(m, dtype=torch.int32, device=F.device)
        if status is None:
            status = torch.empty(m, dtype=torch.int32, device=F.device)
        _check(rve_solve_subset(self.h, _ptr(ids), m, _ptr(F), tol, max_iter, _ptr(sigma), _ptr(iters),
                                _ptr(status), _stream_handle(stream)), "rve_solve_subset")
        return sigma, iters, status

    def solve_host(self, F, tol: float = 0.0, max_iter: int = 0):
        """F: numpy float64 (n, 9) or (n, 3, 3).  Returns numpy (sigma, iters, status)."""
        F = np.ascontiguousarray(F, np.float64).reshape(self.n_rve, 9)
        sigma = np.empty((self.n_rve, 9))
        iters = np.empty(self.n_rve, np.int32)
        status = np.empty(self.n_rve, np.int32)
        _check(rve_solve_host(self.h, _ptr(F), tol, max_iter, _ptr(sigma), _ptr(iters), _ptr(status)),
               "rve_solve_host")
        return sigma, iters, status

    def solve_plain_noalloc(self, r: int, F, tol: float = 0.0, max_iter: int = 0, sigma=None, iters=None,
                            status=None, stream=None):
        """Plain FP64 solve of RVE r without any device allocation (see include/rve.h).
        F: CUDA float64 tensor of 9; outputs are CUDA tensors of 9, 1 and 1 elements."""
        import torch
        if sigma is None:
            sigma = torch.empty(9, dtype=torch.float64, device=F.device)
        if iters is None:
            iters = torch.empty(1, dtype=torch.int32, device=F.device)
        if status is None:
            status = torch.empty(1, dtype=torch.int32, device=F.device)
        _check(rve_solve_plain_noalloc(self.h, r, _ptr(F), tol, max_iter, _ptr(sigma), _ptr(iters), _ptr(status),
                                       _stream_handle(stream)), "rve_solve_plain_noalloc")
        return sigma, iters, status

    def tangent(self, F, h: float = 1e-4, tol: float = 0.0, max_iter: int = 0, stream=None):
        import torch
        n = self.n_rve
        sigma = torch.empty((n, 9), dtype=torch.float64, device=F.device)
        D = torch.empty((n, 81), dtype=torch.float64, device=F.device)
        status = torch.empty(n, dtype=torch.int32, device=F.device)
        _check(rve_tangent(self.h, _ptr(F), h, tol, max_iter, _ptr(sigma), _ptr(D), _ptr(status),
                           _stream_handle(stream)), "rve_tangent")
        return sigma, D, status

    def tangent_mandel(self, F, h: float = 1e-4, tol: float = 0.0, max_iter: int = 0, stream=None):
        """The paper's six-solve tangent: returns (sigma (n, 9), C (n, 6, 6) Mandel, status)."""
        import torch
        n = self.n_rve
        sigma = torch.empty((n, 9), dtype=torch.float64, device=F.device)
        Cm = torch.empty((n, 6, 6), dtype=torch.float64, device=F.device)
        status = torch.empty(n, dtype=torch.int32, device=F.device)
        _check(rve_tangent_mandel(self.h, _ptr(F), h, tol, max_iter, _ptr(sigma), _ptr(Cm), _ptr(status),
                                  _stream_handle(stream)), "rve_tangent_mandel")
        return sigma, Cm, status

    def orientation(self, F, precision: int | None = None, stream=None):
        """Orientation tensors (n, 3, 3) at the state of the last solve in ``precision``;
        the degree of alignment along a unit direction a is (3 a.Omega.a - 1)/2."""
        import torch
        prec = self.opt.precision if precision is None else precision
        om = torch.empty((self.n_rve, 3, 3), dtype=torch.float64, device=F.device)
        _check(rve_orientation(self.h, _ptr(F), prec, _ptr(om), _stream_handle(stream)), "rve_orientation")
        return om

    def bins(self, precision: int | None = None) -> list[dict]:
        prec = self.opt.precision if precision is None else precision
        arr = (rve_bin_info * 64)()
        n = rve_batch_get_bins(self.h, prec, 64, arr)
        if n < 0:
            raise RveError(n, "rve_batch_get_bins")
        return [{f: getattr(arr[i], f) for f, _ in rve_bin_info._fields_} for i in range(n)]

    def autotune(self, F, reps: int = 2, stream=None) -> tuple[float, float]:
        """Tune every bin's launch configuration on deformation gradients F (CUDA tensor);
        returns the summed bin times (ms) before and after."""
        before, after = C.c_double(), C.c_double()
        _check(rve_autotune(self.h, _ptr(F), reps, _stream_handle(stream), C.byref(before), C.byref(after)),
               "rve_autotune")
        return before.value, after.value

    def set_kernel_timing(self, on: bool = True) -> None:
        _check(rve_set_kernel_timing(self.h, 1 if on else 0), "rve_set_kernel_timing")

    def last_kernel_ms(self) -> np.ndarray:
        """Durations (ms) of the fused-kernel launches since timing was last switched."""
        n = rve_last_kernel_ms(self.h, 0, None)
        if n < 0:
            raise RveError(n, "rve_last_kernel_ms")
        out = np.zeros(max(n, 1), np.float64)
        m = rve_last_kernel_ms(self.h, n, out.ctypes.data_as(C.c_void_p))
        if m < 0:
            raise RveError(m, "rve_last_kernel_ms")
        return out[:n]

    def energy(self, precision: int | None = None, stream=None):
        """Energy records (n_rve, 6) of the last solve with energy_check = 1:
        dW, K, D, C, M and the largest relative balance error."""
        import torch
        prec = self.opt.precision if precision is None else precision
        out = torch.empty((self.n_rve, 6), dtype=torch.float64, device=f"cuda:{self.device}")
        _check(rve_energy(self.h, prec, _ptr(out), _stream_handle(stream)), "rve_energy")
        return out.cpu().numpy()

    def reset_state(self, ids=None) -> None:
        if ids is None:
            _check(rve_reset_state(self.h, None, 0), "rve_reset_state")
        else:
            ids = np.ascontiguousarray(ids, np.int64)
            _check(rve_reset_state(self.h, _ptr(ids), ids.shape[0]), "rve_reset_state")

    def positions(self, r: int, F, n_nodes: int, precision: int | None = None):
        F = np.ascontiguousarray(F, np.float64).reshape(9)
        x = np.empty((n_nodes, 3))
        prec = self.opt.precision if precision is None else precision
        _check(rve_get_positions(self.h, r, _ptr(F), prec, _ptr(x)), "rve_get_positions")
        return x

    def set_positions(self, r: int, F, x, precision: int | None = None) -> None:
        F = np.ascontiguousarray(F, np.float64).reshape(9)
        x = np.ascontiguousarray(x, np.float64)
        prec = self.opt.precision if precision is None else precision
        _check(rve_set_positions(self.h, r, _ptr(F), prec, _ptr(x)), "rve_set_positions")


class RveServer:
    """Owner of an ``rve_server`` handle (continuous batching over a resident
    pool: the batch given here plus groups admitted by ``add_rves``)."""

    def __init__(self, batch: RveBatch, n_slots: int = 4, max_wave: int = 1024, hbm_cap_bytes: float = 150e9,
                 wave_iters: int = 0):
        self.batch = batch
        h = _P()
        _check(rve_server_create(C.byref(h), batch.h, n_slots, max_wave, hbm_cap_bytes), "rve_server_create")
        self.h = h
        self._F = np.zeros(9)
        if wave_iters:
            self.set_wave_iters(wave_iters)

    def set_wave_iters(self, wave_iters: int) -> None:
        _check(rve_server_set_wave_iters(self.h, wave_iters), "rve_server_set_wave_iters")

    def add_rves(self, packed) -> int:
        """Admit the networks of ``packed`` (rvegen.Packed layout) into the
        pool; returns the global id of the first (RveError RVE_EADMIT when
        they do not fit under the cap)."""
        p = packed
        keep = [np.ascontiguousarray(p.node_off, np.int64), np.ascontiguousarray(p.X, np.float64),
                np.ascontiguousarray(p.fiber_off, np.int64), np.ascontiguousarray(p.conn, np.int32),
                np.ascontiguousarray(p.L0, np.float64), np.ascontiguousarray(p.EA, np.float64),
                np.ascontiguousarray(p.B, np.float64), np.ascontiguousarray(p.is_boundary, np.uint8),
                None if p.V0 is None else np.ascontiguousarray(p.V0, np.float64)]
        first = _I64(-1)
        _check(rve_server_add_rves(self.h, keep[0].shape[0] - 1, *[_ptr(a) for a in keep], C.byref(first)),
               "rve_server_add_rves")
        return int(first.value)

    def remove_rves(self, first_id: int) -> None:
        _check(rve_server_remove_rves(self.h, first_id), "rve_server_remove_rves")

    def submit(self, rve_id: int, F, tag: int) -> None:
        self._F[:] = np.asarray(F, np.float64).reshape(9)
        _check(rve_server_submit(self.h, rve_id, _ptr(self._F), tag), "rve_server_submit")

    def step(self) -> None:
        _check(rve_server_step(self.h), "rve_server_step")

    def drain(self) -> None:
        _check(rve_server_drain(self.h), "rve_server_drain")

    def poll(self, max_items: int = 65536):
        tags = np.empty(max_items, np.int64)
        sigma = np.empty((max_items, 9))
        iters = np.empty(max_items, np.int32)
        status = np.empty(max_items, np.int32)
        lat = np.empty(max_items)
        n = rve_server_poll(self.h, max_items, _ptr(tags), _ptr(sigma), _ptr(iters), _ptr(status), _ptr(lat))
        if n < 0:
            raise RveError(int(n), "rve_server_poll")
        return tags[:n], sigma[:n], iters[:n], status[:n], lat[:n]

    def stats(self) -> dict:
        st = rve_server_stats()
        _check(rve_server_get_stats(self.h, C.byref(st)), "rve_server_get_stats")
        return {n: getattr(st, n) for n, _ in rve_server_stats._fields_}

    def close(self) -> None:
        if getattr(self, "h", None):
            rve_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
