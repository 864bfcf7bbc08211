"""Python binding of libamgdd (GB300 LS-AMG-DD): argument marshalling only.

Every computation runs in the CUDA library declared by include/amgdd.h; this
module loads it with ctypes, converts arguments to plain pointers and sizes,
and raises on a non-OK status.  There is no CPU fallback: importing works
without a GPU, but every call needs the built library and a CUDA device.

Host arrays are numpy arrays; device arrays are torch CUDA tensors (torch is
used for device memory and streams only).
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libamgdd.so")

AMGDD_OK = 0
STATUS = {0: "ok", -1: "invalid argument", -2: "not SPD", -3: "non-finite", -4: "CG breakdown",
          -5: "no convergence", -6: "out of device memory", -7: "CUDA error", -8: "internal error"}
HOST, DEVICE = 0, 1
FP64, MIXED32, MIXED16 = 0, 1, 2
OP_A, OP_RAS, OP_RAST, OP_RESTRICT, OP_PROLONG, OP_VCYCLE, OP_COARSE, OP_M2 = range(8)
ARR_AGG, ARR_OMEGA_PTR, ARR_OMEGA_IDX, ARR_NOMEGA, ARR_K, ARR_Z, ARR_MU = range(7)
ARR_G_PTR, ARR_G_IDX, ARR_A_PTR, ARR_A_IDX, ARR_P_PTR, ARR_P_IDX = range(7, 13)

EXPORTED = [
    "amgdd_params_default", "amgdd_setup", "amgdd_solve", "amgdd_set_precision", "amgdd_set_max_iter", "amgdd_apply",
    "amgdd_num_levels", "amgdd_level_describe", "amgdd_level_export", "amgdd_hierarchy_stats",
    "amgdd_bytes_model", "amgdd_free", "amgdd_status_string", "amgdd_last_error", "amgdd_profile_vcycle",
    "amgdd_kernel_launches", "amgdd_apply_noalloc", "amgdd_device_bytes", "amgdd_server_params_default",
    "amgdd_server_create", "amgdd_server_add_operator", "amgdd_server_submit", "amgdd_server_poll",
    "amgdd_server_stats", "amgdd_server_destroy", "amgdd_hierarchy_save", "amgdd_hierarchy_load",
    "amgdd_selftest_wait_timeouts", "amgdd_aggregate", "amgdd_struct_size", "amgdd_measure_fp64",
    "amgdd_server_submit_problem",
]
AMGDD_PENDING = 1


class ServerParams(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_int64), ("slots", ctypes.c_int), ("max_batch", ctypes.c_int)]


class Csr(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("mem", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [("L_max", ctypes.c_int), ("n_coarse", ctypes.c_int64), ("thresh", ctypes.c_double),
                ("c_min", ctypes.c_int * 8), ("n_cmin", ctypes.c_int), ("precision", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("schur_rtol", ctypes.c_double), ("use_graph", ctypes.c_int),
                ("check_every", ctypes.c_int), ("tune", ctypes.c_int), ("tune_cache", ctypes.c_char_p),
                ("coarse_overlap", ctypes.c_int), ("coarse_refine", ctypes.c_int),
                ("pdl", ctypes.c_int), ("dense_tail", ctypes.c_int), ("ell", ctypes.c_int),
                ("deterministic", ctypes.c_int), ("cycle", ctypes.c_int),
                ("kappa", ctypes.c_double), ("agg_passes", ctypes.c_int), ("schur_gram", ctypes.c_int),
                ("batch_cols", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("relres", ctypes.c_double),
                ("relres_true", ctypes.c_double), ("solve_ms", ctypes.c_double), ("fallback", ctypes.c_int),
                ("iters_mixed", ctypes.c_int)]


class LevelDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nagg", ctypes.c_int64), ("n_next", ctypes.c_int64),
                ("omega_len", ctypes.c_int64), ("z_len", ctypes.c_int64), ("ngroups", ctypes.c_int64),
                ("g_rows", ctypes.c_int64), ("g_vals", ctypes.c_int64), ("w_vals", ctypes.c_int64),
                ("is_coarsest", ctypes.c_int), ("g_sup_len", ctypes.c_int64), ("a_nnz", ctypes.c_int64),
                ("p_nnz", ctypes.c_int64)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libamgdd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libamgdd.so not found at {path}; build it with "
                           "`python -m paper_2601_04112_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.amgdd_params_default.restype = Params
    lib.amgdd_setup.argtypes = [ctypes.POINTER(Csr), vp, vp, i32, ctypes.POINTER(Params), vp, ctypes.POINTER(vp)]
    lib.amgdd_solve.argtypes = [vp, vp, i32, dbl, vp, vp, ctypes.POINTER(Info)]
    lib.amgdd_set_precision.argtypes = [vp, i32]
    lib.amgdd_set_max_iter.argtypes = [vp, i32]
    lib.amgdd_apply.argtypes = [vp, i32, i32, vp, vp, vp]
    lib.amgdd_apply_noalloc.argtypes = [vp, i32, i32, vp, vp, vp]
    lib.amgdd_apply_noalloc.restype = i32
    lib.amgdd_num_levels.argtypes = [vp]
    lib.amgdd_level_describe.argtypes = [vp, i32, ctypes.POINTER(LevelDesc)]
    lib.amgdd_level_export.argtypes = [vp, i32, i32, vp, ctypes.c_size_t]
    lib.amgdd_hierarchy_stats.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    lib.amgdd_bytes_model.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
    lib.amgdd_free.argtypes = [vp]
    lib.amgdd_hierarchy_save.argtypes = [vp, ctypes.c_char_p]
    lib.amgdd_hierarchy_load.argtypes = [ctypes.c_char_p, vp, ctypes.POINTER(vp)]
    lib.amgdd_selftest_wait_timeouts.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.amgdd_aggregate.argtypes = [ctypes.POINTER(Csr), i32, vp, vp, ctypes.POINTER(ctypes.c_int64)]
    lib.amgdd_free.restype = None
    lib.amgdd_status_string.argtypes = [i32]
    lib.amgdd_status_string.restype = ctypes.c_char_p
    lib.amgdd_last_error.restype = ctypes.c_char_p
    lib.amgdd_profile_vcycle.argtypes = [vp, i32, i32, ctypes.POINTER(dbl), ctypes.POINTER(dbl), i32]
    lib.amgdd_profile_vcycle.restype = i32
    lib.amgdd_kernel_launches.restype = ctypes.c_int64
    lib.amgdd_device_bytes.argtypes = [vp, i32]
    lib.amgdd_device_bytes.restype = ctypes.c_int64
    lib.amgdd_server_params_default.restype = ServerParams
    lib.amgdd_server_create.argtypes = [ctypes.POINTER(ServerParams), ctypes.POINTER(vp)]
    lib.amgdd_server_add_operator.argtypes = [vp, ctypes.c_int64, ctypes.POINTER(Csr), vp, vp, i32,
                                              ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_int64),
                                              ctypes.POINTER(i32)]
    lib.amgdd_server_submit.argtypes = [vp, ctypes.c_int64, vp, i32, dbl, vp, ctypes.POINTER(ctypes.c_int64)]
    lib.amgdd_server_poll.argtypes = [vp, ctypes.c_int64, i32, ctypes.POINTER(Info), ctypes.POINTER(dbl)]
    lib.amgdd_server_submit_problem.argtypes = [vp, ctypes.c_int64, ctypes.POINTER(Csr), vp, vp, i32,
                                                ctypes.POINTER(Params), vp, i32, dbl, vp, ctypes.POINTER(ctypes.c_int64),
                                                ctypes.POINTER(i32)]
    lib.amgdd_server_submit_problem.restype = i32
    lib.amgdd_server_stats.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    lib.amgdd_server_destroy.argtypes = [vp]
    lib.amgdd_server_destroy.restype = None
    for name in ("amgdd_server_create", "amgdd_server_add_operator", "amgdd_server_submit", "amgdd_server_poll",
                 "amgdd_server_stats"):
        getattr(lib, name).restype = i32
    for name in ("amgdd_setup", "amgdd_solve", "amgdd_set_precision", "amgdd_set_max_iter", "amgdd_apply",
                 "amgdd_num_levels",
                 "amgdd_level_describe", "amgdd_level_export", "amgdd_hierarchy_stats", "amgdd_bytes_model"):
        getattr(lib, name).restype = i32
    lib.amgdd_measure_fp64.argtypes = [vp, ctypes.POINTER(dbl)]
    lib.amgdd_measure_fp64.restype = i32
    lib.amgdd_struct_size.argtypes = [i32]
    lib.amgdd_struct_size.restype = ctypes.c_size_t
    for which, st in enumerate((Params, Info, LevelDesc, Csr, ServerParams)):
        if lib.amgdd_struct_size(which) != ctypes.sizeof(st):
            raise RuntimeError(f"{path} was built against another amgdd.h: {st.__name__} is "
                               f"{lib.amgdd_struct_size(which)} bytes there, {ctypes.sizeof(st)} here; rebuild it")
    _lib = lib
    return lib


class AmgddError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(st: int):
    if st != AMGDD_OK:
        raise AmgddError(st, _lib.amgdd_last_error().decode())


def _ptr(a):
    """(pointer, is_device) of a numpy array or torch tensor."""
    if a is None:
        return None, False
    if isinstance(a, np.ndarray):
        return a.ctypes.data, False
    return a.data_ptr(), bool(a.is_cuda)


def _stream(stream):
    if stream is not None:
        return stream
    import torch

    return torch.cuda.current_stream().cuda_stream


def aggregate(rowptr, col, n, passes=1, stream=None):
    """Level-0 aggregates of A = D1 + G^T G by `passes` passes of standard
    aggregation on its graph (amgdd_aggregate).  Host arrays in, a host
    int32 array and the aggregate count out."""
    lib = load_library()
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    dummy = np.zeros(1, dtype=np.float64)  # the pattern only: values are not read
    csr = Csr(m=len(rp) - 1, n=int(n), nnz=int(len(cl)), rowptr=rp.ctypes.data, col=cl.ctypes.data,
              val=dummy.ctypes.data, mem=HOST)
    out = np.empty(int(n), dtype=np.int32)
    na = ctypes.c_int64()
    _check(lib.amgdd_aggregate(ctypes.byref(csr), int(passes), stream, out.ctypes.data, ctypes.byref(na)))
    return out, int(na.value)


def selftest_wait_timeouts(stream=None) -> tuple[int, int]:
    """Statuses of the two bounded-wait probes (AMGDD_ERR_TIMEOUT = -9 when reported)."""
    lib = load_library()
    a, b = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib.amgdd_selftest_wait_timeouts(_stream(stream), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def measure_fp64(stream=None) -> float:
    """Measured FP64 FMA throughput of the current device, GFLOP/s (amgdd_measure_fp64)."""
    lib = load_library()
    g = ctypes.c_double()
    _check(lib.amgdd_measure_fp64(_stream(stream), ctypes.byref(g)))
    return float(g.value)


def kernel_launches() -> int:
    return int(load_library().amgdd_kernel_launches())


def params(**kw) -> Params:
    lib = load_library()
    p = lib.amgdd_params_default()
    for k, v in kw.items():
        if k == "c_min":
            v = list(v)
            for i, c in enumerate(v):
                p.c_min[i] = int(c)
            p.n_cmin = len(v)
        elif k == "tune_cache":
            p.tune_cache = None if v is None else str(v).encode()
        else:
            setattr(p, k, v)
    return p


class Hierarchy:
    """A built LS-AMG-DD hierarchy on the current CUDA device."""

    def __init__(self, rowptr, col, val, n, D1=None, agg=None, overlap=1, stream=None, **kw):
        lib = load_library()
        self._lib = lib
        self._keep = []
        rp = np.ascontiguousarray(rowptr, dtype=np.int64) if isinstance(rowptr, np.ndarray) else rowptr
        cl = np.ascontiguousarray(col, dtype=np.int32) if isinstance(col, np.ndarray) else col
        vl = np.ascontiguousarray(val, dtype=np.float64) if isinstance(val, np.ndarray) else val
        ag = np.ascontiguousarray(agg, dtype=np.int32) if isinstance(agg, np.ndarray) else agg
        d1 = np.ascontiguousarray(D1, dtype=np.float64) if isinstance(D1, np.ndarray) else D1
        self._keep += [rp, cl, vl, ag, d1]
        prp, dev = _ptr(rp)
        csr = Csr(m=len(rp) - 1, n=int(n), nnz=int(len(vl)), rowptr=prp, col=_ptr(cl)[0], val=_ptr(vl)[0],
                  mem=DEVICE if dev else HOST)
        self.params = params(**kw)
        h = ctypes.c_void_p()
        _check(lib.amgdd_setup(ctypes.byref(csr), _ptr(d1)[0], _ptr(ag)[0], int(overlap), ctypes.byref(self.params),
                               _stream(stream), ctypes.byref(h)))
        self._h = h
        self.n = int(n)
        self._keep = []

    @classmethod
    def from_problem(cls, prob, overlap=1, **kw):
        return cls(prob.rowptr, prob.col, prob.val, prob.n, D1=prob.D1, agg=prob.agg, overlap=overlap, **kw)

    def save(self, path):
        """Write the setup inputs, parameters, kernel choices and every level's computed operators (amgdd_hierarchy_save)."""
        _check(self._lib.amgdd_hierarchy_save(self._h, str(path).encode()))

    @classmethod
    def load(cls, path, stream=None):
        """Restore a saved hierarchy: its levels as setup computed them, kernel choices replayed (amgdd_hierarchy_load)."""
        lib = load_library()
        h = ctypes.c_void_p()
        import torch

        st = _stream(stream) if (stream is not None or torch.cuda.is_available()) else None
        _check(lib.amgdd_hierarchy_load(str(path).encode(), st, ctypes.byref(h)))
        obj = cls.__new__(cls)
        obj._lib = lib
        obj._keep = []
        obj._h = h
        obj.n = int(obj.describe(0)["n"])
        obj.params = None
        return obj

    def close(self):
        if getattr(self, "_h", None):
            self._lib.amgdd_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- solve ----------------------------------------------------------------
    def set_precision(self, precision: int):
        _check(self._lib.amgdd_set_precision(self._h, int(precision)))

    def set_max_iter(self, max_iter: int):
        _check(self._lib.amgdd_set_max_iter(self._h, int(max_iter)))

    def solve(self, b, x=None, tol=1e-8, stream=None):
        """Solve A x = b (b: n or n x nrhs, column-major); returns (x, infos)."""
        nrhs = 1 if b.ndim == 1 else b.shape[1]
        if isinstance(b, np.ndarray):
            b = np.asfortranarray(b, dtype=np.float64)
            if x is None:
                x = np.zeros_like(b, order="F")
        else:
            import torch

            if nrhs > 1:
                # the C ABI takes column-major n x nrhs: pass (nrhs, n) row-major storage
                bc = b.t().contiguous()
                xc = torch.zeros_like(bc) if x is None else x.t().contiguous()
                infos = (Info * nrhs)()
                st = self._lib.amgdd_solve(self._h, _ptr(bc)[0], nrhs, float(tol), _ptr(xc)[0], _stream(stream),
                                           infos)
                if st not in (0, -4, -5, -3):
                    _check(st)
                if x is None:
                    x = xc.t()
                else:
                    x.copy_(xc.t())
                return x, [dict(iters=i.iters, status=i.status, relres=i.relres, relres_true=i.relres_true,
                                solve_ms=i.solve_ms, fallback=i.fallback, iters_mixed=i.iters_mixed)
                           for i in infos]
            assert b.is_contiguous()
            if x is None:
                x = torch.zeros_like(b)
        infos = (Info * nrhs)()
        st = self._lib.amgdd_solve(self._h, _ptr(b)[0], nrhs, float(tol), _ptr(x)[0], _stream(stream), infos)
        if st not in (0, -4, -5, -3):
            _check(st)
        return x, [dict(iters=i.iters, status=i.status, relres=i.relres, relres_true=i.relres_true,
                        solve_ms=i.solve_ms, fallback=i.fallback, iters_mixed=i.iters_mixed) for i in infos]

    def apply(self, op: int, level: int, x, y, stream=None):
        """y = op_l x on device FP64 tensors (see AMGDD_OP_*)."""
        _check(self._lib.amgdd_apply(self._h, int(op), int(level), _ptr(x)[0], _ptr(y)[0], _stream(stream)))

    # -- inspection -----------------------------------------------------------
    @property
    def num_levels(self) -> int:
        return self._lib.amgdd_num_levels(self._h)

    def describe(self, level: int) -> dict:
        d = LevelDesc()
        _check(self._lib.amgdd_level_describe(self._h, level, ctypes.byref(d)))
        return {f: getattr(d, f) for f, _ in LevelDesc._fields_}

    def export(self, level: int, which: int) -> np.ndarray:
        d = self.describe(level)
        nag = d["nagg"]
        size = {ARR_AGG: (d["n"], np.int32), ARR_OMEGA_PTR: (nag + 1, np.int64),
                ARR_OMEGA_IDX: (d["omega_len"], np.int32), ARR_NOMEGA: (nag, np.int32), ARR_K: (nag, np.int32),
                ARR_Z: (d["z_len"], np.float64), ARR_G_PTR: (d["ngroups"] + 1, np.int64),
                ARR_G_IDX: (d["g_sup_len"], np.int32), ARR_A_PTR: (d["n"] + 1, np.int64),
                ARR_A_IDX: (d["a_nnz"], np.int32), ARR_P_PTR: (d["n"] + 1, np.int64),
                ARR_P_IDX: (d["p_nnz"], np.int32)}
        if which == ARR_MU:
            cnt = int(self.export(level, ARR_NOMEGA).sum())
            size[ARR_MU] = (cnt, np.float64)
        cnt, dt = size[which]
        out = np.zeros(max(int(cnt), 1), dtype=dt)
        _check(self._lib.amgdd_level_export(self._h, level, which, out.ctypes.data, out.nbytes))
        return out[:cnt]

    def stats(self) -> dict:
        buf = ctypes.create_string_buffer(1 << 16)
        _check(self._lib.amgdd_hierarchy_stats(self._h, buf, len(buf)))
        return json.loads(buf.value.decode())

    def profile_vcycle(self, reps: int = 10, graph: bool = False):
        """Per (level, slot) mean device ms and algorithmic bytes of one V-cycle.

        graph=False: eager launches with events between them.  graph=True: the
        marked cycle replayed as a CUDA graph; also returns the mean ms of one
        replay of the unmarked cycle graph as a third value."""
        nl = self.num_levels
        cap = 8 * nl + 1
        ms = (ctypes.c_double * cap)()
        by = (ctypes.c_double * cap)()
        _check(self._lib.amgdd_profile_vcycle(self._h, int(reps), 1 if graph else 0, ms, by, cap))
        out = np.array(ms)[:8 * nl].reshape(nl, 8), np.array(by)[:8 * nl].reshape(nl, 8)
        return (*out, float(ms[8 * nl])) if graph else out

    def bytes_model(self):
        v, a = ctypes.c_double(), ctypes.c_double()
        _check(self._lib.amgdd_bytes_model(self._h, ctypes.byref(v), ctypes.byref(a)))
        return v.value, a.value

    def device_bytes(self, with_batched=False) -> int:
        """Device bytes held; with_batched: True for a batch of the hierarchy's batch_cols, or a column count."""
        return int(self._lib.amgdd_device_bytes(self._h, int(with_batched)))


class Server:
    """Continuous-batching solve server (amgdd_server_*): operators resident
    on the device within a byte budget, requests batched per operator."""

    def __init__(self, hbm_budget=None, slots=None, max_batch=None):
        self._lib = load_library()
        p = self._lib.amgdd_server_params_default()
        if hbm_budget is not None:
            p.hbm_budget = int(hbm_budget)
        if slots is not None:
            p.slots = int(slots)
        if max_batch is not None:
            p.max_batch = int(max_batch)
        self._s = ctypes.c_void_p()
        _check(self._lib.amgdd_server_create(ctypes.byref(p), ctypes.byref(self._s)))
        self._bufs = {}  # request id -> (b, x, nrhs) kept alive until polled

    def add_operator(self, prob, key: int, overlap: int = 1, **kw):
        """Build (or find, by key) the hierarchy of an inputs.Problem; returns (op id, cached)."""
        rowptr = np.ascontiguousarray(prob.rowptr, dtype=np.int64)
        col = np.ascontiguousarray(prob.col, dtype=np.int32)
        val = np.ascontiguousarray(prob.val, dtype=np.float64)
        agg = np.ascontiguousarray(prob.agg, dtype=np.int32)
        d1 = None if prob.D1 is None else np.ascontiguousarray(prob.D1, dtype=np.float64)
        csr = Csr(len(rowptr) - 1, prob.n, len(col), rowptr.ctypes.data, col.ctypes.data, val.ctypes.data, 0)
        prm = params(**kw)
        op, cached = ctypes.c_int64(), ctypes.c_int()
        _check(self._lib.amgdd_server_add_operator(self._s, int(key), ctypes.byref(csr), _ptr(d1)[0], agg.ctypes.data,
                                                   int(overlap), ctypes.byref(prm), ctypes.byref(op),
                                                   ctypes.byref(cached)))
        return op.value, bool(cached.value)

    def submit(self, op: int, b: np.ndarray, tol: float = 1e-8) -> int:
        """Queue a solve (b: n or n x nrhs host array); returns the request id."""
        b = np.asfortranarray(b, dtype=np.float64)
        nrhs = 1 if b.ndim == 1 else b.shape[1]
        x = np.zeros_like(b, order="F")
        rid = ctypes.c_int64()
        _check(self._lib.amgdd_server_submit(self._s, int(op), b.ctypes.data, nrhs, float(tol), x.ctypes.data,
                                             ctypes.byref(rid)))
        self._bufs[rid.value] = (b, x, nrhs)
        return rid.value

    def submit_problem(self, prob, key: int, b: np.ndarray, tol: float = 1e-8, overlap: int = 1, **kw):
        """Queue a solve that carries its operator (setup on the request path when `key` is not resident);
        returns (request id, cached)."""
        rowptr = np.ascontiguousarray(prob.rowptr, dtype=np.int64)
        col = np.ascontiguousarray(prob.col, dtype=np.int32)
        val = np.ascontiguousarray(prob.val, dtype=np.float64)
        agg = np.ascontiguousarray(prob.agg, dtype=np.int32)
        d1 = None if prob.D1 is None else np.ascontiguousarray(prob.D1, dtype=np.float64)
        csr = Csr(len(rowptr) - 1, prob.n, len(col), rowptr.ctypes.data, col.ctypes.data, val.ctypes.data, 0)
        prm = params(**kw)
        b = np.asfortranarray(b, dtype=np.float64)
        nrhs = 1 if b.ndim == 1 else b.shape[1]
        x = np.zeros_like(b, order="F")
        rid, cached = ctypes.c_int64(), ctypes.c_int()
        _check(self._lib.amgdd_server_submit_problem(self._s, int(key), ctypes.byref(csr), _ptr(d1)[0],
                                                     agg.ctypes.data, int(overlap), ctypes.byref(prm), b.ctypes.data,
                                                     nrhs, float(tol), x.ctypes.data, ctypes.byref(rid),
                                                     ctypes.byref(cached)))
        # the operator's inputs stay alive with the request (the library builds from them later)
        self._bufs[rid.value] = (b, x, nrhs, (rowptr, col, val, agg, d1, csr, prm))
        return rid.value, bool(cached.value)

    def poll(self, rid: int, wait_ms: int = -1):
        """None while pending; else (x, infos, latency_ms, status)."""
        b, x, nrhs = self._bufs[rid][:3]
        infos = (Info * nrhs)()
        lat = ctypes.c_double()
        st = self._lib.amgdd_server_poll(self._s, int(rid), int(wait_ms), infos, ctypes.byref(lat))
        if st == AMGDD_PENDING:
            return None
        del self._bufs[rid]
        if st not in (0, -4, -5, -3):
            _check(st)
        return x, [dict(iters=i.iters, status=i.status, relres=i.relres, relres_true=i.relres_true,
                        fallback=i.fallback) for i in infos], lat.value, st

    def stats(self) -> dict:
        buf = ctypes.create_string_buffer(4096)
        _check(self._lib.amgdd_server_stats(self._s, buf, len(buf)))
        return json.loads(buf.value.decode())

    def close(self):
        if self._s:
            self._lib.amgdd_server_destroy(self._s)
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
