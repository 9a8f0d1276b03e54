"""Thin Python binding of libpairgal (include/pairgal.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels. Device buffers are torch CUDA tensors (torch supplies memory and
streams); host buffers are numpy arrays. The functions keep the C names.
There is no fallback: if libpairgal.so is missing, importing this module
raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpairgal.so")

PG_OK, PG_ERR_INVALID_ARG, PG_ERR_UNSUPPORTED, PG_ERR_OOM, PG_ERR_CUDA, \
    PG_ERR_TIMEOUT, PG_ERR_UNIMPLEMENTED, PG_ERR_CAPACITY = range(8)


class PairgalError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


class pg_params(C.Structure):
    _fields_ = [
        ("box_L", C.c_double), ("mesh_n", C.c_int32), ("assign", C.c_int32),
        ("n_s", C.c_int32), ("s_edges", C.POINTER(C.c_double)), ("n_mu", C.c_int32),
        ("n_r", C.c_int32), ("r_edges", C.POINTER(C.c_double)), ("n_mur", C.c_int32),
        ("rsd_factor", C.c_double), ("r_perp_cut", C.c_double),
        ("precision", C.c_int32), ("bins_per_batch", C.c_int32),
        ("pair_grid", C.c_int32), ("par_edges", C.POINTER(C.c_double)),
    ]


_RESULT_FIELDS = [
    ("dd", "i8", "P"), ("dd_w", "f8", "P"), ("xi_ss", "f8", "P"), ("xi_pg", "f8", "PQ"),
    ("xi_gg", "f8", "Q"), ("b_pg", "f8", "PQ"), ("q_eff", "f8", "PQ"), ("q_eff_sq", "f8", "PQ"),
    ("xi_dw", "f8", "Q"), ("b_pg_agg", "f8", "P"), ("q_eff_agg", "f8", "P"),
    ("xi_dw_agg", "f8", "1"), ("n_cells", "i8", "Q"), ("n_cells_agg", "i8", "1"),
    ("sum_pg", "f8", "PQ"), ("sum_pg_agg", "f8", "P"), ("sum_gg", "f8", "Q"),
    ("sum2_gg", "f8", "Q"), ("sum_gg_agg", "f8", "2"), ("w_perp", "f8", "S"),
]


class pg_smooth_params(C.Structure):
    _fields_ = [("sigma", C.c_double), ("r_s", C.c_double), ("s0", C.c_double), ("r_cut", C.c_double)]


class pg_smooth_result(C.Structure):
    _fields_ = [("dd", C.POINTER(C.c_int64)), ("xi_ss", C.POINTER(C.c_double)),
                ("num", C.POINTER(C.c_double)), ("b_pg", C.POINTER(C.c_double)),
                ("q_eff", C.POINTER(C.c_double)), ("den", C.POINTER(C.c_double)),
                ("xi_dw", C.POINTER(C.c_double))]


class pg_mock(C.Structure):
    _fields_ = [("params", pg_params), ("n_gal", C.c_int64), ("h_pos", C.c_void_p),
                ("h_vel", C.c_void_p), ("h_w", C.c_void_p), ("out", C.c_void_p)]


class pg_batch_stats(C.Structure):
    _fields_ = [("wall_ms", C.c_double), ("mocks_per_s", C.c_double), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("n_plans", C.c_int32), ("n_workspaces", C.c_int32),
                ("gpu_launches", C.c_int64)]


class pg_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_int64), ("ms", C.c_double),
                ("bytes", C.c_double)]


PG_N_FAMILIES = 20


class pg_result(C.Structure):
    _fields_ = [(n, C.POINTER(C.c_int64) if t == "i8" else C.POINTER(C.c_double))
                for n, t, _ in _RESULT_FIELDS]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_1705_03464_gb300.build_lib.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    sig = {
        "pg_status_string": (C.c_char_p, [C.c_int]),
        "pg_plan_create": (C.c_int, [C.POINTER(pg_params), C.POINTER(vp)]),
        "pg_plan_create_shared": (C.c_int, [C.POINTER(pg_params), vp, C.POINTER(vp)]),
        "pg_run_batch": (C.c_int, [vp, i32, vp, vp, vp]),
        "pg_run_batch_streams": (C.c_int, [vp, i32, i32, vp, vp, vp]),
        "pg_selftest_wait": (C.c_int, [vp, C.c_double, vp]),
        "pg_forward_smooth": (C.c_int, [vp, vp, i64, vp, vp, vp, vp, vp]),
        "pg_backward_smooth": (C.c_int, [vp, vp, vp, vp]),
        "pg_autotune": (C.c_int, [C.POINTER(pg_params), i64, vp, vp, vp, vp, i32, vp, vp, vp]),
        "pg_plan_destroy": (None, [vp]),
        "pg_plan_reserve": (C.c_int, [vp, i64, i64]),
        "pg_workspace_bytes": (C.c_size_t, [vp]),
        "pg_forward": (C.c_int, [vp, i64, vp, vp, vp, C.POINTER(pg_result), vp]),
        "pg_forward_host": (C.c_int, [vp, i64, vp, vp, vp, C.POINTER(pg_result), vp]),
        "pg_correlate_points": (C.c_int, [vp, i64, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp]),
        "pg_transform_positions": (C.c_int, [i64, dbl, dbl, vp, vp, vp, vp]),
        "pg_find_pairs": (C.c_int, [vp, i64, vp, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp]),
        "pg_deposit_dense": (C.c_int, [i64, vp, vp, dbl, i32, i32, vp, vp]),
        "pg_deposit_lines": (C.c_int, [vp, i64, vp, vp, vp, i32, vp, vp, vp, vp]),
        "pg_fft_r2c_3d": (C.c_int, [vp, vp, vp, vp]),
        "pg_fft_c2r_3d": (C.c_int, [vp, vp, vp, vp]),
        "pg_pair_counts_static": (C.c_int, [i64, vp, vp, dbl, i32, vp, i32, vp, vp, vp]),
        "pg_backward": (C.c_int, [vp, C.POINTER(pg_result), vp, vp]),
        "pg_hod_weights": (C.c_int, [i64, vp, vp, vp, vp, vp, vp, vp]),
        "pg_hod_chain": (C.c_int, [vp, i64, vp, vp, vp, vp]),
        "pg_hod_weights2": (C.c_int, [i64, vp, vp, vp, vp, vp, vp, vp, vp]),
        "pg_hod_pair_derivs": (C.c_int, [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]),
        "pg_plan_set_profiling": (C.c_int, [vp, i32]),
        "pg_plan_last_stats": (C.c_int, [vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def exported_symbols():
    return [n for n in dir(_lib) if n.startswith("pg_")]


def status_string(s: int) -> str:
    return _lib.pg_status_string(int(s)).decode()


def _check(st, what):
    if st != PG_OK:
        raise PairgalError(st, what)


def _ptr(t):
    """Device/host address of a torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


_TORCH_DT = {"f64": "float64", "f32": "float32", "i64": "int64", "i32": "int32",
             "c64": "complex64", "c128": "complex128"}


def _dev(t, what, dtype, shape, device=None, optional=False):
    """Checks a device argument before its address goes to the library: a
    contiguous CUDA tensor of the given dtype ('f64', 'f32', ...) and shape
    (a tuple; None entries match any size), on `device` if given. The kernels
    read exactly the bytes the shape implies, so a wrong dtype, a strided
    view, a short array or a host tensor would make them read outside the
    buffer. Raises PairgalError(PG_ERR_INVALID_ARG) otherwise."""
    if t is None:
        if optional:
            return None
        raise PairgalError(PG_ERR_INVALID_ARG, f"{what} is required")
    import torch
    bad = None
    if not isinstance(t, torch.Tensor):
        bad = f"a torch tensor, got {type(t).__name__}"
    elif not t.is_cuda:
        bad = "a CUDA tensor"
    elif t.dtype != getattr(torch, _TORCH_DT[dtype]):
        bad = f"dtype {_TORCH_DT[dtype]}, got {t.dtype}"
    elif not t.is_contiguous():
        bad = "contiguous"
    elif t.dim() != len(shape) or any(w is not None and int(g) != int(w) for g, w in zip(t.shape, shape)):
        bad = f"shape {tuple('*' if w is None else w for w in shape)}, got {tuple(t.shape)}"
    elif device is not None and t.device != device:
        bad = f"on {device}, got {t.device}"
    if bad:
        raise PairgalError(PG_ERR_INVALID_ARG, f"{what} must be {bad}")
    return t


def _host_arr(a, what, dtype, shape, optional=False):
    """Host counterpart of _dev: a C-contiguous numpy array of the dtype (a
    copy is made if needed) and the given shape (None entries match any)."""
    if a is None:
        if optional:
            return None
        raise PairgalError(PG_ERR_INVALID_ARG, f"{what} is required")
    a = np.ascontiguousarray(a, dtype=dtype)
    if a.ndim != len(shape) or any(w is not None and g != w for g, w in zip(a.shape, shape)):
        raise PairgalError(PG_ERR_INVALID_ARG,
                           f"{what} must have shape {tuple('*' if w is None else w for w in shape)}, "
                           f"got {a.shape}")
    return a


def _catalogue(pos, vel, w):
    """Device catalogue checks shared by the forward entry points: pos [n, 3]
    float64, vel [n, 3] float32 or None, w [n] float32 or None, one device."""
    if pos is None:
        return 0
    _dev(pos, "pos", "f64", (None, 3))
    n = int(pos.shape[0])
    _dev(vel, "vel", "f32", (n, 3), pos.device, optional=True)
    _dev(w, "w", "f32", (n,), pos.device, optional=True)
    return n


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class Problem:
    """A pg_params with its edge arrays (kept alive here), and host output
    arrays laid out for it; no device state."""

    def __init__(self, box_L, mesh_n, assign, s_edges, n_mu, r_edges, n_mur,
                 rsd_factor=0.0, r_perp_cut=0.0, precision=0, bins_per_batch=0, par_edges=None):
        """par_edges given: the (d_perp, d_par) pair grid, s_edges the d_perp
        edges and par_edges the |d_par| edges (n_mu = len(par_edges) - 1)."""
        self.s_edges = np.ascontiguousarray(s_edges, dtype=np.float64)
        self.r_edges = np.ascontiguousarray(r_edges, dtype=np.float64)
        self.n_s = len(self.s_edges) - 1
        self.n_mu = int(n_mu)
        self.par_edges = None if par_edges is None else np.ascontiguousarray(par_edges, dtype=np.float64)
        if self.par_edges is not None and len(self.par_edges) - 1 != self.n_mu:
            raise ValueError("n_mu must be len(par_edges) - 1 on the (d_perp, d_par) grid")
        self.n_r = len(self.r_edges) - 1
        self.n_mur = int(n_mur)
        self.params = pg_params(
            float(box_L), int(mesh_n), int(assign), self.n_s,
            self.s_edges.ctypes.data_as(C.POINTER(C.c_double)), self.n_mu, self.n_r,
            self.r_edges.ctypes.data_as(C.POINTER(C.c_double)), self.n_mur,
            float(rsd_factor), float(r_perp_cut), int(precision), int(bins_per_batch),
            0 if self.par_edges is None else 1,
            None if self.par_edges is None else self.par_edges.ctypes.data_as(C.POINTER(C.c_double)))
        self.P = self.n_s * self.n_mu
        self.Q = self.n_r * self.n_mur

    @classmethod
    def of(cls, wl, **kw):
        args = dict(box_L=wl.box_L, mesh_n=wl.mesh_n, assign=wl.assign, s_edges=wl.s_edges,
                    n_mu=wl.n_mu, r_edges=wl.r_edges, n_mur=wl.n_mur,
                    rsd_factor=wl.rsd_factor, r_perp_cut=wl.r_perp_cut,
                    precision=wl.precision, bins_per_batch=wl.bins_per_batch)
        args.update(kw)
        return cls(**args)

    def new_result(self):
        """Host arrays for every pg_result field and the struct pointing at them."""
        P, Q = self.P, self.Q
        sizes = {"P": P, "Q": Q, "PQ": P * Q, "1": 1, "2": 2, "S": self.n_s}
        arrs = {}
        res = pg_result()
        for name, t, sz in _RESULT_FIELDS:
            a = np.full(sizes[sz], np.nan if t == "f8" else 0, dtype=np.float64 if t == "f8" else np.int64)
            arrs[name] = a
            ctype = C.c_int64 if t == "i8" else C.c_double
            setattr(res, name, a.ctypes.data_as(C.POINTER(ctype)))
        return res, arrs

    def shape_result(self, arrs):
        out = dict(arrs)
        for k in ("xi_pg", "b_pg", "q_eff", "q_eff_sq", "sum_pg"):
            out[k] = arrs[k].reshape(self.P, self.Q)
        out["xi_dw_agg"] = float(arrs["xi_dw_agg"][0])
        out["n_cells_agg"] = int(arrs["n_cells_agg"][0])
        return out


class Plan(Problem):
    """A pg_plan on the current CUDA device (pg_plan_create / pg_plan_destroy);
    with share_with, a plan that shares that plan's mesh scratch
    (pg_plan_create_shared)."""

    def __init__(self, box_L, mesh_n, assign, s_edges, n_mu, r_edges, n_mur,
                 rsd_factor=0.0, r_perp_cut=0.0, precision=0, bins_per_batch=0, share_with=None,
                 par_edges=None):
        super().__init__(box_L, mesh_n, assign, s_edges, n_mu, r_edges, n_mur, rsd_factor,
                         r_perp_cut, precision, bins_per_batch, par_edges)
        h = C.c_void_p()
        if share_with is None:
            _check(_lib.pg_plan_create(C.byref(self.params), C.byref(h)), "pg_plan_create")
        else:
            _check(_lib.pg_plan_create_shared(C.byref(self.params), share_with.handle, C.byref(h)),
                   "pg_plan_create_shared")
            self._donor = share_with   # keeps the donor's Python object alive
        self.handle = h

    @classmethod
    def of(cls, wl, **kw):
        args = dict(box_L=wl.box_L, mesh_n=wl.mesh_n, assign=wl.assign, s_edges=wl.s_edges,
                    n_mu=wl.n_mu, r_edges=wl.r_edges, n_mur=wl.n_mur,
                    rsd_factor=wl.rsd_factor, r_perp_cut=wl.r_perp_cut,
                    precision=wl.precision, bins_per_batch=wl.bins_per_batch)
        args.update(kw)
        return cls(**args)

    def close(self):
        if getattr(self, "handle", None):
            _lib.pg_plan_destroy(self.handle)
            self.handle = None
        self._donor = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self) -> int:
        return int(_lib.pg_workspace_bytes(self.handle))

    def set_profiling(self, on: bool):
        _check(_lib.pg_plan_set_profiling(self.handle, 1 if on else 0), "pg_plan_set_profiling")

    def last_stats(self):
        """Per kernel family of the last forward or backward call: launches, ms, bytes;
        plus the total number of kernel launches of that call."""
        arr = (pg_kernel_stat * PG_N_FAMILIES)()
        tot = C.c_int64(0)
        _check(_lib.pg_plan_last_stats(self.handle, arr, C.byref(tot)), "pg_plan_last_stats")
        fams = {a.name.decode(): {"launches": int(a.launches), "ms": float(a.ms), "bytes": float(a.bytes)}
                for a in arr}
        return fams, int(tot.value)

    def reserve(self, n_gal_max, n_pairs_max):
        _check(_lib.pg_plan_reserve(self.handle, int(n_gal_max), int(n_pairs_max)), "pg_plan_reserve")



def pg_forward(plan: Plan, pos, vel=None, w=None, stream=None):
    """Full forward path on device tensors: pos [n,3] float64, vel [n,3]
    float32 or None, w [n] float32 or None. Returns host numpy outputs."""
    n = _catalogue(pos, vel, w)
    res, arrs = plan.new_result()
    st = _lib.pg_forward(plan.handle, n, _ptr(pos), _ptr(vel), _ptr(w), C.byref(res), _stream(stream))
    _check(st, "pg_forward")
    return plan.shape_result(arrs)


def pg_forward_host(plan: Plan, pos: np.ndarray, vel=None, w=None, stream=None):
    """Full forward path from host (preferably pinned) arrays: pos [n, 3]
    float64, vel [n, 3] float32 or None, w [n] float32 or None (converted
    to those types if needed)."""
    pos = _host_arr(pos, "pos", np.float64, (None, 3))
    n = int(pos.shape[0])
    vel = _host_arr(vel, "vel", np.float32, (n, 3), optional=True)
    w = _host_arr(w, "w", np.float32, (n,), optional=True)
    res, arrs = plan.new_result()
    st = _lib.pg_forward_host(plan.handle, n, _ptr(pos), _ptr(vel), _ptr(w), C.byref(res), _stream(stream))
    _check(st, "pg_forward_host")
    return plan.shape_result(arrs)


def pg_transform_positions(pos, box_L, rsd_factor=0.0, vel=None, out=None, stream=None):
    import torch
    _dev(pos, "pos", "f64", (None, 3))
    _dev(vel, "vel", "f32", (pos.shape[0], 3), pos.device, optional=True)
    if out is None:
        out = torch.empty_like(pos)
    _dev(out, "out", "f64", tuple(pos.shape), pos.device)
    _check(_lib.pg_transform_positions(int(pos.shape[0]), float(box_L), float(rsd_factor),
                                       _ptr(pos), _ptr(vel), _ptr(out), _stream(stream)),
           "pg_transform_positions")
    return out


def pg_find_pairs(plan: Plan, pos, w=None, with_list=True, stream=None):
    """Pairs of wrapped device positions: counts (and the bin-grouped list)."""
    import torch
    n = _catalogue(pos, None, w)
    dev = pos.device
    dd = torch.zeros(plan.P, dtype=torch.int64, device=dev)
    ddq = torch.zeros(plan.P, dtype=torch.int64, device=dev)
    npairs = C.c_int64(0)
    st = _lib.pg_find_pairs(plan.handle, n, _ptr(pos), _ptr(w), _ptr(dd), _ptr(ddq), 0,
                            None, None, None, None, None, C.byref(npairs), _stream(stream))
    _check(st, "pg_find_pairs")
    out = {"dd": dd, "ddq": ddq, "n_pairs": int(npairs.value)}
    if not with_list:
        return out
    cap = max(1, out["n_pairs"])
    b = torch.empty(cap, dtype=torch.int32, device=dev)
    i = torch.empty(cap, dtype=torch.int32, device=dev)
    j = torch.empty(cap, dtype=torch.int32, device=dev)
    mid = torch.empty((cap, 3), dtype=torch.float64, device=dev)
    wp = torch.empty(cap, dtype=torch.float64, device=dev)
    st = _lib.pg_find_pairs(plan.handle, n, _ptr(pos), _ptr(w), _ptr(dd), _ptr(ddq), cap,
                            _ptr(b), _ptr(i), _ptr(j), _ptr(mid), _ptr(wp), C.byref(npairs),
                            _stream(stream))
    _check(st, "pg_find_pairs")
    m = int(npairs.value)
    out.update({"bin": b[:m], "i": i[:m], "j": j[:m], "mid": mid[:m], "weight": wp[:m]})
    return out


def pg_deposit_dense(pos, w, box_L, mesh_n, assign, mesh=None, stream=None):
    import torch
    _dev(pos, "pos", "f64", (None, 3))
    _dev(w, "w", "f64", (pos.shape[0],), pos.device, optional=True)
    if mesh is None:
        mesh = torch.zeros((mesh_n, mesh_n, mesh_n), dtype=torch.int64, device=pos.device)
    _dev(mesh, "mesh", "i64", (mesh_n, mesh_n, mesh_n), pos.device)
    _check(_lib.pg_deposit_dense(int(pos.shape[0]), _ptr(pos), _ptr(w), float(box_L), int(mesh_n),
                                 int(assign), _ptr(mesh), _stream(stream)), "pg_deposit_dense")
    return mesh


def pg_deposit_lines(plan: Plan, pos, w=None, bins=None, nb=1, stream=None):
    """The forward path's compact-line deposit (pg_deposit_lines) of device
    points pos [n, 3] float64 with weights w [n] float64 or None into nb
    meshes (bins [n] int32 in [0, nb), or None for one mesh). Returns the
    dense int64 meshes [nb, N, N, N] (device), the totals [nb] and the
    touched-line count."""
    import torch
    _dev(pos, "pos", "f64", (None, 3))
    n = int(pos.shape[0])
    _dev(w, "w", "f64", (n,), pos.device, optional=True)
    _dev(bins, "bins", "i32", (n,), pos.device, optional=True)
    N = int(plan.params.mesh_n)
    mesh = torch.empty((int(nb), N, N, N), dtype=torch.int64, device=pos.device)
    qsum = np.zeros(int(nb), dtype=np.int64)
    nl = C.c_int64(0)
    _check(_lib.pg_deposit_lines(plan.handle, n, _ptr(pos), _ptr(w), _ptr(bins), int(nb), _ptr(mesh),
                                 qsum.ctypes.data, C.byref(nl), _stream(stream)), "pg_deposit_lines")
    return mesh, qsum, int(nl.value)


def pg_fft_r2c_3d(plan: Plan, f, out=None, stream=None):
    import torch
    N = int(plan.params.mesh_n)
    dbl = plan.params.precision == 1
    _dev(f, "f", "f64" if dbl else "f32", (N, N, N))
    cdt = torch.complex128 if dbl else torch.complex64
    if out is None:
        out = torch.empty((N, N, N // 2 + 1), dtype=cdt, device=f.device)
    _dev(out, "out", "c128" if dbl else "c64", (N, N, N // 2 + 1), f.device)
    _check(_lib.pg_fft_r2c_3d(plan.handle, _ptr(f), _ptr(out), _stream(stream)), "pg_fft_r2c_3d")
    return out


def pg_fft_c2r_3d(plan: Plan, F, out=None, stream=None):
    import torch
    N = int(plan.params.mesh_n)
    dbl = plan.params.precision == 1
    _dev(F, "F", "c128" if dbl else "c64", (N, N, N // 2 + 1))
    rdt = torch.float64 if dbl else torch.float32
    if out is None:
        out = torch.empty((N, N, N), dtype=rdt, device=F.device)
    _dev(out, "out", "f64" if dbl else "f32", (N, N, N), F.device)
    _check(_lib.pg_fft_c2r_3d(plan.handle, _ptr(F), _ptr(out), _stream(stream)), "pg_fft_c2r_3d")
    return out


def pg_correlate_points(plan: Plan, pts_a, w_a, pts_b, w_b, stream=None):
    """Two device point sets [n, 3] float64 (inside [0, L)) with float64
    weights [n] or None: binned sums of C_ab (pg_correlate_points)."""
    _dev(pts_a, "pts_a", "f64", (None, 3))
    _dev(w_a, "w_a", "f64", (pts_a.shape[0],), pts_a.device, optional=True)
    _dev(pts_b, "pts_b", "f64", (None, 3), pts_a.device)
    _dev(w_b, "w_b", "f64", (pts_b.shape[0],), pts_a.device, optional=True)
    Q = plan.Q
    s1 = np.zeros(Q)
    s2 = np.zeros(Q)
    agg = np.zeros(2)
    nc = np.zeros(Q, dtype=np.int64)
    st = _lib.pg_correlate_points(plan.handle, int(pts_a.shape[0]), _ptr(pts_a), _ptr(w_a),
                                  int(pts_b.shape[0]), _ptr(pts_b), _ptr(w_b), _ptr(s1), _ptr(s2),
                                  _ptr(agg), _ptr(nc), _stream(stream))
    _check(st, "pg_correlate_points")
    return {"sum": s1, "sum2": s2, "agg": agg, "n_cells": nc}


def pg_pair_counts_static(pos, w, box_L, s_edges, n_mu, stream=None):
    """Pair counts (dd, ddq) from the allocation-free entry point; the call
    itself allocates no device memory (the two output tensors are created
    here, by torch, before the call)."""
    import torch
    _catalogue(pos, None, w)
    edges = np.ascontiguousarray(s_edges, dtype=np.float64)
    P = (len(edges) - 1) * int(n_mu)
    dd = torch.empty(P, dtype=torch.int64, device=pos.device)
    ddq = torch.empty(P, dtype=torch.int64, device=pos.device)
    st = _lib.pg_pair_counts_static(int(pos.shape[0]), _ptr(pos), _ptr(w), float(box_L),
                                    len(edges) - 1, _ptr(edges), int(n_mu), _ptr(dd), _ptr(ddq),
                                    _stream(stream))
    _check(st, "pg_pair_counts_static")
    return dd, ddq


GRAD_FIELDS = ("xi_pg", "xi_gg", "b_pg", "q_eff", "q_eff_sq", "xi_dw", "b_pg_agg", "q_eff_agg",
               "xi_dw_agg", "xi_ss", "dd_w", "w_perp")


def pg_backward(plan: Plan, grads: dict, n_gal: int, stream=None):
    """dL/dw (device FP64 tensor [n_gal]) of the last pg_forward on `plan`,
    for L = sum over the given fields of grads[field] * output[field]."""
    import torch
    res = pg_result()
    keep = []
    for name in GRAD_FIELDS:
        if name in grads and grads[name] is not None:
            a = np.ascontiguousarray(np.asarray(grads[name], dtype=np.float64).reshape(-1))
            keep.append(a)
            setattr(res, name, a.ctypes.data_as(C.POINTER(C.c_double)))
    out = torch.empty(max(int(n_gal), 1), dtype=torch.float64, device="cuda")
    st = _lib.pg_backward(plan.handle, C.byref(res), _ptr(out), _stream(stream))
    _check(st, "pg_backward")
    return out[: int(n_gal)]


class PairGalFn:
    """torch.autograd.Function over the library: forward = pg_forward with the
    given per-galaxy weights, backward = pg_backward (spectra recomputed).

        outs = PairGalFn.apply(w, plan, pos, vel)   # w: [n] float32 CUDA, requires_grad
    returns (b_pg, q_eff, xi_pg, xi_gg, b_pg_agg, q_eff_agg) as FP64 tensors on w's device."""

    NAMES = ("b_pg", "q_eff", "xi_pg", "xi_gg", "b_pg_agg", "q_eff_agg")

    @staticmethod
    def _fn():
        import torch

        class _F(torch.autograd.Function):
            @staticmethod
            def forward(ctx, w, plan, pos, vel):
                out = pg_forward(plan, pos, vel, w)
                ctx.plan = plan
                ctx.n = int(pos.shape[0])
                ctx.shapes = [out[k].shape for k in PairGalFn.NAMES]
                return tuple(torch.as_tensor(np.ascontiguousarray(out[k]), dtype=torch.float64,
                                             device=w.device) for k in PairGalFn.NAMES)

            @staticmethod
            def backward(ctx, *gouts):
                grads = {k: (g.detach().cpu().numpy() if g is not None else None)
                         for k, g in zip(PairGalFn.NAMES, gouts)}
                gw = pg_backward(ctx.plan, grads, ctx.n)
                return gw.to(torch.float32), None, None, None

        return _F

    @classmethod
    def apply(cls, w, plan, pos, vel=None):
        if not hasattr(cls, "_F"):
            cls._F = cls._fn()
        return cls._F.apply(w, plan, pos, vel)


def pg_hod_weights(mass, kind, kh, theta, with_grad=True, stream=None):
    """Soft HOD weights w [n] FP32 and dw/dtheta [n, 5] FP64 (device tensors)."""
    import torch
    _dev(mass, "mass", "f64", (None,))
    n = int(mass.shape[0])
    _dev(kind, "kind", "i32", (n,), mass.device)
    _dev(kh, "kh", "f32", (n,), mass.device)
    th = _host_arr(theta, "theta", np.float64, (5,))
    w = torch.empty(max(n, 1), dtype=torch.float32, device=mass.device)
    dw = torch.empty((max(n, 1), 5), dtype=torch.float64, device=mass.device) if with_grad else None
    _check(_lib.pg_hod_weights(n, _ptr(mass), _ptr(kind), _ptr(kh), _ptr(th), _ptr(w), _ptr(dw),
                               _stream(stream)), "pg_hod_weights")
    return w[:n], (dw[:n] if dw is not None else None)


def pg_hod_weights2(mass, kind, kh, theta, stream=None):
    """Soft HOD weights w [n] FP32, dw/dtheta [n, 5] and d2w/dtheta2
    [n, 5, 5] FP64 (device tensors; the last expanded from the library's
    upper triangle)."""
    import torch
    _dev(mass, "mass", "f64", (None,))
    n = int(mass.shape[0])
    _dev(kind, "kind", "i32", (n,), mass.device)
    _dev(kh, "kh", "f32", (n,), mass.device)
    th = _host_arr(theta, "theta", np.float64, (5,))
    m = max(n, 1)
    w = torch.empty(m, dtype=torch.float32, device=mass.device)
    dw = torch.empty((m, 5), dtype=torch.float64, device=mass.device)
    d2 = torch.empty((m, 15), dtype=torch.float64, device=mass.device)
    _check(_lib.pg_hod_weights2(n, _ptr(mass), _ptr(kind), _ptr(kh), _ptr(th), _ptr(w), _ptr(dw),
                                _ptr(d2), _stream(stream)), "pg_hod_weights2")
    return w[:n], dw[:n], _tri_to_full(d2[:n])


_TRI = [(j, k) for j in range(5) for k in range(j, 5)]


def _tri_to_full(t):
    """[..., 15] upper triangle (row order) -> [..., 5, 5] symmetric."""
    import torch
    lib = torch if not isinstance(t, np.ndarray) else np
    if lib is np:
        out = np.zeros(t.shape[:-1] + (5, 5))
    else:
        out = torch.zeros(tuple(t.shape[:-1]) + (5, 5), dtype=t.dtype, device=t.device)
    for q, (j, k) in enumerate(_TRI):
        out[..., j, k] = t[..., q]
        out[..., k, j] = t[..., q]
    return out


def _full_to_tri(h):
    import torch
    idx_j = [j for j, _ in _TRI]
    idx_k = [k for _, k in _TRI]
    if isinstance(h, np.ndarray):
        return np.ascontiguousarray(h[..., idx_j, idx_k])
    return h[..., idx_j, idx_k].contiguous()


def pg_hod_pair_derivs(plan: Plan, pos, vel, w, dw, d2w, stream=None):
    """Exact HOD-parameter derivatives of xi per pair bin (and of w(d_perp)
    on the grid): pg_hod_pair_derivs on device tensors pos [n, 3] float64,
    vel [n, 3] float32 or None, w [n] float32, dw [n, 5] float64 and d2w
    [n, 5, 5] (or [n, 15]) float64. Returns host arrays xi [P], dxi [P, 5],
    d2xi [P, 5, 5] and w_perp [n_s], dw_perp [n_s, 5], d2w_perp [n_s, 5, 5]."""
    n = _catalogue(pos, vel, w)
    if w is None:
        raise PairgalError(PG_ERR_INVALID_ARG, "w is required")
    _dev(dw, "dw", "f64", (n, 5), pos.device)
    if d2w is not None and d2w.dim() == 3:
        d2w = _full_to_tri(d2w)
    _dev(d2w, "d2w", "f64", (n, 15), pos.device)
    xi = np.zeros((plan.P, 21))
    wp = np.zeros((plan.n_s, 21))
    _check(_lib.pg_hod_pair_derivs(plan.handle, n, _ptr(pos), _ptr(vel), _ptr(w), _ptr(dw), _ptr(d2w),
                                   xi.ctypes.data, wp.ctypes.data, _stream(stream)), "pg_hod_pair_derivs")
    return {"xi": xi[:, 0], "dxi": xi[:, 1:6], "d2xi": _tri_to_full(xi[:, 6:]),
            "w_perp": wp[:, 0], "dw_perp": wp[:, 1:6], "d2w_perp": _tri_to_full(wp[:, 6:])}


def pg_hod_chain(plan: Plan, wbar, dw, stream=None):
    _dev(wbar, "wbar", "f64", (None,))
    _dev(dw, "dw", "f64", (wbar.shape[0], 5), wbar.device)
    out = np.zeros(5)
    _check(_lib.pg_hod_chain(plan.handle, int(wbar.shape[0]), _ptr(wbar), _ptr(dw), _ptr(out),
                             _stream(stream)), "pg_hod_chain")
    return out


def hod_gradient(plan: Plan, pos, vel, mass, kind, kh, theta, grads, stream=None):
    """Outputs at HOD parameters theta and dL/dtheta for L = sum grads * outputs:
    soft weights -> pg_forward -> pg_backward -> chain, all on the device."""
    w, dw = pg_hod_weights(mass, kind, kh, theta, True, stream)
    out = pg_forward(plan, pos, vel, w, stream)
    wbar = pg_backward(plan, grads, int(pos.shape[0]), stream)
    return out, pg_hod_chain(plan, wbar, dw, stream)


def hod_gradient_smooth(plan: Plan, w_params, pos, vel, mass, kind, kh, theta, grads, stream=None):
    """The smooth-W estimator's outputs at HOD parameters theta and dL/dtheta
    for L = sum grads * outputs: soft weights -> pg_forward_smooth ->
    pg_backward_smooth -> chain, all on the device."""
    w, dw = pg_hod_weights(mass, kind, kh, theta, True, stream)
    out = pg_forward_smooth(plan, w_params, pos, vel, w, stream)
    wbar = pg_backward_smooth(plan, grads, int(pos.shape[0]), stream)
    return out, pg_hod_chain(plan, wbar, dw, stream)


def _host(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def pg_run_batch(problems, catalogues, stream=None, n_streams=1, _streams_entry=False):
    """Many mocks through the forward path: problems[i] a Problem (or Plan),
    catalogues[i] = (pos [n,3] float64, vel [n,3] float32 or None, w [n]
    float32 or None), host arrays. n_streams = 1: pg_run_batch (one stream,
    plans built ahead); > 1: pg_run_batch_streams (runners on their own
    streams claiming mocks from one work queue). Returns (outputs per mock,
    latency_ms per mock, stats dict)."""
    n = len(problems)
    if len(catalogues) != n:
        raise ValueError("one catalogue per problem")
    mocks = (pg_mock * max(n, 1))()
    keep, results = [], []
    for i, (pr, cat) in enumerate(zip(problems, catalogues)):
        pos, vel, w = (tuple(cat) + (None, None))[:3]
        pos, vel, w = _host(pos, np.float64), _host(vel, np.float32), _host(w, np.float32)
        res, arrs = pr.new_result()
        keep += [pos, vel, w, res]
        results.append(arrs)
        m = mocks[i]
        m.params = pr.params
        m.n_gal = int(pos.shape[0])
        m.h_pos = pos.ctypes.data
        m.h_vel = None if vel is None else vel.ctypes.data
        m.h_w = None if w is None else w.ctypes.data
        m.out = C.addressof(res)
    lat = np.full(max(n, 1), np.nan)
    st = pg_batch_stats()
    if n_streams == 1 and not _streams_entry:
        _check(_lib.pg_run_batch(C.addressof(mocks), n, lat.ctypes.data, C.byref(st), _stream(stream)),
               "pg_run_batch")
    else:
        _check(_lib.pg_run_batch_streams(C.addressof(mocks), n, int(n_streams), lat.ctypes.data, C.byref(st),
                                         _stream(stream)), "pg_run_batch_streams")
    stats = {k: getattr(st, k) for k, _ in pg_batch_stats._fields_}
    return [pr.shape_result(a) for pr, a in zip(problems, results)], lat[:n], stats


def pg_run_batch_streams(problems, catalogues, n_streams=2, stream=None):
    """pg_run_batch_streams: the batch through n_streams runner threads, each
    on its own stream, claiming mocks from one work queue (same returns as
    pg_run_batch; the outputs are bit-identical to it)."""
    return pg_run_batch(problems, catalogues, stream=stream, n_streams=int(n_streams), _streams_entry=True)


def pg_autotune(problem, pos, vel=None, w=None, candidates=(4, 8, 16, 32), stream=None):
    """Batch-size autotuner (pg_autotune) on host arrays: returns (best
    bins_per_batch, {candidate: ms})."""
    pos, vel, w = _host(pos, np.float64), _host(vel, np.float32), _host(w, np.float32)
    cand = np.ascontiguousarray(candidates, dtype=np.int32)
    ms = np.zeros(len(cand))
    best = C.c_int32(0)
    _check(_lib.pg_autotune(C.byref(problem.params), int(pos.shape[0]), pos.ctypes.data,
                            None if vel is None else vel.ctypes.data,
                            None if w is None else w.ctypes.data, cand.ctypes.data, len(cand),
                            C.byref(best), ms.ctypes.data, _stream(stream)), "pg_autotune")
    return int(best.value), {int(c): float(t) for c, t in zip(cand, ms)}


def autotune_cached(problem, pos, vel=None, w=None, cache_path=None, candidates=(4, 8, 16, 32),
                    stream=None):
    """pg_autotune with its result cached in a JSON file keyed by mesh size,
    precision and device name (cache_path, or the PG_TUNE_CACHE environment
    variable; no caching if neither is set)."""
    import json
    path = cache_path or os.environ.get("PG_TUNE_CACHE")
    key = None
    try:
        import torch
        dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "none"
    except Exception:
        dev = "unknown"
    key = f"N{problem.params.mesh_n}-p{problem.params.precision}-{dev}"
    table = {}
    if path and os.path.exists(path):
        with open(path) as f:
            table = json.load(f)
    if key in table:
        return int(table[key]["bins_per_batch"]), table[key].get("ms", {})
    best, ms = pg_autotune(problem, pos, vel, w, candidates, stream)
    if path:
        table[key] = {"bins_per_batch": best, "ms": ms}
        with open(path, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
    return best, ms


def pg_selftest_wait(plan: Plan, limit_ms: float, stream=None) -> int:
    """Failure-detection test of the bounded device waits: returns the status
    (PG_ERR_TIMEOUT when the wait gave up, the expected outcome)."""
    return int(_lib.pg_selftest_wait(plan.handle, float(limit_ms), _stream(stream)))


# Table tab:weightings: (sigma, r_s, s0, r_cut) for d_p,max = 10 and 30 Mpc/h
W_DP10 = (30.0, 20.0, 0.8, 10.0)
W_DP30 = (50.0, 35.0, 0.5, 20.0)


def pg_forward_smooth(plan: Plan, w_params, pos, vel=None, w=None, stream=None):
    """The paper's own smooth-W estimator (pg_forward_smooth) on device
    tensors; w_params = (sigma, r_s, s0, r_cut). Returns host numpy outputs
    per (s, mu) pair bin plus den and xi_dw."""
    n = _catalogue(pos, vel, w)
    P = plan.P
    arrs = {"dd": np.zeros(P, np.int64), "xi_ss": np.full(P, np.nan), "num": np.full(P, np.nan),
            "b_pg": np.full(P, np.nan), "q_eff": np.full(P, np.nan), "den": np.full(1, np.nan),
            "xi_dw": np.full(1, np.nan)}
    res = pg_smooth_result(*[arrs[k].ctypes.data_as(C.POINTER(C.c_int64 if k == "dd" else C.c_double))
                             for k, _ in pg_smooth_result._fields_])
    prm = pg_smooth_params(*[float(v) for v in w_params])
    _check(_lib.pg_forward_smooth(plan.handle, C.byref(prm), n, _ptr(pos), _ptr(vel), _ptr(w),
                                  C.byref(res), _stream(stream)), "pg_forward_smooth")
    out = dict(arrs)
    out["den"] = float(arrs["den"][0])
    out["xi_dw"] = float(arrs["xi_dw"][0])
    return out


SMOOTH_GRAD_FIELDS = ("xi_ss", "num", "b_pg", "q_eff", "den", "xi_dw")


def pg_backward_smooth(plan: Plan, grads: dict, n_gal: int, stream=None):
    """dL/dw (device FP64 tensor [n_gal]) of the last pg_forward_smooth on
    `plan`, for L = sum over the given fields of grads[field] * output[field]."""
    import torch
    res = pg_smooth_result()
    keep = []
    for name in SMOOTH_GRAD_FIELDS:
        if name in grads and grads[name] is not None:
            a = np.ascontiguousarray(np.asarray(grads[name], dtype=np.float64).reshape(-1))
            keep.append(a)
            setattr(res, name, a.ctypes.data_as(C.POINTER(C.c_double)))
    out = torch.empty(max(int(n_gal), 1), dtype=torch.float64, device="cuda")
    _check(_lib.pg_backward_smooth(plan.handle, C.byref(res), _ptr(out), _stream(stream)), "pg_backward_smooth")
    return out[: int(n_gal)]
