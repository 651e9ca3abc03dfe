"""GB300 boundary-integral Poisson-Boltzmann solver with polarizable multipoles.

A thin binding over the C ABI of ``libbempol.so`` (see ``include/bempol.h``):
argument marshalling only, every step of the computation runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams.

The shared library is built in-tree by ``paper_1810_03698_gb300.build``; importing
this package without it raises ImportError (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbempol.so")

HOST, DEVICE = 0, 1
OP_FP64_DIRECT, OP_FP32_DIRECT, OP_FP32_TREE, OP_FP64_TREE = 0, 1, 2, 3
OP_NAMES = {"fp64_direct": 0, "fp32_direct": 1, "fp32_tree": 2, "fp64_tree": 3}
REFINE_EVERY, REFINE_FINAL = 0, 1
REFINE_NAMES = {"every": 0, "final": 1}
NEAR_RULES = {"semi_analytical": 0, "exact": 0, "gauss19": 19}

STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_MESH", 3: "ERR_SITES", 4: "ERR_NOT_CONVERGED", 5: "ERR_CUDA",
          6: "ERR_TIMEOUT", 7: "ERR_OOM", 8: "ERR_STATE"}


class Params(C.Structure):
    _fields_ = [
        ("eps_in", C.c_double), ("eps_out", C.c_double), ("kappa", C.c_double),
        ("gauss_k", C.c_int), ("near_factor", C.c_double),
        ("theta", C.c_double), ("order", C.c_int), ("leaf", C.c_int),
        ("gmres_tol", C.c_double), ("gmres_restart", C.c_int), ("gmres_maxit", C.c_int),
        ("scf_tol", C.c_double), ("sor_omega", C.c_double), ("scf_maxit", C.c_int),
        ("op", C.c_int), ("residual_op", C.c_int), ("inner_tol", C.c_double), ("refine_maxit", C.c_int),
        ("thole_a", C.c_double), ("refine_scope", C.c_int), ("thole_perm", C.c_int), ("near_rule", C.c_int),
    ]


class Result(C.Structure):
    _fields_ = [
        ("dG_solv_kcal", C.c_double), ("G_diss", C.c_double), ("G_vac", C.c_double),
        ("scf_iters_diss", C.c_int), ("scf_iters_vac", C.c_int), ("gmres_iters_total", C.c_int),
        ("matvecs_total", C.c_int), ("n_solves", C.c_int), ("last_rel_residual", C.c_double),
        ("t_setup_ms", C.c_double), ("t_scf_ms", C.c_double), ("t_total_ms", C.c_double),
        ("phi", C.c_void_p), ("dphidn", C.c_void_p), ("site_reaction", C.c_void_p),
        ("mu_diss", C.c_void_p), ("mu_vac", C.c_void_p), ("where", C.c_int), ("residual_matvecs", C.c_int),
    ]


class SystemResult(C.Structure):
    _fields_ = [
        ("dG_solv_kcal", C.c_double), ("G_diss", C.c_double), ("G_vac", C.c_double),
        ("scf_iters_diss", C.c_int), ("scf_iters_vac", C.c_int), ("gmres_iters", C.c_int),
        ("n_solves", C.c_int), ("last_rel_residual", C.c_double), ("converged", C.c_int),
        ("n_panels", C.c_int64), ("n_sites", C.c_int64),
    ]


class GradientInfo(C.Structure):
    _fields_ = [
        ("scf_iters_diss", C.c_int), ("scf_iters_vac", C.c_int), ("gmres_iters_total", C.c_int),
        ("n_solves", C.c_int), ("converged", C.c_int), ("t_ms", C.c_double),
    ]


class TuneResult(C.Structure):
    _fields_ = [("leaf", C.c_int), ("theta", C.c_double), ("order", C.c_int), ("matvec_ms", C.c_double),
                ("rel_err", C.c_double), ("candidates", C.c_int)]


class Stats(C.Structure):
    _fields_ = [
        ("kernel_launches", C.c_int64), ("pair_launches", C.c_int64), ("pair_ms", C.c_double),
        ("far_launches", C.c_int64), ("far_ms", C.c_double), ("pair_interactions", C.c_int64),
        ("far_evaluations", C.c_int64), ("tree_products", C.c_int64), ("tree_ms", C.c_double),
        ("rhs_calls", C.c_int64), ("rhs_ms", C.c_double), ("reaction_calls", C.c_int64), ("reaction_ms", C.c_double),
        ("site_field_calls", C.c_int64), ("site_field_ms", C.c_double),
        ("mesh_validate_ms", C.c_double), ("mesh_geometry_ms", C.c_double), ("mesh_blocks_ms", C.c_double),
        ("mesh_tree_ms", C.c_double), ("mesh_near_ms", C.c_double),
        ("tree64_products", C.c_int64), ("tree64_ms", C.c_double),
    ]


class Peaks(C.Structure):
    _fields_ = [("fp32_fma_tflops", C.c_double), ("fp64_fma_tflops", C.c_double), ("mufu_rsqrt_gops", C.c_double),
                ("mufu_ex2_gops", C.c_double), ("ms_fp32", C.c_double), ("ms_fp64", C.c_double),
                ("ms_rsqrt", C.c_double), ("ms_ex2", C.c_double), ("sm_count", C.c_int),
                ("clock_mhz_attr", C.c_double)]


# exchange callback of a sharded context: (user, stream) -> None
ExchangeFn = C.CFUNCTYPE(None, C.c_void_p, C.POINTER(C.c_int64), C.c_int, C.c_void_p)


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1810_03698_gb300.build`")
    lib = C.CDLL(LIB_PATH)
    vp, i64, i32, dp = C.c_void_p, C.c_int64, C.c_int, C.c_double
    sig = {
        "bempol_default_params": (None, [C.POINTER(Params)]),
        "bempol_create": (i32, [C.POINTER(Params), i32, C.POINTER(vp)]),
        "bempol_set_params": (i32, [vp, C.POINTER(Params)]),
        "bempol_destroy": (None, [vp]),
        "bempol_last_error": (C.c_char_p, [vp]),
        "bempol_set_mesh": (i32, [vp, i64, vp, i64, vp, i32, vp]),
        "bempol_set_sites": (i32, [vp, i64, vp, vp, vp, vp, vp, vp, i32, vp]),
        "bempol_set_mesh_systems": (i32, [vp, i64, vp, i64, vp, vp, vp, i32, vp]),
        "bempol_set_mesh_stern": (i32, [vp, i64, vp, i64, vp, i64, vp, i64, vp, i32, vp]),
        "bempol_set_sites_systems": (i32, [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, i32, vp]),
        "bempol_systems": (i32, [vp, C.POINTER(i64), C.POINTER(i64)]),
        "bempol_solve": (i32, [vp, vp, C.POINTER(Result)]),
        "bempol_solve_systems": (i32, [vp, vp, C.POINTER(Result), C.POINTER(SystemResult), i64]),
        "bempol_matvec": (i32, [vp, vp, vp, i32, vp]),
        "bempol_matvec_transposed": (i32, [vp, vp, vp, i32, vp]),
        "bempol_autotune": (i32, [vp, dp, C.POINTER(TuneResult), vp]),
        "bempol_gradient": (i32, [vp, vp, vp, vp, vp, vp, C.POINTER(GradientInfo), i32]),
        "bempol_rhs": (i32, [vp, vp, vp, i32, vp]),
        "bempol_site_reaction": (i32, [vp, vp, vp, i32, vp]),
        "bempol_site_reaction_noalloc": (i32, [vp, vp, vp, i32, vp]),
        "bempol_multipole_field": (i32, [vp, vp, i32, vp, vp]),
        "bempol_sizes": (i32, [vp, C.POINTER(i64), C.POINTER(C.c_int32), C.POINTER(i64), C.POINTER(i64),
                               C.POINTER(i64), C.POINTER(i64)]),
        "bempol_get_geometry": (i32, [vp, vp, vp, vp, vp, vp, vp]),
        "bempol_stats_enable": (i32, [vp, i32]),
        "bempol_stats_read": (i32, [vp, C.POINTER(Stats), i32]),
        "bempol_measure_peaks": (i32, [i32, i32, i32, C.POINTER(Peaks)]),
        "bempol_near_rule19": (i32, [vp]),
        "bempol_far_coefficients": (i32, [i32, vp, vp, vp, vp, vp]),
        "bempol_shard_rows": (i32, [i64, vp, i32, vp]),
        "bempol_set_shard": (i32, [vp, i32, i32, vp, ExchangeFn, vp]),
        "bempol_shard_bounds": (i32, [vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()
lib = _lib


class BempolError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def default_params(**kw) -> Params:
    p = Params()
    _lib.bempol_default_params(C.byref(p))
    for k, v in kw.items():
        if k in ("op", "residual_op") and isinstance(v, str):
            v = OP_NAMES[v]
        if k == "refine_scope" and isinstance(v, str):
            v = REFINE_NAMES[v]
        if k == "near_rule" and isinstance(v, str):
            v = NEAR_RULES[v]
        setattr(p, k, v)
    return p


def _ptr(a):
    """(pointer, where) of a numpy array (host) or torch tensor (host or device)."""
    if a is None:
        return None, HOST
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data, HOST
    if not a.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return a.data_ptr(), (DEVICE if a.is_cuda else HOST)


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


class Solver:
    """One context of the library: a mesh, its sites and the solver parameters."""

    def __init__(self, params: Params | None = None, device: int = 0, **kw):
        self.params = params if params is not None else default_params(**kw)
        h = C.c_void_p()
        st = _lib.bempol_create(C.byref(self.params), device, C.byref(h))
        if st != 0:
            raise BempolError(st, "bempol_create failed")
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            _lib.bempol_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        if st != 0:
            raise BempolError(st, _lib.bempol_last_error(self._h).decode())

    def set_params(self, **kw):
        for k, v in kw.items():
            if k in ("op", "residual_op") and isinstance(v, str):
                v = OP_NAMES[v]
            if k == "refine_scope" and isinstance(v, str):
                v = REFINE_NAMES[v]
            if k == "near_rule" and isinstance(v, str):
                v = NEAR_RULES[v]
            setattr(self.params, k, v)
        self._chk(_lib.bempol_set_params(self._h, C.byref(self.params)))

    def set_mesh(self, verts, tris, system=None, body=None, stream=None):
        """Surface(s).  ``system`` / ``body`` (int32 per triangle) give several bodies
        and independent systems (bempol_set_mesh_systems); None = one body."""
        pv, wv = _ptr(verts)
        pt, wt = _ptr(tris)
        if wv != wt:
            raise ValueError("verts and tris must both be host or both be device arrays")
        if system is None and body is None:
            self._chk(_lib.bempol_set_mesh(self._h, verts.shape[0], pv, tris.shape[0], pt, wv, _stream(stream)))
            return
        ps, ws = _ptr(system)
        pb, wb = _ptr(body)
        for w, a in ((ws, system), (wb, body)):
            if a is not None and w != wv:
                raise ValueError("system/body arrays must live where the mesh arrays live")
        self._chk(_lib.bempol_set_mesh_systems(self._h, verts.shape[0], pv, tris.shape[0], pt, ps, pb, wv,
                                               _stream(stream)))

    def set_mesh_stern(self, verts1, tris1, verts2, tris2, stream=None):
        """Dielectric boundary (verts1, tris1) inside the ion-exclusion surface (verts2,
        tris2), host arrays (bempol_set_mesh_stern); panels in caller order are the first
        surface's, then the second's."""
        v1 = np.ascontiguousarray(verts1, dtype=np.float64)
        t1 = np.ascontiguousarray(tris1, dtype=np.int32)
        v2 = np.ascontiguousarray(verts2, dtype=np.float64)
        t2 = np.ascontiguousarray(tris2, dtype=np.int32)
        self._chk(_lib.bempol_set_mesh_stern(self._h, v1.shape[0], v1.ctypes.data, t1.shape[0], t1.ctypes.data,
                                             v2.shape[0], v2.ctypes.data, t2.shape[0], t2.ctypes.data, HOST,
                                             _stream(stream)))

    def set_sites(self, pos, q, d, Q, alpha, group=None, system=None, body=None, stream=None):
        """Point multipoles; with several bodies/systems pass ``system`` / ``body`` per
        site (sites ordered by system, then body)."""
        arrs = [pos, q, d, Q, alpha] + [a for a in (group, system, body) if a is not None]
        ptrs = [_ptr(a) for a in arrs]
        where = {w for _, w in ptrs}
        if len(where) != 1:
            raise ValueError("site arrays must all be host or all be device")
        w = where.pop()
        pg, ps, pb = _ptr(group)[0], _ptr(system)[0], _ptr(body)[0]
        if system is None and body is None:
            self._chk(_lib.bempol_set_sites(self._h, pos.shape[0], ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[3][0],
                                            ptrs[4][0], pg, w, _stream(stream)))
        else:
            self._chk(_lib.bempol_set_sites_systems(self._h, pos.shape[0], ptrs[0][0], ptrs[1][0], ptrs[2][0],
                                                    ptrs[3][0], ptrs[4][0], pg, ps, pb, w, _stream(stream)))

    def systems(self):
        ns, nb = C.c_int64(), C.c_int64()
        self._chk(_lib.bempol_systems(self._h, C.byref(ns), C.byref(nb)))
        return ns.value, nb.value

    def sizes(self):
        v = [C.c_int64(), C.c_int32(), C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()]
        self._chk(_lib.bempol_sizes(self._h, *[C.byref(x) for x in v]))
        return dict(zip(["n_panels", "gauss_k", "n_sites", "n_near", "n_cells", "n_leaves"], [x.value for x in v]))

    def solve(self, stream=None, outputs=False, where="host", allow_unconverged=False, per_system=False):
        """Run the SCF + BEM solve; returns a dict of scalars (and arrays if ``outputs``).
        With ``per_system`` every system of the context is solved together
        (bempol_solve_systems) and ``out["systems"]`` lists each one's results."""
        r = Result()
        arrays = {}
        if outputs:
            sz = self.sizes()
            n, ns = sz["n_panels"], sz["n_sites"]
            if where == "host":
                mk = lambda k: np.zeros(k)
                r.where = HOST
            else:
                import torch
                mk = lambda k: torch.zeros(k, dtype=torch.float64, device=f"cuda:{self.device}")
                r.where = DEVICE
            arrays = {"phi": mk(n), "dphidn": mk(n), "site_reaction": mk(ns * 10), "mu_diss": mk(ns * 3),
                      "mu_vac": mk(ns * 3)}
            for k, a in arrays.items():
                setattr(r, k, _ptr(a)[0])
        per = None
        if per_system:
            nsys = self.systems()[0]
            per = (SystemResult * nsys)()
            st = _lib.bempol_solve_systems(self._h, _stream(stream), C.byref(r), per, nsys)
        else:
            st = _lib.bempol_solve(self._h, _stream(stream), C.byref(r))
        if st != 0 and not (allow_unconverged and st == 4):
            self._chk(st)
        out = {k: getattr(r, k) for k, _ in Result._fields_ if k not in arrays and k != "where"}
        out["status"] = st
        if per is not None:
            out["systems"] = [{k: getattr(x, k) for k, _ in SystemResult._fields_} for x in per]
        for k, a in arrays.items():
            out[k] = a
        return out

    def matvec(self, x, y, op=OP_FP64_DIRECT, stream=None):
        self._chk(_lib.bempol_matvec(self._h, _ptr(x)[0], _ptr(y)[0], OP_NAMES.get(op, op), _stream(stream)))

    def matvec_transposed(self, x, y, op=OP_FP64_DIRECT, stream=None):
        self._chk(_lib.bempol_matvec_transposed(self._h, _ptr(x)[0], _ptr(y)[0], OP_NAMES.get(op, op),
                                                _stream(stream)))

    def gradient(self, stream=None, allow_unconverged=False, units="paper", as_tensors=False):
        """Adjoint gradient of the last solve's Delta G_solv with respect to every site's
        q, d, Q and position (``units`` "paper" or "kcal"): dict of arrays ``q`` [ns],
        ``d`` [ns, 3], ``Q`` [ns, 3, 3], ``pos`` [ns, 3] (numpy, or device tensors with
        ``as_tensors``) and ``info``."""
        import torch
        ns = self.sizes()["n_sites"]
        dev = f"cuda:{self.device}"
        gq = torch.zeros(ns, dtype=torch.float64, device=dev)
        gd = torch.zeros(ns * 3, dtype=torch.float64, device=dev)
        gQ = torch.zeros(ns * 9, dtype=torch.float64, device=dev)
        gp = torch.zeros(ns * 3, dtype=torch.float64, device=dev)
        info = GradientInfo()
        st = _lib.bempol_gradient(self._h, _stream(stream), _ptr(gq)[0], _ptr(gd)[0], _ptr(gQ)[0], _ptr(gp)[0],
                                  C.byref(info), {"paper": 0, "kcal": 1}[units])
        if st != 0 and not (allow_unconverged and st == 4):
            self._chk(st)
        if as_tensors:
            return {"q": gq, "d": gd.reshape(-1, 3), "Q": gQ.reshape(-1, 3, 3), "pos": gp.reshape(-1, 3),
                    "info": {k: getattr(info, k) for k, _ in GradientInfo._fields_}, "status": st}
        return {"q": gq.cpu().numpy(), "d": gd.cpu().numpy().reshape(-1, 3), "Q": gQ.cpu().numpy().reshape(-1, 3, 3),
                "pos": gp.cpu().numpy().reshape(-1, 3),
                "info": {k: getattr(info, k) for k, _ in GradientInfo._fields_}, "status": st}

    def rhs(self, b, p=None, op=OP_FP64_DIRECT, stream=None):
        self._chk(_lib.bempol_rhs(self._h, _ptr(p)[0], _ptr(b)[0], OP_NAMES.get(op, op), _stream(stream)))

    def site_reaction(self, x, out, op=OP_FP64_DIRECT, stream=None):
        self._chk(_lib.bempol_site_reaction(self._h, _ptr(x)[0], _ptr(out)[0], OP_NAMES.get(op, op),
                                            _stream(stream)))

    def site_reaction_noalloc(self, x, out, op=OP_FP64_DIRECT, stream=None):
        """Same as site_reaction, with no device allocation during the call (fixed scratch)."""
        self._chk(_lib.bempol_site_reaction_noalloc(self._h, _ptr(x)[0], _ptr(out)[0], OP_NAMES.get(op, op),
                                                    _stream(stream)))

    def multipole_field(self, out, mu=None, mode=0, stream=None):
        self._chk(_lib.bempol_multipole_field(self._h, _ptr(mu)[0], mode, _ptr(out)[0], _stream(stream)))

    def set_shard(self, rank: int, world: int, exchange=None):
        """Compute only this rank's treecode rows (bempol_set_shard).  ``exchange(buf,
        bounds)`` receives the library's product in ``buf`` (a device float64 tensor
        [2N], internal panel order, this rank's rows valid) and the row bounds, and must
        fill the other ranks' rows, e.g. ``lambda b, bd: allgather_rows(b, bd, rank,
        world)``.  world = 1 turns sharding off."""
        if world <= 1:
            self._chk(_lib.bempol_set_shard(self._h, 0, 1, None, ExchangeFn(), None))
            self._shard = None
            return
        import torch
        n = self.sizes()["n_panels"]
        buf = torch.zeros(2 * n, dtype=torch.float64, device=f"cuda:{self.device}")

        def cb(user, bounds, nw, stream):
            exchange(buf, [int(bounds[k]) for k in range(nw + 1)])

        fn = ExchangeFn(cb)
        self._shard = (buf, fn, None, world)   # the library holds raw pointers to buf and fn
        self._chk(_lib.bempol_set_shard(self._h, rank, world, _ptr(buf)[0], fn, None))

    def shard_bounds(self):
        """Row bounds [world + 1] of the current sharding (internal panel order)."""
        world = 1 if getattr(self, "_shard", None) is None else self._shard[3]
        b = np.zeros(world + 1, dtype=np.int64)
        self._chk(_lib.bempol_shard_bounds(self._h, b.ctypes.data))
        return [int(v) for v in b]

    def autotune(self, target_err=1e-5, stream=None):
        """Pick leaf, theta and order for the current mesh (bempol_autotune); returns the
        choice and updates this Solver's parameters."""
        r = TuneResult()
        self._chk(_lib.bempol_autotune(self._h, float(target_err), C.byref(r), _stream(stream)))
        self.params.leaf, self.params.theta, self.params.order = r.leaf, r.theta, r.order
        return {k: getattr(r, k) for k, _ in TuneResult._fields_}

    def stats_enable(self, on=True):
        self._chk(_lib.bempol_stats_enable(self._h, 1 if on else 0))

    def stats(self, reset=False):
        st = Stats()
        self._chk(_lib.bempol_stats_read(self._h, C.byref(st), 1 if reset else 0))
        return {k: getattr(st, k) for k, _ in Stats._fields_}

    def geometry(self):
        sz = self.sizes()
        n, nnz = sz["n_panels"], sz["n_near"]
        out = {"centroid": np.zeros((n, 3)), "normal": np.zeros((n, 3)), "area": np.zeros(n),
               "near_ptr": np.zeros(n + 1, dtype=np.int64), "near_col": np.zeros(max(nnz, 1), dtype=np.int32),
               "near_corr": np.zeros((max(nnz, 1), 4))}
        self._chk(_lib.bempol_get_geometry(self._h, *[out[k].ctypes.data for k in
                                                      ("centroid", "normal", "area", "near_ptr", "near_col",
                                                       "near_corr")]))
        out["near_col"] = out["near_col"][:nnz]
        out["near_corr"] = out["near_corr"][:nnz]
        return out


def measure_peaks(device: int = 0, iters: int = 65536, reps: int = 3) -> dict:
    """FP32 / FP64 FMA and MUFU (rsqrt, 2^x) throughput of the device
    (bempol_measure_peaks)."""
    r = Peaks()
    st = _lib.bempol_measure_peaks(device, iters, reps, C.byref(r))
    if st != 0:
        raise BempolError(st, "bempol_measure_peaks failed")
    return {k: getattr(r, k) for k, _ in Peaks._fields_}


def near_rule19() -> np.ndarray:
    """The library's 19-node triangle rule [19, 4]: l1, l2, l3, weight (bempol_near_rule19,
    host only)."""
    out = np.zeros((19, 4), dtype=np.float64)
    st = _lib.bempol_near_rule19(out.ctypes.data)
    if st != 0:
        raise BempolError(st, "bempol_near_rule19 failed")
    return out


def far_coefficients(order: int):
    """The treecode's far-field coefficient table at `order` (bempol_far_coefficients, host
    only): (ptr [NB + 1], moment [terms], coef [terms]), CSR over the NB entries."""
    ne = C.c_int64(0)
    nt = C.c_int64(0)
    st = _lib.bempol_far_coefficients(int(order), C.addressof(ne), C.addressof(nt), None, None, None)
    if st != 0:
        raise BempolError(st, "bempol_far_coefficients failed")
    ptr = np.zeros(ne.value + 1, dtype=np.int32)
    mom = np.zeros(nt.value, dtype=np.int32)
    coef = np.zeros(nt.value, dtype=np.float64)
    st = _lib.bempol_far_coefficients(int(order), C.addressof(ne), C.addressof(nt), ptr.ctypes.data,
                                      mom.ctypes.data, coef.ctypes.data)
    if st != 0:
        raise BempolError(st, "bempol_far_coefficients failed")
    return ptr, mom, coef


def shard_rows(n_units: int, world: int, cost=None):
    """Contiguous ranges of nearly equal cost (bempol_shard_rows, host only)."""
    b = np.zeros(world + 1, dtype=np.int64)
    c = None if cost is None else np.ascontiguousarray(cost, dtype=np.float64)
    st = _lib.bempol_shard_rows(int(n_units), None if c is None else c.ctypes.data, int(world), b.ctypes.data)
    if st != 0:
        raise BempolError(st, "bempol_shard_rows: bad arguments")
    return [int(v) for v in b]


def allgather_rows(buf, bounds, rank: int, world: int, group=None):
    """The exchange of a sharded product: rank r holds rows [bounds[r], bounds[r+1]) of
    both halves of ``buf`` ([2N]: phi rows, then psi rows); after the call every rank
    holds every row.  One torch.distributed all-gather of the ranks' row blocks (padded
    to the longest), on any backend (NCCL for device tensors, gloo for host tensors)."""
    import torch
    import torch.distributed as dist
    n = bounds[-1]
    lens = [bounds[k + 1] - bounds[k] for k in range(world)]
    m = max(lens)
    lo, hi = bounds[rank], bounds[rank + 1]
    mine = torch.zeros(2 * m, dtype=buf.dtype, device=buf.device)
    mine[:hi - lo] = buf[lo:hi]
    mine[m:m + hi - lo] = buf[n + lo:n + hi]
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    for k in range(world):
        a, e = bounds[k], bounds[k + 1]
        buf[a:e] = parts[k][:e - a]
        buf[n + a:n + e] = parts[k][m:m + e - a]
    return buf


KCAL_PER_UNIT = 4.0 * 3.141592653589793 * 332.0637132991921  # kcal/mol per e^2/A (vacuum permittivity 1)


def _torch_function():
    import torch

    class SolvationEnergy(torch.autograd.Function):
        """Delta G_solv (kcal/mol) of a Solver's mesh with sites (pos, q, d, Q) as a
        differentiable function: forward = bempol_set_sites + bempol_solve, backward =
        bempol_gradient (the adjoint of the BEM solve and of the induced-dipole
        relaxation).  alpha and the polarisation groups are fixed inputs; the quadrupole
        gradient is the symmetric traceless one.  The backward uses the Solver's last
        solve, so no other solve may run on that Solver between forward and backward."""

        @staticmethod
        def forward(ctx, solver, pos, q, d, Q, alpha, group=None):
            c = lambda t: t.detach().to(torch.float64).contiguous()
            solver.set_sites(c(pos), c(q), c(d), c(Q).reshape(-1, 9), c(alpha),
                             None if group is None else group.to(torch.int32).contiguous())
            r = solver.solve()
            ctx.solver = solver
            ctx.dev = pos.device
            return torch.tensor(r["dG_solv_kcal"], dtype=torch.float64, device=pos.device)

        @staticmethod
        def backward(ctx, g):
            gr = ctx.solver.gradient(units="kcal", as_tensors=True)   # kcal/mol per unit, from the library
            k = g.to(torch.float64)
            t = lambda a: a.to(ctx.dev) * k
            return None, t(gr["pos"]), t(gr["q"]), t(gr["d"]), t(gr["Q"]), None, None

    return SolvationEnergy


def solvation_energy(solver, pos, q, d, Q, alpha, group=None):
    """Differentiable Delta G_solv in kcal/mol (torch.autograd), see ``SolvationEnergy``."""
    return _torch_function().apply(solver, pos, q, d, Q, alpha, group)


def _param_kw(par, overrides):
    kw = dict(eps_in=par.eps_in, eps_out=par.eps_out, kappa=par.kappa, gauss_k=par.gauss_k,
              near_factor=par.near_factor, theta=par.theta, order=par.order, leaf=par.leaf,
              gmres_tol=par.gmres_tol, gmres_restart=par.gmres_restart, gmres_maxit=par.gmres_maxit,
              scf_tol=par.scf_tol, sor_omega=par.sor_omega, scf_maxit=par.scf_maxit, thole_a=par.thole_a,
              thole_perm=int(bool(getattr(par, "damp_permanent", False))),
              near_rule=NEAR_RULES[getattr(par, "near_rule", "exact")])
    kw.update(overrides)
    return kw


def batch_solver(problems, device: int = 0, stream=None, **overrides) -> Solver:
    """One Solver holding several ``gen.Problem`` s as independent systems (system k =
    problems[k]; each problem's ``panel_body`` and ``sites.body`` give its bodies).
    Parameters come from the first problem."""
    verts, tris, psys, pbody = [], [], [], []
    cols = {k: [] for k in ("pos", "q", "d", "Q", "alpha", "group", "system", "body")}
    voff = goff = 0
    for k, pr in enumerate(problems):
        verts.append(np.asarray(pr.verts, dtype=np.float64))
        tris.append(np.asarray(pr.tris, dtype=np.int64) + voff)
        voff += pr.verts.shape[0]
        psys.append(np.full(pr.tris.shape[0], k, dtype=np.int32))
        pb = getattr(pr, "panel_body", None)
        pbody.append(np.zeros(pr.tris.shape[0], np.int32) if pb is None else np.asarray(pb, np.int32))
        st = pr.sites
        order = np.argsort(st.body, kind="stable")
        cols["pos"].append(st.pos[order])
        cols["q"].append(st.q[order])
        cols["d"].append(st.d[order])
        cols["Q"].append(st.Q[order].reshape(-1, 9))
        cols["alpha"].append(st.alpha[order])
        cols["group"].append(np.asarray(st.group, np.int64)[order] + goff)
        goff += int(np.max(st.group)) + 1 if st.n else 0
        cols["system"].append(np.full(st.n, k, np.int32))
        cols["body"].append(np.asarray(st.body, np.int32)[order])
    s = Solver(device=device, **_param_kw(problems[0].params, overrides))
    s.set_mesh(np.ascontiguousarray(np.vstack(verts)), np.ascontiguousarray(np.vstack(tris), dtype=np.int32),
               system=np.concatenate(psys), body=np.ascontiguousarray(np.concatenate(pbody)), stream=stream)
    cat = {k: np.concatenate(v) for k, v in cols.items()}
    s.set_sites(np.ascontiguousarray(cat["pos"]), np.ascontiguousarray(cat["q"]), np.ascontiguousarray(cat["d"]),
                np.ascontiguousarray(cat["Q"]), np.ascontiguousarray(cat["alpha"]),
                np.ascontiguousarray(cat["group"], dtype=np.int32), system=np.ascontiguousarray(cat["system"]),
                body=np.ascontiguousarray(cat["body"]), stream=stream)
    return s


def problem_solver(problem, device: int = 0, stream=None, **overrides) -> Solver:
    """A Solver loaded with a ``gen.Problem`` (mesh and sites from host arrays); a
    problem with several bodies (``panel_body``) is loaded as one system of bodies."""
    if getattr(problem, "panel_body", None) is not None:
        return batch_solver([problem], device=device, stream=stream, **overrides)
    s = Solver(device=device, **_param_kw(problem.params, overrides))
    s.set_mesh(np.ascontiguousarray(problem.verts, dtype=np.float64),
               np.ascontiguousarray(problem.tris, dtype=np.int32), stream=stream)
    st = problem.sites
    s.set_sites(np.ascontiguousarray(st.pos), np.ascontiguousarray(st.q), np.ascontiguousarray(st.d),
                np.ascontiguousarray(st.Q.reshape(-1, 9)), np.ascontiguousarray(st.alpha),
                np.ascontiguousarray(st.group, dtype=np.int32), stream=stream)
    return s
