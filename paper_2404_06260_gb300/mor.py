"""ctypes binding of libmor (include/mor.h).  Argument marshalling only: every step of
the method runs in the library's CUDA kernels.  PyTorch provides device memory and
the CUDA stream.  Importing this module loads the library and raises if it is absent.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from ._build import LIB

MOR_OK = 0
MOR_ERR_NOT_CONVERGED = -4
MOR_ERR_TIMEOUT = -5
FP64 = 0
MIXED = 1

if not os.path.exists(LIB):
    raise ImportError("libmor.so is not built (%s); run paper_2404_06260_gb300._build.build()"
                      % LIB)
_lib = ctypes.CDLL(LIB)

_P = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_dbl = ctypes.c_double


class _MeshC(ctypes.Structure):
    _fields_ = [("n_nodes", _i64), ("n_tets", _i64), ("tets", _P), ("dirichlet", _P),
                ("xyz_dev", _P), ("tets_dev", _P), ("kappa_dev", _P)]


class _MeshHostC(ctypes.Structure):
    _fields_ = [("n_nodes", _i64), ("n_tets", _i64), ("tets", _P), ("dirichlet", _P),
                ("xyz", _P), ("kappa", _P)]


class BasisOpts(ctypes.Structure):
    _fields_ = [("rank", _i32), ("oversample", _i32), ("ranks", _P), ("eps", _dbl),
                ("seed", ctypes.c_uint64),
                ("precision", _i32), ("sketch", _i32), ("cg_rtol", _dbl),
                ("max_iter", _i32), ("replace_every", _i32), ("normwise", _i32),
                ("drift_restart", _dbl),
                ("sketch_rtol", _dbl), ("tau", _dbl), ("orth_tol", _dbl),
                ("coarse_rows", _i32), ("h1_weighted", _i32), ("sketch_div", _i32),
                ("sub_begin", _i32),
                ("sub_end", _i32), ("tc_gram", _i32), ("explicit_svd", _i32)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", _i32), ("converged", _i32), ("rel_residual", _dbl),
                ("energy", _dbl)]


def _sig(name, res, *args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


_sig("mor_build_subdomains", _i32, ctypes.POINTER(_MeshC), _P, _i32, _P, ctypes.POINTER(_P))
_sig("mor_build_subdomains_host", _i32, ctypes.POINTER(_MeshHostC), _P, _i32, _i32, _P,
     ctypes.POINTER(_P))
_sig("mor_build_subdomains_streamed", _i32, ctypes.POINTER(_MeshC), _P, _i32, _i32, _P,
     ctypes.POINTER(_P))
_sig("mor_debug_plan_check", _i32, _i64, _i64, _P, _P, _P, _P, _i32, _i32, _i32, _P)
_sig("mor_subdomains_counts", _i32, _P, ctypes.POINTER(_i32), _P)
_sig("mor_subdomains_indices", _i32, _P, _i32, _i32, _P)
_sig("mor_basis_opts_default", _i32, ctypes.POINTER(BasisOpts))
_sig("mor_build_bases", _i32, _P, ctypes.POINTER(BasisOpts), _P, ctypes.POINTER(_P))
_sig("mor_bases_info", _i32, _P, ctypes.POINTER(_i32), ctypes.POINTER(_i32), _P,
     ctypes.POINTER(_i64))
_sig("mor_bases_sigma", _i32, _P, _P)
_sig("mor_bases_get_Q", _i32, _P, _i32, _P)
_sig("mor_bases_get_rbb", _i32, _P, _i32, _P)
_sig("mor_bases_get_bt", _i32, _P, _P)
_sig("mor_bases_stats", _i32, _P, _P)
_sig("mor_project", _i32, _P, _P, _P, ctypes.POINTER(_P))
_sig("mor_reduced_info", _i32, _P, ctypes.POINTER(_i64), ctypes.POINTER(_i64))
_sig("mor_reduced_dense", _i32, _P, _P)
_sig("mor_solve_reduced", _i32, _P, _dbl, _i32, _P, _P, ctypes.POINTER(SolveInfo))
_sig("mor_solve_reduced_noalloc", _i32, _i32, _i32, _P, _P, _P, _P, _P, _dbl, _i32, _P, _P,
     ctypes.POINTER(SolveInfo))
_sig("mor_lift", _i32, _P, _P, _P, _P, _P)
_sig("mor_set_wait_budget", _i32, _dbl)
_sig("mor_debug_wait_timeout", _i32, _dbl, ctypes.POINTER(_i32))
_sig("mor_energy_norm", _i32, _P, _P, _P, ctypes.POINTER(_dbl), _P)
_sig("mor_debug_tc_gram", _i32, _i64, _i32, _i32, _P, _P, _P, _P)
_sig("mor_debug_coarse_inverse", _i32, _i32, _P, _P, _P)
_sig("mor_debug_sketch_rhs", _i32, _P, ctypes.POINTER(BasisOpts), _i32, _P, _P)
_sig("mor_profile_enable", _i32, _i32)
_sig("mor_profile_reset", _i32)
_sig("mor_profile_query", _i32, _i32, _P)
_sig("mor_kernel_launches", _i32, ctypes.POINTER(_i64))
_sig("mor_autotune", _i32, _i32)
_sig("mor_autotune_report", _i32, _P, _i32, ctypes.POINTER(_i32))
_sig("mor_free_subdomains", None, _P)
_sig("mor_free_bases", None, _P)
_sig("mor_free_reduced", None, _P)
_sig("mor_last_error", ctypes.c_char_p)

EXPORTED = ["mor_build_subdomains", "mor_build_subdomains_host",
            "mor_build_subdomains_streamed", "mor_subdomains_counts",
            "mor_subdomains_indices",
            "mor_basis_opts_default", "mor_build_bases", "mor_bases_info", "mor_bases_sigma",
            "mor_bases_get_Q", "mor_bases_get_rbb", "mor_bases_get_bt", "mor_bases_stats", "mor_project",
            "mor_reduced_info", "mor_reduced_dense", "mor_solve_reduced",
            "mor_solve_reduced_noalloc", "mor_set_wait_budget", "mor_debug_wait_timeout",
            "mor_lift",
            "mor_energy_norm", "mor_debug_sketch_rhs", "mor_debug_plan_check",
            "mor_debug_tc_gram", "mor_debug_coarse_inverse",
            "mor_profile_enable",
            "mor_profile_reset", "mor_profile_query", "mor_kernel_launches", "mor_autotune",
            "mor_autotune_report", "mor_free_subdomains",
            "mor_free_bases", "mor_free_reduced", "mor_last_error"]


class MorError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libmor error %d: %s" % (code, msg))
        self.code = code


def _check(rc):
    if rc != MOR_OK:
        raise MorError(rc, _lib.mor_last_error().decode())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return _P(stream.cuda_stream)


def _ptr(a):
    if isinstance(a, torch.Tensor):
        return _P(a.data_ptr())
    return a.ctypes.data_as(_P)


class Mesh:
    """Host arrays for step 1 and device copies for the kernels (kept alive here)."""

    def __init__(self, xyz, tets, kappa, dirichlet, device="cuda"):
        self.tets_h = np.ascontiguousarray(tets, dtype=np.int32)
        self.dir_h = np.ascontiguousarray(dirichlet, dtype=np.uint8)
        self.xyz_d = torch.as_tensor(np.ascontiguousarray(xyz, np.float64), device=device)
        self.tets_d = torch.as_tensor(self.tets_h, device=device)
        self.kappa_d = torch.as_tensor(np.ascontiguousarray(kappa, np.float64), device=device)
        self.n_nodes = int(self.xyz_d.shape[0])
        self.n_tets = int(self.tets_h.shape[0])

    @classmethod
    def from_device(cls, xyz_d, tets_d, kappa_d, tets_host, dirichlet_host):
        """Wrap device tensors already on the GPU (plus the host copies step 1 needs)."""
        self = cls.__new__(cls)
        self.tets_h = np.ascontiguousarray(tets_host, dtype=np.int32)
        self.dir_h = np.ascontiguousarray(dirichlet_host, dtype=np.uint8)
        self.xyz_d, self.tets_d, self.kappa_d = xyz_d, tets_d, kappa_d
        self.n_nodes = int(xyz_d.shape[0])
        self.n_tets = int(self.tets_h.shape[0])
        return self

    def _c(self):
        return _MeshC(self.n_nodes, self.n_tets, _ptr(self.tets_h), _ptr(self.dir_h),
                      _P(self.xyz_d.data_ptr()), _P(self.tets_d.data_ptr()),
                      _P(self.kappa_d.data_ptr()))


class _HostMeshInfo:
    """Sizes of a mesh whose device copies belong to the library's handle."""

    def __init__(self, n_nodes, n_tets):
        self.n_nodes, self.n_tets = n_nodes, n_tets


class Subdomains:
    """Step 1.  wave > 0 builds a streamed plan (mor_build_subdomains_streamed):
    mor_build_bases then works in waves of `wave` subdomains."""

    def __init__(self, mesh: Mesh, owner, r_hops: int, stream=None, wave: int = 0):
        self.mesh = mesh
        self._owner = np.ascontiguousarray(owner, dtype=np.int32)
        self.streamed = wave > 0
        h = _P()
        mc = mesh._c()
        if self.streamed:
            _check(_lib.mor_build_subdomains_streamed(ctypes.byref(mc), _ptr(self._owner),
                                                      int(r_hops), int(wave),
                                                      _stream(stream), ctypes.byref(h)))
        else:
            _check(_lib.mor_build_subdomains(ctypes.byref(mc), _ptr(self._owner),
                                             int(r_hops), _stream(stream), ctypes.byref(h)))
        self.h = h
        n = _i32()
        _check(_lib.mor_subdomains_counts(h, ctypes.byref(n), None))
        self.n_sub = n.value
        self.counts = np.zeros((self.n_sub, 7), dtype=np.int64)
        _check(_lib.mor_subdomains_counts(h, None, _ptr(self.counts)))

    @classmethod
    def from_host(cls, xyz, tets, kappa, dirichlet, owner, r_hops: int, stream=None,
                  wave: int = 0):
        """Step 1 from host arrays (mor_build_subdomains_host): the library copies the
        mesh to the device itself; numpy arrays or (pinned) CPU tensors."""
        self = cls.__new__(cls)
        arrs = []

        def host(a, dt):
            if isinstance(a, torch.Tensor):
                assert a.device.type == "cpu" and a.is_contiguous() and a.dtype == dt[1]
                arrs.append(a)
                return _P(a.data_ptr()), int(a.shape[0])
            a = np.ascontiguousarray(a, dtype=dt[0])
            arrs.append(a)
            return a.ctypes.data_as(_P), int(a.shape[0])

        px, nn = host(xyz, (np.float64, torch.float64))
        pt, nt = host(tets, (np.int32, torch.int32))
        pk, _ = host(kappa, (np.float64, torch.float64))
        pd, _ = host(dirichlet, (np.uint8, torch.uint8))
        self._owner = np.ascontiguousarray(owner, dtype=np.int32)
        self.mesh = _HostMeshInfo(nn, nt)
        self.streamed = wave > 0
        h = _P()
        mc = _MeshHostC(nn, nt, pt, pd, px, pk)
        _check(_lib.mor_build_subdomains_host(ctypes.byref(mc), _ptr(self._owner),
                                              int(r_hops), int(wave), _stream(stream),
                                              ctypes.byref(h)))
        self.h = h
        n = _i32()
        _check(_lib.mor_subdomains_counts(h, ctypes.byref(n), None))
        self.n_sub = n.value
        self.counts = np.zeros((self.n_sub, 7), dtype=np.int64)
        _check(_lib.mor_subdomains_counts(h, None, _ptr(self.counts)))
        return self

    def indices(self, sub: int, which: int) -> np.ndarray:
        # streamed plans keep no index sets (count -1): the library answers MOR_ERR_STATE
        n = int(self.counts[sub, which])
        out = np.zeros(max(n, 1), dtype=np.int32)
        _check(_lib.mor_subdomains_indices(self.h, int(sub), int(which), _ptr(out)))
        return out[:max(n, 0)]

    def __del__(self):
        if getattr(self, "h", None):
            _lib.mor_free_subdomains(self.h)
            self.h = None


def basis_opts(**kw) -> BasisOpts:
    """Defaults of mor_basis_opts_default overridden by keywords; `ranks` may be a
    sequence of per-subdomain ranks (kept alive on the returned object)."""
    o = BasisOpts()
    _check(_lib.mor_basis_opts_default(ctypes.byref(o)))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": FP64, "mixed": MIXED}[v]
        if k == "sketch" and isinstance(v, str):
            v = {"field": 0, "paper": 1}[v]
        if k == "ranks":
            arr = np.ascontiguousarray(v, dtype=np.int32)
            o._ranks = arr
            v = _ptr(arr)
        setattr(o, k, v)
    return o


class Bases:
    def __init__(self, sd: Subdomains, opts: BasisOpts, stream=None):
        self.sd = sd
        h = _P()
        rc = _lib.mor_build_bases(sd.h, ctypes.byref(opts), _stream(stream), ctypes.byref(h))
        self.h = h
        self.converged = rc == MOR_OK
        if rc not in (MOR_OK, MOR_ERR_NOT_CONVERGED) or not h:
            _check(rc)
        kq, k = _i32(), _i32()
        self.kept = np.zeros(sd.n_sub, dtype=np.int32)
        tot = _i64()
        _check(_lib.mor_bases_info(h, ctypes.byref(kq), ctypes.byref(k), _ptr(self.kept),
                                   ctypes.byref(tot)))
        self.kq, self.k, self.total_kept = kq.value, k.value, tot.value

    def sigma(self) -> np.ndarray:
        out = np.zeros((self.sd.n_sub, self.k))
        _check(_lib.mor_bases_sigma(self.h, _ptr(out)))
        return out

    def Q(self, sub: int) -> np.ndarray:
        out = np.zeros((int(self.sd.counts[sub, 3]), self.kq))
        _check(_lib.mor_bases_get_Q(self.h, int(sub), _ptr(out)))
        return out

    def rbb(self, sub: int) -> np.ndarray:
        m = int(self.sd.counts[sub, 1])
        out = np.zeros((m, m))
        _check(_lib.mor_bases_get_rbb(self.h, int(sub), _ptr(out)))
        return out

    def bt(self) -> np.ndarray:
        out = np.zeros((self.sd.n_sub, self.kq))
        _check(_lib.mor_bases_get_bt(self.h, _ptr(out)))
        return out

    def stats(self) -> np.ndarray:
        out = np.zeros(8, dtype=np.int64)
        _check(_lib.mor_bases_stats(self.h, _ptr(out)))
        return out

    def __del__(self):
        if getattr(self, "h", None):
            _lib.mor_free_bases(self.h)
            self.h = None


class Reduced:
    def __init__(self, sd: Subdomains, bases: Bases, stream=None):
        self.sd, self.bases = sd, bases
        h = _P()
        _check(_lib.mor_project(sd.h, bases.h, _stream(stream), ctypes.byref(h)))
        self.h = h
        dim, nb = _i64(), _i64()
        _check(_lib.mor_reduced_info(h, ctypes.byref(dim), ctypes.byref(nb)))
        self.dim, self.n_blocks = dim.value, nb.value

    def dense(self) -> np.ndarray:
        out = np.zeros((self.dim, self.dim))
        _check(_lib.mor_reduced_dense(self.h, _ptr(out)))
        return out

    def solve(self, rtol=1e-12, max_iter=20000, stream=None, x=None):
        if x is None:
            x = torch.zeros(self.dim, dtype=torch.float64, device="cuda")
        info = SolveInfo()
        rc = _lib.mor_solve_reduced(self.h, float(rtol), int(max_iter), _stream(stream),
                                    _P(x.data_ptr()), ctypes.byref(info))
        if rc not in (MOR_OK, MOR_ERR_NOT_CONVERGED):
            _check(rc)
        return x, dict(iterations=info.iterations, converged=bool(info.converged),
                       rel_residual=info.rel_residual, energy=info.energy)

    def __del__(self):
        if getattr(self, "h", None):
            _lib.mor_free_reduced(self.h)
            self.h = None


def set_wait_budget(seconds: float):
    _check(_lib.mor_set_wait_budget(float(seconds)))


def debug_wait_timeout(seconds: float) -> bool:
    """True when a bounded wait on a flag nothing sets ran out and returned."""
    t = _i32()
    rc = _lib.mor_debug_wait_timeout(float(seconds), ctypes.byref(t))
    if rc not in (MOR_OK, MOR_ERR_TIMEOUT):
        _check(rc)
    return bool(t.value)


def lift(sd: Subdomains, bases: Bases, x, stream=None):
    u = torch.empty(sd.mesh.n_nodes, dtype=torch.float64, device="cuda")
    _check(_lib.mor_lift(sd.h, bases.h, _P(x.data_ptr()), _P(u.data_ptr()), _stream(stream)))
    return u


def energy_norm(sd: Subdomains, u1, u2=None, stream=None) -> float:
    out = _dbl()
    _check(_lib.mor_energy_norm(sd.h, _P(u1.data_ptr()),
                                _P(u2.data_ptr()) if u2 is not None else None,
                                ctypes.byref(out), _stream(stream)))
    return out.value


def sketch_rhs(sd: Subdomains, opts: BasisOpts, sub: int, stream=None) -> np.ndarray:
    n = int(sd.counts[sub, 0] + sd.counts[sub, 1])
    out = np.zeros((n, opts.rank + opts.oversample))
    _check(_lib.mor_debug_sketch_rhs(sd.h, ctypes.byref(opts), int(sub), _ptr(out),
                                     _stream(stream)))
    return out


def tc_gram(X, Y, stream=None):
    """G = X^T Y on the tensor cores (mor_debug_tc_gram); X, Y binary64 CUDA tensors."""
    assert X.is_cuda and Y.is_cuda and X.dtype == torch.float64 and Y.dtype == torch.float64
    X, Y = X.contiguous(), Y.contiguous()
    G = torch.empty((X.shape[1], Y.shape[1]), dtype=torch.float64, device=X.device)
    _check(_lib.mor_debug_tc_gram(int(X.shape[0]), int(X.shape[1]), int(Y.shape[1]),
                                  _P(X.data_ptr()), _P(Y.data_ptr()), _P(G.data_ptr()),
                                  _stream(stream)))
    return G


def coarse_inverse(E, stream=None):
    """The coarse level's inverse of an SPD aggregate matrix (mor_debug_coarse_inverse);
    E a binary64 CUDA tensor n x n."""
    assert E.is_cuda and E.dtype == torch.float64 and E.shape[0] == E.shape[1]
    E = E.contiguous()
    out = torch.empty_like(E)
    _check(_lib.mor_debug_coarse_inverse(int(E.shape[0]), _P(E.data_ptr()), _P(out.data_ptr()),
                                         _stream(stream)))
    return out


def profile(on: bool):
    _check(_lib.mor_profile_enable(1 if on else 0))


def profile_reset():
    _check(_lib.mor_profile_reset())


def profile_query(family: int):
    out = np.zeros(4)
    _check(_lib.mor_profile_query(int(family), _ptr(out)))
    return dict(launches=out[0], ms=out[1], bytes=out[2])


KERNEL_FAMILIES = {0: "cg_spmm_pq<f32>", 1: "cg_spmm_pq<f64>", 2: "cg_update_xr<f32>",
                   3: "cg_update_xr<f64>", 4: "cg_update_p<f32>", 5: "cg_update_p<f64>",
                   6: "cg_coarse<f32>", 7: "cg_coarse<f64>"}


def autotune(on):
    """True / False: tuning on or off; None: clear the cache (mor_autotune)."""
    _check(_lib.mor_autotune(-1 if on is None else (1 if on else 0)))


def autotune_report():
    out = np.zeros((64, 8), dtype=np.int64)
    n = _i32()
    _check(_lib.mor_autotune_report(_ptr(out), 64, ctypes.byref(n)))
    names = ["1 record, 256 threads", "2 records, 256 threads", "1 record, 128 threads",
             "2 records, 128 threads"]
    return [dict(binary64=bool(r[0]), columns=int(r[1]), slot_width=int(r[2]),
                 chosen=names[int(r[3])], us=[int(x) for x in r[4:8]])
            for r in out[:n.value]]


def kernel_launches() -> int:
    out = _i64()
    _check(_lib.mor_kernel_launches(ctypes.byref(out)))
    return out.value


def plan_check(mesh, owner, r_hops: int, wave: int, coarse_rows: int = 35) -> dict:
    """Host-only consistency check of step 1 (mor_debug_plan_check); needs no GPU."""
    tets = np.ascontiguousarray(mesh.tets, dtype=np.int32)
    dirichlet = np.ascontiguousarray(mesh.dirichlet, dtype=np.uint8)
    own = np.ascontiguousarray(owner, dtype=np.int32)
    xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
    out = np.zeros(8, dtype=np.int64)
    _check(_lib.mor_debug_plan_check(int(mesh.n_nodes), int(mesh.n_tets), _ptr(tets),
                                     _ptr(dirichlet), _ptr(own), _ptr(xyz), int(r_hops),
                                     int(wave), int(coarse_rows), _ptr(out)))
    keys = ["n_sub", "rows", "waves", "wave_mismatches", "aggregate_violations",
            "max_slots", "max_aggregates", "owned"]
    return dict(zip(keys, out.tolist()))
