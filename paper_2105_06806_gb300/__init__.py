"""Python binding of libedgb.so (include/edgb.h): argument marshalling only.

Every step of the exact-diagonalisation path runs in the CUDA library; this
module converts Python/NumPy/PyTorch arguments to the C structures, passes
device pointers (``tensor.data_ptr()``) and CUDA streams
(``torch.cuda.current_stream().cuda_stream``) through, and raises
``EDError`` on a non-OK status.  There is no CPU fallback: when the library
is missing, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libedgb.so")

ED_OK, ED_PENDING = 0, 1
ED_ERR_ARG, ED_ERR_UNSUPPORTED, ED_ERR_OOM, ED_ERR_CUDA = -1, -2, -3, -4
ED_ERR_TIMEOUT, ED_ERR_NOT_CONVERGED, ED_ERR_BUSY, ED_ERR_NOT_FOUND = -5, -6, -7, -8
FP64, FP32, FP32_POLISH = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp32": FP32, "fp32_polish": FP32_POLISH}

EXPORTED = [
    "ed_sector_build", "ed_sector_get_info", "ed_sector_copy_tables", "ed_sector_copy_w",
    "ed_sector_free", "ed_matvec", "ed_matvec_blocked", "ed_sector_blocked_kernel",
    "ed_sector_tune_info", "ed_sector_set_kernel",
    "ed_sector_permute", "ed_lanczos_ground", "ed_gf_lanczos", "ed_gf_lanczos_z", "ed_sigma",
    "ed_observables", "ed_solve", "ed_eph_matvec", "ed_eph_lanczos_ground",
    "ed_eph_gf_lanczos_z", "ed_lanczos_states", "ed_espace_truncate", "ed_gf_thermal_z",
    "ed_chi_z", "ed_chi_ab_z", "ed_chi_tau", "ed_orbital_sector_dims", "ed_lanczos_ground_orbital",
    "ed_server_create", "ed_submit", "ed_poll", "ed_wait", "ed_server_destroy",
    "ed_server_inject_alloc_failure", "ed_batch_stats", "ed_residual_noalloc", "ed_status_string",
    "ed_last_error",
    "ed_kernel_launches", "ed_memory_trim", "ed_memory_cached",
]


class EDError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = f"{what}: status {status}"
        try:
            L = lib()
            msg += f" ({L.ed_status_string(status).decode()})"
            last = L.ed_last_error().decode()
            if last:
                msg += f" — {last}"
        except Exception:
            pass
        super().__init__(msg)


# ----------------------------------------------------------------- structs

DP = C.POINTER(C.c_double)


class ed_model(C.Structure):
    _fields_ = [("norb", C.c_int32), ("nbath", C.c_int32), ("U", C.c_double),
                ("Ust", C.c_double), ("Jh", C.c_double), ("Jx", C.c_double),
                ("Jp", C.c_double), ("e_imp", DP), ("e_bath", DP), ("v_bath", DP)]


class ed_sector_info(C.Structure):
    _fields_ = [("ns", C.c_int32), ("norb", C.c_int32), ("nbath", C.c_int32),
                ("nup", C.c_int32), ("ndw", C.c_int32), ("dim_up", C.c_int64),
                ("dim_dw", C.c_int64), ("dim", C.c_int64), ("nnz_up", C.c_int64),
                ("nnz_dw", C.c_int64), ("device_bytes", C.c_int64),
                ("blocked_stride", C.c_int64), ("blocked_dim", C.c_int64)]


class ed_lanczos_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("max_iter", C.c_int32), ("tol", C.c_double),
                ("seed", C.c_uint64), ("polish_steps", C.c_int32), ("want_vector", C.c_int32),
                ("basis_mib", C.c_int32), ("reserved", C.c_int32)]


class ed_lanczos_result(C.Structure):
    _fields_ = [("e0", C.c_double), ("e0_raw", C.c_double), ("residual", C.c_double),
                ("residual_estimate", C.c_double), ("iterations", C.c_int32),
                ("polish_iterations", C.c_int32), ("stop_reason", C.c_int32),
                ("matvecs", C.c_int32), ("matvecs_fp64", C.c_int32), ("reserved", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


ED_MAX_NORB = 5


class ed_phonon(C.Structure):
    _fields_ = [("w0", C.c_double), ("g", C.c_double * ED_MAX_NORB), ("nph", C.c_int32),
                ("reserved", C.c_int32)]


class ed_gf_info(C.Structure):
    _fields_ = [("weight_particle", C.c_double), ("weight_hole", C.c_double),
                ("steps_particle", C.c_int32), ("steps_hole", C.c_int32)]


class ed_solve_opts(C.Structure):
    _fields_ = [("lanczos", ed_lanczos_opts), ("gf_steps", C.c_int32), ("nmats", C.c_int32),
                ("beta", C.c_double), ("gf_precision", C.c_int)]


class ed_solve_result(C.Structure):
    _fields_ = [("ground", ed_lanczos_result), ("t_build_s", C.c_double),
                ("t_ground_s", C.c_double), ("t_gf_s", C.c_double), ("gf_chains", C.c_int32),
                ("gf_steps_total", C.c_int32), ("gf_product_bytes", C.c_double)]


class ed_server_opts(C.Structure):
    _fields_ = [("slots", C.c_int32), ("device_mem_budget", C.c_int64),
                ("queue_capacity", C.c_int32)]


class ed_request(C.Structure):
    _fields_ = [("model", ed_model), ("nup", C.c_int32), ("ndw", C.c_int32),
                ("opts", ed_solve_opts)]


class ed_result(C.Structure):
    _fields_ = [("status", C.c_int), ("e0", C.c_double), ("ground", ed_lanczos_result),
                ("norb", C.c_int32), ("nmats", C.c_int32), ("t_submit_s", C.c_double),
                ("t_start_s", C.c_double), ("t_done_s", C.c_double)]


# ----------------------------------------------------------------- loading

_lib = None
_lock = threading.Lock()


def lib():
    """The loaded CUDA library; raises when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                "(the exact-diagonalisation path has no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
        sig = {
            "ed_sector_build": [C.POINTER(ed_model), i32, i32, vp, C.POINTER(vp)],
            "ed_sector_get_info": [vp, C.POINTER(ed_sector_info)],
            "ed_sector_copy_tables": [vp, i32, vp, vp, vp, vp, vp, vp],
            "ed_sector_copy_w": [vp, vp],
            "ed_sector_free": [vp],
            "ed_matvec": [vp, C.c_int, vp, vp, i64, vp],
            "ed_matvec_blocked": [vp, C.c_int, vp, vp, i64, vp],
            "ed_sector_blocked_kernel": [vp, C.c_int, C.POINTER(i32)],
            "ed_sector_tune_info": [vp, C.c_int, C.POINTER(i32), vp],
            "ed_sector_set_kernel": [vp, C.c_int, i32],
            "ed_sector_permute": [vp, C.c_int, i32, vp, i64, vp, i64, vp],
            "ed_lanczos_ground": [vp, C.POINTER(ed_lanczos_opts), C.POINTER(ed_lanczos_result),
                                  vp, vp],
            "ed_gf_lanczos": [vp, C.c_int, vp, C.c_double, i32, i32, i32, C.c_double, i32, vp,
                              C.POINTER(ed_gf_info), vp],
            "ed_solve": [C.POINTER(ed_model), i32, i32, C.POINTER(ed_solve_opts),
                         C.POINTER(ed_solve_result), vp, vp, vp],
            "ed_server_create": [C.POINTER(ed_server_opts), C.POINTER(vp)],
            "ed_submit": [vp, C.POINTER(ed_request), C.POINTER(u64)],
            "ed_poll": [vp, u64, C.POINTER(ed_result), vp],
            "ed_wait": [vp, u64, C.c_double],
            "ed_server_destroy": [vp],
            "ed_server_inject_alloc_failure": [vp, i32],
            "ed_residual_noalloc": [vp, vp, i64, vp, vp],
            "ed_batch_stats": [C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)],
            "ed_memory_trim": [i64],
            "ed_memory_cached": [C.POINTER(i64), C.POINTER(i64)],
            "ed_gf_lanczos_z": [vp, C.c_int, vp, C.c_double, i32, i32, i32, vp, i32, vp,
                                C.POINTER(ed_gf_info), vp],
            "ed_sigma": [C.POINTER(ed_model), i32, i32, vp, i32, vp, vp, vp],
            "ed_observables": [vp, C.c_int, vp, i64, vp, vp],
            "ed_eph_matvec": [vp, C.POINTER(ed_phonon), C.c_int, vp, vp, i64, vp],
            "ed_eph_lanczos_ground": [vp, C.POINTER(ed_phonon), C.POINTER(ed_lanczos_opts),
                                      C.POINTER(ed_lanczos_result), vp, vp],
            "ed_eph_gf_lanczos_z": [vp, C.POINTER(ed_phonon), C.c_int, vp, C.c_double, i32, i32,
                                    i32, vp, i32, vp, C.POINTER(ed_gf_info), vp],
            "ed_lanczos_states": [vp, C.POINTER(ed_lanczos_opts), i32, vp,
                                  C.POINTER(ed_lanczos_result), vp, vp],
            "ed_espace_truncate": [i32, vp, vp, C.c_double, C.c_double, i32, i32, vp, vp,
                                   C.POINTER(i32)],
            "ed_gf_thermal_z": [i32, vp, vp, vp, C.c_double, C.c_double, i32, C.c_int, i32, i32,
                                i32, vp, i32, vp, vp, vp],
            "ed_chi_z": [vp, C.c_int, vp, C.c_double, i32, i32, i32, vp, i32, vp, vp, vp],
            "ed_chi_ab_z": [vp, C.c_int, vp, C.c_double, i32, i32, i32, i32, vp, i32, vp, vp],
            "ed_chi_tau": [vp, C.c_int, vp, C.c_double, i32, i32, i32, C.c_double, vp, i32, vp,
                           vp],
            "ed_orbital_sector_dims": [vp, vp, vp, C.POINTER(i64), C.POINTER(i64)],
            "ed_lanczos_ground_orbital": [vp, vp, vp, C.POINTER(ed_lanczos_opts),
                                          C.POINTER(ed_lanczos_result), vp, vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.ed_status_string.argtypes = [C.c_int]
        L.ed_status_string.restype = C.c_char_p
        L.ed_last_error.argtypes = []
        L.ed_last_error.restype = C.c_char_p
        L.ed_kernel_launches.argtypes = []
        L.ed_kernel_launches.restype = i64
        _lib = L
        return L


def _check(st, what):
    if st != ED_OK:
        raise EDError(st, what)


def kernel_launches() -> int:
    return int(lib().ed_kernel_launches())


def _stream_ptr(stream=None):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ----------------------------------------------------------------- model

class Model:
    """ed_model with owned contiguous arrays (any object with the fields of
    workloads.ImpurityModel)."""

    def __init__(self, m):
        self.norb, self.nbath = int(m.norb), int(m.nbath)
        self.e_imp = np.ascontiguousarray(np.broadcast_to(m.e_imp, (2, self.norb)), dtype=np.float64)
        self.e_bath = np.ascontiguousarray(
            np.broadcast_to(m.e_bath, (2, self.norb, self.nbath)), dtype=np.float64)
        self.v_bath = np.ascontiguousarray(
            np.broadcast_to(m.v_bath, (2, self.norb, self.nbath)), dtype=np.float64)
        self.c = ed_model(self.norb, self.nbath, float(m.U), float(m.Ust), float(m.Jh),
                          float(getattr(m, "Jx", 0.0)), float(getattr(m, "Jp", 0.0)),
                          self.e_imp.ctypes.data_as(DP), self.e_bath.ctypes.data_as(DP),
                          self.v_bath.ctypes.data_as(DP))

    @property
    def ns(self):
        return self.norb * (self.nbath + 1)


def as_model(m) -> Model:
    return m if isinstance(m, Model) else Model(m)


# ----------------------------------------------------------------- sector

class Sector:
    """Owns an ed_sector handle (device LUTs, CSR and diagonal tables)."""

    def __init__(self, model, nup, ndw, stream=None):
        self.model = as_model(model)
        h = C.c_void_p()
        _check(lib().ed_sector_build(C.byref(self.model.c), int(nup), int(ndw),
                                     C.c_void_p(_stream_ptr(stream)), C.byref(h)),
               "ed_sector_build")
        self.h = h
        inf = ed_sector_info()
        _check(lib().ed_sector_get_info(self.h, C.byref(inf)), "ed_sector_get_info")
        self.info = {k: getattr(inf, k) for k, _ in inf._fields_}
        self.nup, self.ndw = int(nup), int(ndw)
        self.dim = self.info["dim"]
        self.dim_up, self.dim_dw = self.info["dim_up"], self.info["dim_dw"]
        self.blocked_dim = self.info["blocked_dim"]
        self.blocked_stride = self.info["blocked_stride"]
        import torch
        self.device = torch.cuda.current_device()  # the device holding the tables

    def free(self):
        if self.h:
            _check(lib().ed_sector_free(self.h), "ed_sector_free")
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.free()

    def tables(self, spin):
        d = self.dim_up if spin == 0 else self.dim_dw
        nnz = self.info["nnz_up"] if spin == 0 else self.info["nnz_dw"]
        out = dict(map=np.zeros(d, np.uint32), rowptr=np.zeros(d + 1, np.int32),
                   col=np.zeros(max(nnz, 1), np.int32), val=np.zeros(max(nnz, 1), np.float64),
                   ediag=np.zeros(d, np.float64), imask=np.zeros(d, np.uint8))
        _check(lib().ed_sector_copy_tables(
            self.h, int(spin), out["map"].ctypes.data, out["rowptr"].ctypes.data,
            out["col"].ctypes.data, out["val"].ctypes.data, out["ediag"].ctypes.data,
            out["imask"].ctypes.data), "ed_sector_copy_tables")
        out["col"], out["val"] = out["col"][:nnz], out["val"][:nnz]
        return out

    def blocked_kernel(self, precision="fp32"):
        """Product kernel of the block-major layout in `precision`: "tiled",
        "elementwise" or "two_pass" (ed_sector_blocked_kernel)."""
        k = C.c_int32()
        _check(lib().ed_sector_blocked_kernel(self.h, _prec(precision), C.byref(k)),
               "ed_sector_blocked_kernel")
        return {0: "tiled", 1: "elementwise", 2: "two_pass"}[k.value]

    def tune_info(self, precision="fp32"):
        """(kernel in use, {"tiled": ms, "elementwise": ms}) of the autotuner
        (ed_sector_tune_info; -1 ms where this sector did not time a kernel)."""
        k = C.c_int32()
        ms = np.zeros(2)
        _check(lib().ed_sector_tune_info(self.h, _prec(precision), C.byref(k), ms.ctypes.data),
               "ed_sector_tune_info")
        return {0: "tiled", 1: "elementwise", 2: "two_pass"}[k.value], \
            {"tiled": float(ms[0]), "elementwise": float(ms[1])}

    def set_kernel(self, kernel, precision="fp32"):
        """Pin the block-major product kernel of this sector (ed_sector_set_kernel)."""
        code = {"tiled": 0, "elementwise": 1, "two_pass": 2}[kernel]
        _check(lib().ed_sector_set_kernel(self.h, _prec(precision), code), "ed_sector_set_kernel")

    def wtable(self):
        nm = 1 << self.model.norb
        w = np.zeros((nm, nm))
        _check(lib().ed_sector_copy_w(self.h, w.ctypes.data), "ed_sector_copy_w")
        return w


def _prec(p):
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def _psi_ptr(psi, precision):
    """Device pointer of a ground state handed to a chain or an observable:
    a contiguous CUDA tensor, float64 for fp64 / fp32_polish, float32 for
    fp32 (the layout the C-ABI reads)."""
    import torch
    want = torch.float32 if _prec(precision) == PRECISIONS["fp32"] else torch.float64
    if not (psi.is_cuda and psi.is_contiguous() and psi.dtype == want):
        raise ValueError(f"psi must be a contiguous CUDA {want} tensor for {precision!r}")
    return C.c_void_p(psi.data_ptr())


def matvec(sector: Sector, v, w, precision="fp64", stream=None):
    """w = H v for device tensors (float64 for fp64, float32 otherwise)."""
    if v.numel() != w.numel():
        raise ValueError("v and w differ in length")
    _check(lib().ed_matvec(sector.h, _prec(precision), C.c_void_p(v.data_ptr()),
                           C.c_void_p(w.data_ptr()), int(v.numel()),
                           C.c_void_p(_stream_ptr(stream))), "ed_matvec")


def matvec_blocked(sector: Sector, v, w, precision="fp64", stream=None):
    """w = H v with both vectors in block-major order."""
    if v.numel() != w.numel():
        raise ValueError("v and w differ in length")
    _check(lib().ed_matvec_blocked(sector.h, _prec(precision), C.c_void_p(v.data_ptr()),
                                   C.c_void_p(w.data_ptr()), int(v.numel()),
                                   C.c_void_p(_stream_ptr(stream))), "ed_matvec_blocked")


def permute(sector: Sector, x, out, to_blocked=True, precision="fp64", stream=None):
    """Converts a sector vector between sector order and block-major order."""
    _check(lib().ed_sector_permute(sector.h, _prec(precision), int(bool(to_blocked)),
                                   C.c_void_p(x.data_ptr()), int(x.numel()),
                                   C.c_void_p(out.data_ptr()), int(out.numel()),
                                   C.c_void_p(_stream_ptr(stream))), "ed_sector_permute")


def trim_memory(keep_bytes=0):
    """Return the library pool's cached device blocks beyond keep_bytes to
    the device (ed_memory_trim; like torch.cuda.empty_cache for PyTorch)."""
    _check(lib().ed_memory_trim(int(keep_bytes)), "ed_memory_trim")


def memory_cached():
    """(reserved, used) bytes of the library's device pool (ed_memory_cached)."""
    r, u = C.c_int64(), C.c_int64()
    _check(lib().ed_memory_cached(C.byref(r), C.byref(u)), "ed_memory_cached")
    return r.value, u.value


def batch_stats():
    """Counters of the batched Green's-function launches of this process
    (ed_batch_stats): launches, chains run in them, most solves merged into
    one launch."""
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().ed_batch_stats(C.byref(a), C.byref(b), C.byref(c)), "ed_batch_stats")
    return {"launches": a.value, "chains": b.value, "max_solves": c.value}


def residual_noalloc(sector: Sector, psi, stream=None):
    """(E, ||H psi - E psi|| / ||psi||) of an FP64 sector-order vector without
    any device allocation (scratch in a static device array; the sector
    dimension must not exceed ED_NOALLOC_MAX_DIM = 2**20).

    ``psi`` must be a contiguous float64 CUDA tensor on the sector's device:
    the C entry point reads it as ``double`` elements, so anything else is
    rejected here with ED_ERR_ARG before the library is called."""
    import torch
    if not (isinstance(psi, torch.Tensor) and psi.dtype == torch.float64 and psi.is_cuda
            and psi.is_contiguous() and psi.device.index == getattr(sector, "device", None)):
        raise EDError(ED_ERR_ARG, "ed_residual_noalloc: psi must be a contiguous float64 "
                                  "CUDA tensor on the sector's device")
    out = np.zeros(2, dtype=np.float64)
    _check(lib().ed_residual_noalloc(sector.h, C.c_void_p(psi.data_ptr()), int(psi.numel()),
                                     C.c_void_p(out.ctypes.data), C.c_void_p(_stream_ptr(stream))),
           "ed_residual_noalloc")
    return float(out[0]), float(out[1])


def lanczos_ground(sector: Sector, precision="fp64", max_iter=0, tol=0.0, seed=0x5EED,
                   polish_steps=0, psi=None, want_vector=None, stream=None, allow_maxit=False,
                   basis_mib=0):
    o = ed_lanczos_opts(_prec(precision), int(max_iter), float(tol), int(seed),
                        int(polish_steps), int(bool(psi is not None) if want_vector is None
                                               else bool(want_vector)), int(basis_mib), 0)
    r = ed_lanczos_result()
    st = lib().ed_lanczos_ground(sector.h, C.byref(o), C.byref(r),
                                 C.c_void_p(psi.data_ptr() if psi is not None else 0),
                                 C.c_void_p(_stream_ptr(stream)))
    if st == ED_ERR_NOT_CONVERGED and allow_maxit:
        st = ED_OK
    _check(st, "ed_lanczos_ground")
    return r.as_dict()


def gf_lanczos(sector: Sector, psi, e0, orb, spin, precision="fp64", nsteps=200, beta=100.0,
               nmats=512, stream=None):
    G = np.zeros(2 * nmats, dtype=np.float64)
    info = ed_gf_info()
    _check(lib().ed_gf_lanczos(sector.h, _prec(precision), _psi_ptr(psi, precision),
                               float(e0), int(orb), int(spin), int(nsteps), float(beta),
                               int(nmats), G.ctypes.data, C.byref(info),
                               C.c_void_p(_stream_ptr(stream))), "ed_gf_lanczos")
    return G.view(np.complex128), {k: getattr(info, k) for k, _ in info._fields_}


def gf_lanczos_z(sector: Sector, psi, e0, orb, spin, z, precision="fp64", nsteps=200,
                 stream=None):
    """G_{orb,spin}(z) at arbitrary complex frequencies z (ed_gf_lanczos_z):
    z = 1j * w_n gives the Matsubara axis, z = w + 1j * eta the real axis."""
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.complex128).reshape(-1))
    G = np.zeros(zz.size, dtype=np.complex128)
    info = ed_gf_info()
    _check(lib().ed_gf_lanczos_z(sector.h, _prec(precision), _psi_ptr(psi, precision),
                                 float(e0), int(orb), int(spin), int(nsteps),
                                 C.c_void_p(zz.ctypes.data), int(zz.size),
                                 C.c_void_p(G.ctypes.data), C.byref(info),
                                 C.c_void_p(_stream_ptr(stream))), "ed_gf_lanczos_z")
    return G, {k: getattr(info, k) for k, _ in info._fields_}


def sigma(model, orb, spin, z, G, stream=None):
    """Sigma(z) = G0(z)^-1 - G(z)^-1 of the model's normal bath (ed_sigma)."""
    m = as_model(model)
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.complex128).reshape(-1))
    gg = np.ascontiguousarray(np.asarray(G, dtype=np.complex128).reshape(-1))
    if gg.size != zz.size:
        raise EDError(ED_ERR_ARG, "sigma: G and z differ in length")
    out = np.zeros(zz.size, dtype=np.complex128)
    _check(lib().ed_sigma(C.byref(m.c), int(orb), int(spin), C.c_void_p(zz.ctypes.data),
                          int(zz.size), C.c_void_p(gg.ctypes.data), C.c_void_p(out.ctypes.data),
                          C.c_void_p(_stream_ptr(stream))), "ed_sigma")
    return out


def observables(sector: Sector, psi, precision="fp64", stream=None):
    """Impurity densities, density-density correlators and interaction energy
    of a sector-order state (ed_observables): dict with dens[2][norb],
    nn[2][2][norb][norb], e_int, norm."""
    no = sector.info["norb"]
    out = np.zeros(2 * no + 4 * no * no + 2, dtype=np.float64)
    _check(lib().ed_observables(sector.h, _prec(precision), _psi_ptr(psi, precision),
                                int(psi.numel()), C.c_void_p(out.ctypes.data),
                                C.c_void_p(_stream_ptr(stream))), "ed_observables")
    return {"dens": out[:2 * no].reshape(2, no).copy(),
            "nn": out[2 * no:2 * no + 4 * no * no].reshape(2, 2, no, no).copy(),
            "e_int": float(out[-2]), "norm": float(out[-1])}


def phonon(w0, g, nph):
    """ed_phonon record: frequency w0, couplings g[alpha] (zero-padded), cut-off N_ph."""
    gg = np.zeros(ED_MAX_NORB)
    gv = np.atleast_1d(np.asarray(g, dtype=np.float64))
    gg[:gv.size] = gv
    return ed_phonon(float(w0), (C.c_double * ED_MAX_NORB)(*gg), int(nph), 0)


def eph_matvec(sector: Sector, ph, v, w, precision="fp64", stream=None):
    """w = H v on the coupled electron-phonon sector (ed_eph_matvec); v, w of
    D * (nph + 1) elements, phonon index slowest."""
    _check(lib().ed_eph_matvec(sector.h, C.byref(ph), _prec(precision), C.c_void_p(v.data_ptr()),
                               C.c_void_p(w.data_ptr()), int(v.numel()),
                               C.c_void_p(_stream_ptr(stream))), "ed_eph_matvec")


def eph_lanczos_ground(sector: Sector, ph, precision="fp64", max_iter=0, tol=0.0, seed=0x5EED,
                       polish_steps=0, psi=None, stream=None):
    o = ed_lanczos_opts(_prec(precision), int(max_iter), float(tol), int(seed),
                        int(polish_steps), 1, 0, 0)
    r = ed_lanczos_result()
    _check(lib().ed_eph_lanczos_ground(sector.h, C.byref(ph), C.byref(o), C.byref(r),
                                       C.c_void_p(psi.data_ptr() if psi is not None else 0),
                                       C.c_void_p(_stream_ptr(stream))), "ed_eph_lanczos_ground")
    return r.as_dict()


def eph_gf_lanczos_z(sector: Sector, ph, psi, e0, orb, spin, z, precision="fp64", nsteps=200,
                     stream=None):
    """G(z) of the coupled model (ed_eph_gf_lanczos_z)."""
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.complex128).reshape(-1))
    G = np.zeros(zz.size, dtype=np.complex128)
    info = ed_gf_info()
    _check(lib().ed_eph_gf_lanczos_z(sector.h, C.byref(ph), _prec(precision),
                                     C.c_void_p(psi.data_ptr()), float(e0), int(orb), int(spin),
                                     int(nsteps), C.c_void_p(zz.ctypes.data), int(zz.size),
                                     C.c_void_p(G.ctypes.data), C.byref(info),
                                     C.c_void_p(_stream_ptr(stream))), "ed_eph_gf_lanczos_z")
    return G, {k: getattr(info, k) for k, _ in info._fields_}


def _occ(t):
    a = np.ascontiguousarray(np.asarray(t, dtype=np.int32))
    return a, C.c_void_p(a.ctypes.data)


def orbital_sector_dims(sector: Sector, nup_orb, ndw_orb):
    """(D_up, D_dw) of the finer sector with these per-orbital occupations."""
    (a, pa), (b, pb) = _occ(nup_orb), _occ(ndw_orb)
    du, dd = C.c_int64(), C.c_int64()
    _check(lib().ed_orbital_sector_dims(sector.h, pa, pb, C.byref(du), C.byref(dd)),
           "ed_orbital_sector_dims")
    return int(du.value), int(dd.value)


def lanczos_ground_orbital(sector: Sector, nup_orb, ndw_orb, precision="fp64", max_iter=0,
                           tol=0.0, seed=0x5EED, polish_steps=0, psi=None, stream=None):
    """Ground state of a finer (per-orbital) sector (ed_lanczos_ground_orbital);
    psi (optional, D elements) receives it in the sector order of `sector`."""
    (a, pa), (b, pb) = _occ(nup_orb), _occ(ndw_orb)
    o = ed_lanczos_opts(_prec(precision), int(max_iter), float(tol), int(seed),
                        int(polish_steps), 1, 0, 0)
    r = ed_lanczos_result()
    _check(lib().ed_lanczos_ground_orbital(sector.h, pa, pb, C.byref(o), C.byref(r),
                                           C.c_void_p(psi.data_ptr() if psi is not None else 0),
                                           C.c_void_p(_stream_ptr(stream))),
           "ed_lanczos_ground_orbital")
    return r.as_dict()


CHI_KINDS = {"spin": 0, "charge": 1, "pair": 2, "exciton": 3}


def chi_z(sector: Sector, psi, e0, kind, orb, z, precision="fp64", nsteps=200, stream=None):
    """Impurity susceptibility C_O(z) at T = 0 (ed_chi_z): kind "spin"
    (S^z), "charge" (n) or "pair" (d_dw d_up); returns (C, (n+, n-))."""
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.complex128).reshape(-1))
    out = np.zeros(zz.size, dtype=np.complex128)
    w = np.zeros(2)
    _check(lib().ed_chi_z(sector.h, _prec(precision), _psi_ptr(psi, precision), float(e0),
                          CHI_KINDS[kind], int(orb), int(nsteps), C.c_void_p(zz.ctypes.data),
                          int(zz.size), C.c_void_p(out.ctypes.data), C.c_void_p(w.ctypes.data),
                          C.c_void_p(_stream_ptr(stream))), "ed_chi_z")
    return out, (float(w[0]), float(w[1]))


def chi_tau(sector: Sector, psi, e0, kind, orb, tau, beta, precision="fp64", nsteps=200,
            stream=None):
    """Susceptibility C(tau) at T = 0 for tau in [0, beta] (ed_chi_tau)."""
    tt = np.ascontiguousarray(np.asarray(tau, dtype=np.float64).reshape(-1))
    out = np.zeros(tt.size, dtype=np.float64)
    _check(lib().ed_chi_tau(sector.h, _prec(precision), _psi_ptr(psi, precision), float(e0),
                            CHI_KINDS[kind], int(orb), int(nsteps), float(beta),
                            C.c_void_p(tt.ctypes.data), int(tt.size),
                            C.c_void_p(out.ctypes.data), C.c_void_p(_stream_ptr(stream))),
           "ed_chi_tau")
    return out


def chi_ab_z(sector: Sector, psi, e0, kind, orb_a, orb_b, z, precision="fp64", nsteps=200,
             stream=None):
    """Inter-orbital spin or charge function C_ab(z) at T = 0, or the
    excitonic function of the orbital pair (kind "exciton") (ed_chi_ab_z)."""
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.complex128).reshape(-1))
    out = np.zeros(zz.size, dtype=np.complex128)
    _check(lib().ed_chi_ab_z(sector.h, _prec(precision), _psi_ptr(psi, precision), float(e0),
                             CHI_KINDS[kind], int(orb_a), int(orb_b), int(nsteps),
                             C.c_void_p(zz.ctypes.data), int(zz.size),
                             C.c_void_p(out.ctypes.data), C.c_void_p(_stream_ptr(stream))),
           "ed_chi_ab_z")
    return out


def lanczos_states(sector: Sector, nstates, precision="fp64", max_iter=0, tol=0.0,
                   seed=0x5EED, polish_steps=0, psis=None, stream=None):
    """The nstates lowest eigenpairs of the sector (ed_lanczos_states): returns
    (energies, [result dicts]); psis (optional device tensor of nstates x D)
    receives the states in sector order."""
    o = ed_lanczos_opts(_prec(precision), int(max_iter), float(tol), int(seed),
                        int(polish_steps), 1, 0, 0)
    E = np.zeros(int(nstates))
    res = (ed_lanczos_result * int(nstates))()
    _check(lib().ed_lanczos_states(sector.h, C.byref(o), int(nstates), C.c_void_p(E.ctypes.data),
                                   res, C.c_void_p(psis.data_ptr() if psis is not None else 0),
                                   C.c_void_p(_stream_ptr(stream))), "ed_lanczos_states")
    return E, [r.as_dict() for r in res]


def espace_truncate(energies_per_sector, beta, cutoff, ntotal=0, step=2):
    """Annealing truncation of the eigenspace list (ed_espace_truncate):
    returns (weights per sector, next state counts, number kept)."""
    counts = np.array([len(e) for e in energies_per_sector], dtype=np.int32)
    flat = np.ascontiguousarray(np.concatenate([np.asarray(e, dtype=np.float64)
                                                for e in energies_per_sector]))
    w = np.zeros(flat.size)
    nxt = np.zeros(counts.size, dtype=np.int32)
    nk = C.c_int32()
    _check(lib().ed_espace_truncate(int(counts.size), C.c_void_p(counts.ctypes.data),
                                    C.c_void_p(flat.ctypes.data), float(beta), float(cutoff),
                                    int(ntotal), int(step), C.c_void_p(w.ctypes.data),
                                    C.c_void_p(nxt.ctypes.data), C.byref(nk)),
           "ed_espace_truncate")
    out, o = [], 0
    for c in counts:
        out.append(w[o:o + c].copy())
        o += c
    return out, [int(x) for x in nxt], int(nk.value)


def gf_thermal_z(sectors, psis, energies, beta, cutoff, orb, spin, z, precision="fp64",
                 nsteps=200, ntotal=0, stream=None):
    """Finite-temperature G(z) = sum_i w_i G_i(z) (ed_gf_thermal_z): returns
    (G, weights)."""
    n = len(sectors)
    hs = (C.c_void_p * n)(*[s.h for s in sectors])
    ps = (C.c_void_p * n)(*[_psi_ptr(p, precision).value for p in psis])
    E = np.ascontiguousarray(np.asarray(energies, dtype=np.float64))
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.complex128).reshape(-1))
    G = np.zeros(zz.size, dtype=np.complex128)
    w = np.zeros(n)
    _check(lib().ed_gf_thermal_z(n, hs, ps, C.c_void_p(E.ctypes.data), float(beta), float(cutoff),
                                 int(ntotal), _prec(precision), int(orb), int(spin), int(nsteps),
                                 C.c_void_p(zz.ctypes.data), int(zz.size),
                                 C.c_void_p(G.ctypes.data), C.c_void_p(w.ctypes.data),
                                 C.c_void_p(_stream_ptr(stream))), "ed_gf_thermal_z")
    return G, w


def solve_opts(precision="fp32_polish", gf_precision=None, nmats=512, beta=100.0,
               gf_steps=200, max_iter=0, tol=0.0, seed=0x5EED, polish_steps=0, basis_mib=0):
    p = _prec(precision)
    gp = _prec(gf_precision) if gf_precision is not None else (FP64 if p == FP64 else FP32)
    return ed_solve_opts(ed_lanczos_opts(p, int(max_iter), float(tol), int(seed),
                                         int(polish_steps), 0, int(basis_mib), 0),
                         int(gf_steps), int(nmats), float(beta), gp)


def solve(model, nup, ndw, stream=None, psi=None, **kw):
    """One impurity solve (ed_solve): returns (result dict, G[2][norb][nmats]);
    `psi` (optional device tensor of D elements) receives the ground state."""
    m = as_model(model)
    o = solve_opts(**kw)
    r = ed_solve_result()
    G = np.zeros(2 * 2 * m.norb * max(o.nmats, 0), dtype=np.float64)
    _check(lib().ed_solve(C.byref(m.c), int(nup), int(ndw), C.byref(o), C.byref(r),
                          C.c_void_p(G.ctypes.data if o.nmats > 0 else 0),
                          C.c_void_p(psi.data_ptr() if psi is not None else 0),
                          C.c_void_p(_stream_ptr(stream))), "ed_solve")
    out = r.ground.as_dict()
    out.update(t_build_s=r.t_build_s, t_ground_s=r.t_ground_s, t_gf_s=r.t_gf_s,
               gf_chains=r.gf_chains, gf_steps_total=r.gf_steps_total,
               gf_product_bytes=r.gf_product_bytes)
    return out, G.view(np.complex128).reshape(2, m.norb, max(o.nmats, 0))


class Server:
    """Continuous-batching request loop (ed_server_*)."""

    def __init__(self, slots=8, device_mem_budget=0, queue_capacity=0):
        o = ed_server_opts(int(slots), int(device_mem_budget), int(queue_capacity))
        h = C.c_void_p()
        _check(lib().ed_server_create(C.byref(o), C.byref(h)), "ed_server_create")
        self.h = h
        self._keep = {}

    def submit(self, model, nup, ndw, **kw):
        m = as_model(model)
        req = ed_request(m.c, int(nup), int(ndw), solve_opts(**kw))
        t = C.c_uint64()
        st = lib().ed_submit(self.h, C.byref(req), C.byref(t))
        if st != ED_OK:
            raise EDError(st, "ed_submit")
        self._keep[t.value] = (m.norb, req.opts.nmats)
        return t.value

    def poll(self, ticket):
        """None while pending; else (result dict, G[2][norb][nmats])."""
        norb, nmats = self._keep.get(ticket, (1, 0))
        r = ed_result()
        G = np.zeros(2 * 2 * norb * max(nmats, 0) + 2, dtype=np.float64)
        st = lib().ed_poll(self.h, C.c_uint64(ticket), C.byref(r), C.c_void_p(G.ctypes.data))
        if st == ED_PENDING:
            return None
        _check(st, "ed_poll")
        self._keep.pop(ticket, None)
        out = r.ground.as_dict()
        out.update(status=r.status, e0=r.e0, t_submit_s=r.t_submit_s, t_start_s=r.t_start_s,
                   t_done_s=r.t_done_s)
        return out, G[:-2].view(np.complex128).reshape(2, norb, max(nmats, 0))

    def wait(self, ticket, timeout_s=60.0):
        return lib().ed_wait(self.h, C.c_uint64(ticket), float(timeout_s))

    def inject_alloc_failure(self, count):
        _check(lib().ed_server_inject_alloc_failure(self.h, int(count)), "inject")

    def close(self):
        if self.h:
            _check(lib().ed_server_destroy(self.h), "ed_server_destroy")
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
