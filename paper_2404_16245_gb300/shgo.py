"""Thin ctypes binding of libshgo.so (the C ABI declared in include/shgo.h).

Argument marshalling only: every step of the integral path runs in the library's CUDA kernels.
PyTorch supplies device memory and streams.  Importing this module loads the library and fails
loudly if it has not been built (``__graft_entry__.build()`` or ``python -m
paper_2404_16245_gb300.build``); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SHGO_OK = 0
SHGO_PREC_FP64 = 0
SHGO_PREC_FP32_BULK = 1
SHGO_PREC_FP32_PLAIN = 2
LMAX = 8

_STATUS = {0: "SHGO_OK", 1: "SHGO_ERR_INVALID_ARG", 2: "SHGO_ERR_UNSUPPORTED_L", 3: "SHGO_ERR_OOM",
           4: "SHGO_ERR_CUDA", 5: "SHGO_ERR_TIMEOUT", 6: "SHGO_ERR_NUMERIC"}


class ShgoError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class shgo_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("device", ctypes.c_int32), ("flags", ctypes.c_int32)]


SHGO_FLAG_BLOCK_SPARSE = 1
SHGO_FLAG_NO_PRIM_BOUND = 2


class shgo_centers(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("xyz", ctypes.c_void_p)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libshgo.so is not built ({_build.LIB}); run __graft_entry__.build()")
    lib = ctypes.CDLL(_build.LIB)
    i32p = ctypes.POINTER(ctypes.c_int32)
    f64p = ctypes.POINTER(ctypes.c_double)
    lib.shgo_basis_create.argtypes = [ctypes.c_int32, i32p, i32p, f64p, f64p, f64p, ctypes.POINTER(shgo_options),
                                      ctypes.POINTER(ctypes.c_void_p)]
    lib.shgo_basis_create.restype = ctypes.c_int
    lib.shgo_basis_create_shard.argtypes = [ctypes.c_int32, i32p, i32p, f64p, f64p, f64p, ctypes.POINTER(shgo_options),
                                            ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]
    lib.shgo_basis_create_shard.restype = ctypes.c_int
    lib.shgo_host_shard_of_pairs.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                             i32p]
    lib.shgo_host_shard_of_pairs.restype = ctypes.c_int
    lib.shgo_basis_nbf.argtypes = [ctypes.c_void_p]
    lib.shgo_basis_nbf.restype = ctypes.c_int64
    lib.shgo_basis_npairs.argtypes = [ctypes.c_void_p]
    lib.shgo_basis_npairs.restype = ctypes.c_int64
    lib.shgo_nuclear_attraction.argtypes = [ctypes.c_void_p, ctypes.POINTER(shgo_centers), ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p]
    lib.shgo_nuclear_attraction.restype = ctypes.c_int
    lib.shgo_nuclear_attraction_timed.argtypes = [ctypes.c_void_p, ctypes.POINTER(shgo_centers), ctypes.c_void_p,
                                                  ctypes.c_void_p, ctypes.c_void_p, f64p]
    lib.shgo_nuclear_attraction_timed.restype = ctypes.c_int
    lib.shgo_nuclear_attraction_noalloc.argtypes = [ctypes.c_int32, i32p, i32p, f64p, f64p, f64p,
                                                    ctypes.POINTER(shgo_centers), ctypes.c_void_p, ctypes.c_void_p,
                                                    ctypes.c_void_p]
    lib.shgo_nuclear_attraction_noalloc.restype = ctypes.c_int
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.shgo_batch_create.argtypes = [ctypes.c_int32, i32p, i64p, ctypes.c_int32, i32p, i32p, f64p, f64p, f64p,
                                      ctypes.POINTER(shgo_options), ctypes.POINTER(ctypes.c_void_p)]
    lib.shgo_batch_create.restype = ctypes.c_int
    lib.shgo_batch_layout.argtypes = [ctypes.c_void_p, i64p, i64p]
    lib.shgo_batch_layout.restype = ctypes.c_int
    lib.shgo_batch_out_size.argtypes = [ctypes.c_void_p]
    lib.shgo_batch_out_size.restype = ctypes.c_int64
    lib.shgo_nuclear_attraction_batched.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                    ctypes.c_void_p, ctypes.c_void_p]
    lib.shgo_nuclear_attraction_batched.restype = ctypes.c_int
    lib.shgo_basis_nclasses.argtypes = [ctypes.c_void_p]
    lib.shgo_basis_nclasses.restype = ctypes.c_int32
    lib.shgo_basis_class_stats.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, i32p, f64p]
    lib.shgo_basis_class_stats.restype = ctypes.c_int
    lib.shgo_nuclear_attraction_class_timed.argtypes = [ctypes.c_void_p, ctypes.POINTER(shgo_centers),
                                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, f64p]
    lib.shgo_nuclear_attraction_class_timed.restype = ctypes.c_int
    lib.shgo_esp.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(shgo_centers), ctypes.c_void_p,
                             ctypes.c_void_p]
    lib.shgo_esp.restype = ctypes.c_int
    lib.shgo_esp_gradient.argtypes = lib.shgo_esp.argtypes
    lib.shgo_esp_gradient.restype = ctypes.c_int
    lib.shgo_nuclear_attraction_deriv.argtypes = [ctypes.c_void_p, ctypes.POINTER(shgo_centers), ctypes.c_void_p,
                                                  ctypes.c_void_p, ctypes.c_void_p]
    lib.shgo_nuclear_attraction_deriv.restype = ctypes.c_int
    lib.shgo_nuclear_attraction_gradient.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(shgo_centers),
                                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.shgo_nuclear_attraction_gradient.restype = ctypes.c_int
    lib.shgo_nuclear_field.argtypes = lib.shgo_nuclear_attraction_deriv.argtypes
    lib.shgo_nuclear_field.restype = ctypes.c_int
    lib.shgo_host_deriv_transform.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, f64p, f64p, f64p]
    lib.shgo_host_deriv_transform.restype = ctypes.c_int
    lib.shgo_host_deriv_lowering.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, f64p]
    lib.shgo_host_deriv_lowering.restype = ctypes.c_int
    lib.shgo_overlap.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.shgo_overlap.restype = ctypes.c_int
    lib.shgo_coulomb_2c.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.shgo_coulomb_2c.restype = ctypes.c_int
    lib.shgo_eri.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.shgo_eri.restype = ctypes.c_int
    lib.shgo_eri_jk.argtypes = [ctypes.c_void_p] * 5
    lib.shgo_eri_jk.restype = ctypes.c_int
    lib.shgo_basis_flops.argtypes = [ctypes.c_void_p, ctypes.c_int64, f64p, f64p]
    lib.shgo_basis_flops.restype = ctypes.c_int
    lib.shgo_basis_deriv_flops.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, f64p]
    lib.shgo_basis_deriv_flops.restype = ctypes.c_int
    lib.shgo_basis_esp_flops.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, f64p]
    lib.shgo_basis_esp_flops.restype = ctypes.c_int
    lib.shgo_sparse_layout.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64)]
    lib.shgo_sparse_layout.restype = ctypes.c_int
    lib.shgo_basis_set_time_limit.argtypes = [ctypes.c_void_p, ctypes.c_double]
    lib.shgo_basis_set_time_limit.restype = ctypes.c_int
    lib.shgo_basis_sync.argtypes = [ctypes.c_void_p]
    lib.shgo_basis_sync.restype = ctypes.c_int
    lib.shgo_measure_fma_rate.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, f64p, f64p]
    lib.shgo_measure_fma_rate.restype = ctypes.c_int
    lib.shgo_measure_fma_rate_shape.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_void_p, f64p, f64p]
    lib.shgo_measure_fma_rate_shape.restype = ctypes.c_int
    lib.shgo_basis_launches.argtypes = [ctypes.c_void_p]
    lib.shgo_basis_launches.restype = ctypes.c_int64
    lib.shgo_free.argtypes = [ctypes.c_void_p]
    lib.shgo_free.restype = None
    lib.shgo_last_error.argtypes = []
    lib.shgo_last_error.restype = ctypes.c_char_p
    lib.shgo_host_solid_harmonics.argtypes = [ctypes.c_int32, ctypes.c_int64, f64p, f64p]
    lib.shgo_host_solid_harmonics.restype = ctypes.c_int
    lib.shgo_host_gaunt.argtypes = [ctypes.c_int32] * 6
    lib.shgo_host_gaunt.restype = ctypes.c_double
    lib.shgo_host_translation.argtypes = [ctypes.c_int32] * 5
    lib.shgo_host_translation.restype = ctypes.c_double
    lib.shgo_host_boys.argtypes = [ctypes.c_int32, ctypes.c_double, f64p]
    lib.shgo_host_boys.restype = ctypes.c_int
    lib.shgo_host_laplacian_coef.argtypes = [ctypes.c_int32] * 3
    lib.shgo_host_laplacian_coef.restype = ctypes.c_double
    lib.shgo_host_eri_eps.argtypes = [ctypes.c_int32] * 3
    lib.shgo_host_eri_eps.restype = ctypes.c_double
    return lib


_lib = _load()


def _check(status: int) -> None:
    if status != SHGO_OK:
        raise ShgoError(status, _lib.shgo_last_error().decode())


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    handle = getattr(stream, "cuda_stream", stream)
    return ctypes.c_void_p(int(handle) if handle else 0)


# ------------------------------------------------------------------ C-ABI names
def shgo_basis_create(n_shells, l, n_prim, exponents, coefs, shell_xyz, precision=SHGO_PREC_FP64, device=-1,
                      flags=0, shard=None):
    """Returns an opaque handle (int).  Host arrays are copied by the library.  shard = (index, count) builds
    that shard of the basis (shgo_basis_create_shard)."""
    l = np.ascontiguousarray(l, dtype=np.int32)
    n_prim = np.ascontiguousarray(n_prim, dtype=np.int32)
    exponents = np.ascontiguousarray(exponents, dtype=np.float64)
    coefs = np.ascontiguousarray(coefs, dtype=np.float64)
    shell_xyz = np.ascontiguousarray(shell_xyz, dtype=np.float64).reshape(-1)
    opt = shgo_options(int(precision), int(device), int(flags))
    handle = ctypes.c_void_p()
    args = (int(n_shells), _ptr(l, ctypes.c_int32), _ptr(n_prim, ctypes.c_int32), _ptr(exponents, ctypes.c_double),
            _ptr(coefs, ctypes.c_double), _ptr(shell_xyz, ctypes.c_double), ctypes.byref(opt))
    if shard is None:
        _check(_lib.shgo_basis_create(*args, ctypes.byref(handle)))
    else:
        _check(_lib.shgo_basis_create_shard(*args, int(shard[0]), int(shard[1]), ctypes.byref(handle)))
    return handle.value


def host_shard_of_pairs(l, n_prim, shard_count: int) -> np.ndarray:
    """Shard of every shell pair (library pair order) when one basis is split over shard_count devices."""
    l = np.ascontiguousarray(l, dtype=np.int32)
    n_prim = np.ascontiguousarray(n_prim, dtype=np.int32)
    n = ctypes.c_int64(0)
    _check(_lib.shgo_host_shard_of_pairs(len(l), _ptr(l, ctypes.c_int32), _ptr(n_prim, ctypes.c_int32),
                                         int(shard_count), ctypes.byref(n), None))
    out = np.zeros(max(n.value, 1), dtype=np.int32)
    _check(_lib.shgo_host_shard_of_pairs(len(l), _ptr(l, ctypes.c_int32), _ptr(n_prim, ctypes.c_int32),
                                         int(shard_count), ctypes.byref(n), _ptr(out, ctypes.c_int32)))
    return out[:n.value]


def shgo_nuclear_attraction(basis, n_centers, centers_ptr, charges_ptr, out_ptr, stream=None):
    """Raw call: device pointers as ints, stream a torch.cuda.Stream, a raw handle or None."""
    c = shgo_centers(int(n_centers), ctypes.c_void_p(int(centers_ptr) if centers_ptr else 0))
    _check(_lib.shgo_nuclear_attraction(ctypes.c_void_p(basis), ctypes.byref(c),
                                        ctypes.c_void_p(int(charges_ptr) if charges_ptr else 0),
                                        ctypes.c_void_p(int(out_ptr) if out_ptr else 0), _stream_handle(stream)))


def shgo_nuclear_attraction_timed(basis, n_centers, centers_ptr, charges_ptr, out_ptr, stream=None):
    """As shgo_nuclear_attraction; blocks and returns the two phase durations in ms."""
    c = shgo_centers(int(n_centers), ctypes.c_void_p(int(centers_ptr) if centers_ptr else 0))
    ms = np.zeros(2)
    _check(_lib.shgo_nuclear_attraction_timed(ctypes.c_void_p(basis), ctypes.byref(c),
                                              ctypes.c_void_p(int(charges_ptr) if charges_ptr else 0),
                                              ctypes.c_void_p(int(out_ptr) if out_ptr else 0), _stream_handle(stream),
                                              _ptr(ms, ctypes.c_double)))
    return float(ms[0]), float(ms[1])


def shgo_basis_flops(basis, n_centers: int):
    """(flops per phase [2], (shell triples, primitive triples)) of one call with n_centers nuclei."""
    f = np.zeros(2)
    t = np.zeros(2)
    _check(_lib.shgo_basis_flops(ctypes.c_void_p(basis), int(n_centers), _ptr(f, ctypes.c_double),
                                 _ptr(t, ctypes.c_double)))
    return f, t


def shgo_basis_deriv_flops(basis, n_centers: int, field: bool = False):
    """Algorithmic FP64 operations of one derivative (or field) call: (coupling, pair passes + combine)."""
    f = np.zeros(2)
    _check(_lib.shgo_basis_deriv_flops(ctypes.c_void_p(basis), int(n_centers), int(bool(field)),
                                       _ptr(f, ctypes.c_double)))
    return f


def shgo_basis_esp_flops(basis, n_points: int, gradient: bool = False):
    """Algorithmic FP64 operations of one potential (or gradient) call: (adjoint pass, per-point pass)."""
    f = np.zeros(2)
    _check(_lib.shgo_basis_esp_flops(ctypes.c_void_p(basis), int(n_points), int(bool(gradient)),
                                     _ptr(f, ctypes.c_double)))
    return f


def shgo_basis_set_time_limit(basis, seconds: float) -> None:
    _check(_lib.shgo_basis_set_time_limit(ctypes.c_void_p(basis), float(seconds)))


def shgo_basis_sync(basis) -> None:
    """Waits for the basis's last call; raises ShgoError (SHGO_ERR_TIMEOUT) if it hit the time limit."""
    _check(_lib.shgo_basis_sync(ctypes.c_void_p(basis)))


def shgo_measure_fma_rate(precision: int, iters: int, stream=None):
    """(flops per second, ms) of the FP64 or FP32 multiply-add microbenchmark (one timed launch)."""
    rate = ctypes.c_double()
    ms = ctypes.c_double()
    _check(_lib.shgo_measure_fma_rate(int(precision), int(iters), _stream_handle(stream), ctypes.byref(rate),
                                      ctypes.byref(ms)))
    return float(rate.value), float(ms.value)


def shgo_measure_fma_rate_shape(precision: int, iters: int, chains: int, threads_per_sm: int, stream=None):
    """(flops per second, ms) of the multiply-add microbenchmark with a chosen launch shape."""
    rate = ctypes.c_double()
    ms = ctypes.c_double()
    _check(_lib.shgo_measure_fma_rate_shape(int(precision), int(iters), int(chains), int(threads_per_sm),
                                            _stream_handle(stream), ctypes.byref(rate), ctypes.byref(ms)))
    return float(rate.value), float(ms.value)


def shgo_basis_launches(basis) -> int:
    return int(_lib.shgo_basis_launches(ctypes.c_void_p(basis)))


def shgo_nuclear_attraction_noalloc(n_shells, l, n_prim, exponents, coefs, shell_xyz, n_centers, centers_ptr,
                                    charges_ptr, out_ptr, stream=None):
    """Allocation-free call (host basis arrays, device nuclei/charges/output as int pointers).

    For callers that may not allocate device memory: it uses only the library's static device
    scratch array (see include/shgo.h).  Calls that overlap on the GPU race on that array."""
    l = np.ascontiguousarray(l, dtype=np.int32)
    n_prim = np.ascontiguousarray(n_prim, dtype=np.int32)
    exponents = np.ascontiguousarray(exponents, dtype=np.float64)
    coefs = np.ascontiguousarray(coefs, dtype=np.float64)
    shell_xyz = np.ascontiguousarray(shell_xyz, dtype=np.float64).reshape(-1)
    c = shgo_centers(int(n_centers), ctypes.c_void_p(int(centers_ptr) if centers_ptr else 0))
    _check(_lib.shgo_nuclear_attraction_noalloc(
        int(n_shells), _ptr(l, ctypes.c_int32), _ptr(n_prim, ctypes.c_int32), _ptr(exponents, ctypes.c_double),
        _ptr(coefs, ctypes.c_double), _ptr(shell_xyz, ctypes.c_double), ctypes.byref(c),
        ctypes.c_void_p(int(charges_ptr) if charges_ptr else 0), ctypes.c_void_p(int(out_ptr) if out_ptr else 0),
        _stream_handle(stream)))


def shgo_free(basis) -> None:
    _lib.shgo_free(ctypes.c_void_p(basis))


def shgo_basis_nbf(basis) -> int:
    return int(_lib.shgo_basis_nbf(ctypes.c_void_p(basis)))


def shgo_basis_npairs(basis) -> int:
    return int(_lib.shgo_basis_npairs(ctypes.c_void_p(basis)))


# ------------------------------------------------------------------ convenience wrappers
def shgo_sparse_layout(basis):
    """(nblocks, ndoubles, offset[npairs]) of a block-sparse basis (offset -1 for an omitted pair)."""
    nb = ctypes.c_int64()
    nd = ctypes.c_int64()
    off = np.zeros(max(shgo_basis_npairs(basis), 0), dtype=np.int64)
    _check(_lib.shgo_sparse_layout(ctypes.c_void_p(basis), ctypes.byref(nb), ctypes.byref(nd),
                                   _ptr(off, ctypes.c_int64)))
    return int(nb.value), int(nd.value), off


class Basis:
    """Owns a shgo_basis handle built from a basis dict (see workloads.py)."""

    def __init__(self, basis: dict, precision: int = SHGO_PREC_FP64, device: int = -1, flags: int = 0,
                 shard=None):
        self.handle = shgo_basis_create(len(basis["l"]), basis["l"], basis["nprim"], basis["exps"], basis["coefs"],
                                        basis["xyz"], precision, device, flags, shard)
        self.nbf = shgo_basis_nbf(self.handle)
        self.npairs = shgo_basis_npairs(self.handle)
        self.n_shells = len(basis["l"])
        self.sparse = bool(flags & SHGO_FLAG_BLOCK_SPARSE)
        if self.sparse:
            self.nblocks, self.ndoubles, self.offset = shgo_sparse_layout(self.handle)

    def out_shape(self):
        """Shape of V's output array: (nbf, nbf), or (ndoubles,) for a block-sparse basis."""
        return (max(self.ndoubles, 1),) if self.sparse else (self.nbf, self.nbf)

    def close(self) -> None:
        if getattr(self, "handle", None):
            shgo_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nuclear_attraction(basis: Basis, centers, charges, out=None, stream=None):
    """V (nbf x nbf, FP64, device tensor).  centers [n, 3] and charges [n] are CUDA float64 tensors."""
    import torch
    if not (centers.is_cuda and charges.is_cuda):
        raise ValueError("centers and charges must be CUDA tensors")
    if centers.dtype != torch.float64 or charges.dtype != torch.float64:
        raise ValueError("centers and charges must be float64")
    centers = centers.contiguous()
    charges = charges.contiguous()
    if out is None:
        out = torch.empty(basis.out_shape(), dtype=torch.float64, device=centers.device)
    if not out.is_contiguous() or out.dtype != torch.float64 or tuple(out.shape) != basis.out_shape():
        raise ValueError(f"out must be a contiguous float64 {list(basis.out_shape())} tensor")
    n = centers.shape[0] if centers.numel() else 0
    shgo_nuclear_attraction(basis.handle, n, centers.data_ptr() if n else 0, charges.data_ptr() if n else 0,
                            out.data_ptr(), stream)
    return out


def shgo_basis_class_stats(basis, n_centers):
    """Per class: list of (la, lb, shell_triples, integrals, coupling_flops, pair_flops)."""
    rows = []
    for c in range(int(_lib.shgo_basis_nclasses(ctypes.c_void_p(basis)))):
        ll = np.zeros(2, dtype=np.int32)
        st = np.zeros(4)
        _check(_lib.shgo_basis_class_stats(ctypes.c_void_p(basis), int(n_centers), c, _ptr(ll, ctypes.c_int32),
                                           _ptr(st, ctypes.c_double)))
        rows.append((int(ll[0]), int(ll[1]), *map(float, st)))
    return rows


def shgo_nuclear_attraction_class_timed(basis, n_centers, centers_ptr, charges_ptr, out_ptr, stream=None):
    """Per class device times (ms) of the coupling and pair kernels, classes run one after another."""
    n = int(_lib.shgo_basis_nclasses(ctypes.c_void_p(basis)))
    ms = np.zeros(2 * max(n, 1))
    c = shgo_centers(int(n_centers), ctypes.c_void_p(int(centers_ptr) if centers_ptr else 0))
    _check(_lib.shgo_nuclear_attraction_class_timed(ctypes.c_void_p(basis), ctypes.byref(c),
                                                    ctypes.c_void_p(int(charges_ptr) if charges_ptr else 0),
                                                    ctypes.c_void_p(int(out_ptr) if out_ptr else 0),
                                                    _stream_handle(stream), _ptr(ms, ctypes.c_double)))
    return ms[:2 * n].reshape(n, 2)


def shgo_esp(basis, density_ptr, n_points, points_ptr, phi_ptr, stream=None):
    c = shgo_centers(int(n_points), ctypes.c_void_p(int(points_ptr) if points_ptr else 0))
    _check(_lib.shgo_esp(ctypes.c_void_p(basis), ctypes.c_void_p(int(density_ptr) or 0), ctypes.byref(c),
                         ctypes.c_void_p(int(phi_ptr) if phi_ptr else 0), _stream_handle(stream)))


def esp(basis, density, points, out=None, stream=None):
    """phi[k] = sum_ab D_ab <a|1/|r - points[k]||b> (FP64 device tensor [n]); density [nbf, nbf] and
    points [n, 3] are CUDA float64 tensors."""
    import torch
    density = density.contiguous()
    points = points.contiguous()
    if tuple(density.shape) != (basis.nbf, basis.nbf) or density.dtype != torch.float64:
        raise ValueError("density must be a float64 [nbf, nbf] tensor")
    n = points.shape[0] if points.numel() else 0
    if out is None:
        out = torch.empty(max(n, 1), dtype=torch.float64, device=points.device)
    shgo_esp(basis.handle, density.data_ptr(), n, points.data_ptr() if n else 0, out.data_ptr(), stream)
    return out[:n]


def shgo_esp_gradient(basis, density_ptr, n_points, points_ptr, grad_ptr, stream=None):
    c = shgo_centers(int(n_points), ctypes.c_void_p(int(points_ptr) if points_ptr else 0))
    _check(_lib.shgo_esp_gradient(ctypes.c_void_p(basis), ctypes.c_void_p(int(density_ptr) or 0), ctypes.byref(c),
                                  ctypes.c_void_p(int(grad_ptr) if grad_ptr else 0), _stream_handle(stream)))


def esp_gradient(basis, density, points, out=None, stream=None):
    """grad[k] = d phi_k / d points[k] (FP64 device tensor [n, 3])."""
    import torch
    density = density.contiguous()
    points = points.contiguous()
    if tuple(density.shape) != (basis.nbf, basis.nbf) or density.dtype != torch.float64:
        raise ValueError("density must be a float64 [nbf, nbf] tensor")
    n = points.shape[0] if points.numel() else 0
    if out is None:
        out = torch.empty((max(n, 1), 3), dtype=torch.float64, device=points.device)
    shgo_esp_gradient(basis.handle, density.data_ptr(), n, points.data_ptr() if n else 0, out.data_ptr(), stream)
    return out[:n]


def shgo_nuclear_attraction_deriv(basis, n_centers, centers_ptr, charges_ptr, out_ptr, stream=None):
    c = shgo_centers(int(n_centers), ctypes.c_void_p(int(centers_ptr) if centers_ptr else 0))
    _check(_lib.shgo_nuclear_attraction_deriv(ctypes.c_void_p(basis), ctypes.byref(c),
                                              ctypes.c_void_p(int(charges_ptr) if charges_ptr else 0),
                                              ctypes.c_void_p(int(out_ptr) if out_ptr else 0), _stream_handle(stream)))


def shgo_nuclear_field(basis, n_centers, centers_ptr, charges_ptr, out_ptr, stream=None):
    c = shgo_centers(int(n_centers), ctypes.c_void_p(int(centers_ptr) if centers_ptr else 0))
    _check(_lib.shgo_nuclear_field(ctypes.c_void_p(basis), ctypes.byref(c),
                                   ctypes.c_void_p(int(charges_ptr) if charges_ptr else 0),
                                   ctypes.c_void_p(int(out_ptr) if out_ptr else 0), _stream_handle(stream)))


def _deriv_args(basis, centers, charges, out):
    import torch
    if not (centers.is_cuda and charges.is_cuda):
        raise ValueError("centers and charges must be CUDA tensors")
    if centers.dtype != torch.float64 or charges.dtype != torch.float64:
        raise ValueError("centers and charges must be float64")
    centers = centers.contiguous()
    charges = charges.contiguous()
    shape = (3, basis.nbf, basis.nbf)
    if out is None:
        out = torch.empty(shape, dtype=torch.float64, device=centers.device)
    if not out.is_contiguous() or out.dtype != torch.float64 or tuple(out.shape) != shape:
        raise ValueError(f"out must be a contiguous float64 {list(shape)} tensor")
    n = centers.shape[0] if centers.numel() else 0
    return centers, charges, out, n


def nuclear_attraction_deriv(basis: Basis, centers, charges, out=None, stream=None):
    """dV/d(bra centre): [3, nbf, nbf] FP64 device tensor, out[X][a][b] = d V_ab / d A_X with A the centre of
    a's shell (b's held fixed); the derivative by b's centre is out[X][b][a]."""
    centers, charges, out, n = _deriv_args(basis, centers, charges, out)
    shgo_nuclear_attraction_deriv(basis.handle, n, centers.data_ptr() if n else 0, charges.data_ptr() if n else 0,
                                  out.data_ptr(), stream)
    return out


def nuclear_field(basis: Basis, centers, charges, out=None, stream=None):
    """Field integrals sum_C Z_C dV/dC_X: [3, nbf, nbf] FP64 device tensor (symmetric in a, b)."""
    centers, charges, out, n = _deriv_args(basis, centers, charges, out)
    shgo_nuclear_field(basis.handle, n, centers.data_ptr() if n else 0, charges.data_ptr() if n else 0,
                       out.data_ptr(), stream)
    return out


def shgo_nuclear_attraction_gradient(basis, density_ptr, n_centers, centers_ptr, charges_ptr, grad_ptr, stream=None):
    c = shgo_centers(int(n_centers), ctypes.c_void_p(int(centers_ptr) if centers_ptr else 0))
    _check(_lib.shgo_nuclear_attraction_gradient(ctypes.c_void_p(basis), ctypes.c_void_p(int(density_ptr) or 0),
                                                 ctypes.byref(c),
                                                 ctypes.c_void_p(int(charges_ptr) if charges_ptr else 0),
                                                 ctypes.c_void_p(int(grad_ptr) if grad_ptr else 0),
                                                 _stream_handle(stream)))


def nuclear_attraction_gradient(basis: Basis, density, centers, charges, out=None, stream=None):
    """grad[s][X] = sum_{a in s} sum_b (P_ab + P_ba) dV_ab/dA_X (A the centre of shell s): [n_shells, 3] FP64
    device tensor; density [nbf, nbf], centers [n, 3], charges [n] are CUDA float64 tensors."""
    import torch
    if not (centers.is_cuda and charges.is_cuda):
        raise ValueError("centers and charges must be CUDA tensors")
    if centers.dtype != torch.float64 or charges.dtype != torch.float64:
        raise ValueError("centers and charges must be float64")
    centers = centers.contiguous()
    charges = charges.contiguous()
    n = centers.shape[0] if centers.numel() else 0
    density = density.contiguous()
    if tuple(density.shape) != (basis.nbf, basis.nbf) or density.dtype != torch.float64 or not density.is_cuda:
        raise ValueError("density must be a CUDA float64 [nbf, nbf] tensor")
    ns = basis.n_shells
    if out is None:
        out = torch.empty((max(ns, 1), 3), dtype=torch.float64, device=centers.device)
    shgo_nuclear_attraction_gradient(basis.handle, density.data_ptr(), n, centers.data_ptr() if n else 0,
                                     charges.data_ptr() if n else 0, out.data_ptr(), stream)
    return out[:ns]


def field_matrices(basis: Basis, centers, stream=None):
    """Per-nucleus field-integral matrices: [n, 3, nbf, nbf], entry C = d/dC_X <a|1/|r - C||b> (unit charge),
    one shgo_nuclear_field call per nucleus."""
    import torch
    centers = centers.contiguous()
    n = centers.shape[0] if centers.numel() else 0
    out = torch.empty((n, 3, basis.nbf, basis.nbf), dtype=torch.float64, device=centers.device)
    one = torch.ones(1, dtype=torch.float64, device=centers.device)
    for k in range(n):
        nuclear_field(basis, centers[k:k + 1], one, out=out[k], stream=stream)
    return out


def host_deriv_transform(lam: int, comp: int, p: float, r1):
    """The derivative steps on one coupling block of order lam + 1 (host copy of the device tables): returns
    (raised, field) in the layout of order lam, raised = the block of x_c times the one-centre integrand,
    field = the block of d_c of it (exponent p)."""
    r1 = np.ascontiguousarray(r1, dtype=np.float64)
    n = (lam + 1) * (lam + 2) * (lam + 3) // 6
    raised = np.zeros(n)
    field = np.zeros(n)
    _check(_lib.shgo_host_deriv_transform(int(lam), int(comp), float(p), _ptr(r1, ctypes.c_double),
                                          _ptr(raised, ctypes.c_double), _ptr(field, ctypes.c_double)))
    return raised, field


def host_deriv_lowering(l: int, comp: int, m: int) -> np.ndarray:
    """Coefficients of d_c S_lm = sum_M' w[M' + l - 1] S_{l-1,M'} (host copy of the device table)."""
    w = np.zeros(max(2 * l - 1, 1))
    _check(_lib.shgo_host_deriv_lowering(int(l), int(comp), int(m), _ptr(w, ctypes.c_double)))
    return w[:2 * l - 1]


def shgo_overlap(basis, out_ptr, stream=None):
    _check(_lib.shgo_overlap(ctypes.c_void_p(basis), ctypes.c_void_p(int(out_ptr) or 0), _stream_handle(stream)))


def overlap(basis, out=None, stream=None, device="cuda"):
    """S (FP64 device tensor): [nbf, nbf] for a Basis, the concatenated per-molecule blocks for a
    Batch (see Batch.block)."""
    import torch
    if isinstance(basis, Basis):
        shape = (basis.nbf, basis.nbf)
    else:
        shape = (max(basis.out_size, 1),)
    if out is None:
        out = torch.empty(shape, dtype=torch.float64, device=device)
    if not out.is_contiguous() or out.dtype != torch.float64 or tuple(out.shape) != shape:
        raise ValueError(f"out must be a contiguous float64 {list(shape)} tensor")
    shgo_overlap(basis.handle, out.data_ptr(), stream)
    return out


def shgo_coulomb_2c(basis, out_ptr, stream=None):
    _check(_lib.shgo_coulomb_2c(ctypes.c_void_p(basis), ctypes.c_void_p(int(out_ptr) or 0), _stream_handle(stream)))


def coulomb_2c(basis, out=None, stream=None, device="cuda"):
    """Two-centre Coulomb integrals (a|b) (FP64 device tensor), laid out as overlap()."""
    import torch
    if isinstance(basis, Basis):
        shape = (basis.nbf, basis.nbf)
    else:
        shape = (max(basis.out_size, 1),)
    if out is None:
        out = torch.empty(shape, dtype=torch.float64, device=device)
    if not out.is_contiguous() or out.dtype != torch.float64 or tuple(out.shape) != shape:
        raise ValueError(f"out must be a contiguous float64 {list(shape)} tensor")
    shgo_coulomb_2c(basis.handle, out.data_ptr(), stream)
    return out


def shgo_eri(basis, out_ptr, stream=None):
    _check(_lib.shgo_eri(ctypes.c_void_p(basis), ctypes.c_void_p(int(out_ptr) or 0), _stream_handle(stream)))


def eri(basis, out=None, stream=None, device="cuda"):
    """Four-centre electron-repulsion integrals (ij|kl) of a basis (FP64 device tensor nbf^4)."""
    import torch
    if not isinstance(basis, Basis):
        raise ValueError("eri takes a Basis, not a Batch")
    shape = (basis.nbf,) * 4
    if out is None:
        out = torch.empty(shape, dtype=torch.float64, device=device)
    if not out.is_contiguous() or out.dtype != torch.float64 or tuple(out.shape) != shape:
        raise ValueError(f"out must be a contiguous float64 {list(shape)} tensor")
    shgo_eri(basis.handle, out.data_ptr(), stream)
    return out


def shgo_eri_jk(basis, dens_ptr, j_ptr, k_ptr, stream=None):
    _check(_lib.shgo_eri_jk(ctypes.c_void_p(basis), ctypes.c_void_p(int(dens_ptr) or 0),
                            ctypes.c_void_p(int(j_ptr) or 0), ctypes.c_void_p(int(k_ptr) or 0), _stream_handle(stream)))


def eri_jk(basis, density, coulomb=True, exchange=True, stream=None):
    """Coulomb J[p,q] = sum_rs (pq|rs) D[r,s] and exchange K[p,r] = sum_qs (pq|rs) D[q,s] of a device density
    (FP64 nbf x nbf); returns (J, K), None for the one not asked for."""
    import torch
    if not isinstance(basis, Basis):
        raise ValueError("eri_jk takes a Basis, not a Batch")
    n = basis.nbf
    if not density.is_contiguous() or density.dtype != torch.float64 or tuple(density.shape) != (n, n):
        raise ValueError(f"density must be a contiguous float64 [{n}, {n}] tensor")
    J = torch.empty((n, n), dtype=torch.float64, device=density.device) if coulomb else None
    K = torch.empty((n, n), dtype=torch.float64, device=density.device) if exchange else None
    shgo_eri_jk(basis.handle, density.data_ptr(), J.data_ptr() if J is not None else 0,
                K.data_ptr() if K is not None else 0, stream)
    return J, K


def host_solid_harmonics(l: int, xyz) -> np.ndarray:
    pts = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((pts.shape[0], 2 * l + 1))
    _check(_lib.shgo_host_solid_harmonics(int(l), pts.shape[0], _ptr(pts, ctypes.c_double), _ptr(out, ctypes.c_double)))
    return out


def host_gaunt(l1, m1, l2, m2, L, M) -> float:
    return float(_lib.shgo_host_gaunt(l1, m1, l2, m2, L, M))


def host_translation(la, ma, l1, m1, nu) -> float:
    return float(_lib.shgo_host_translation(la, ma, l1, m1, nu))


def host_laplacian_coef(L: int, k: int, j: int) -> float:
    return float(_lib.shgo_host_laplacian_coef(L, k, j))


def host_eri_eps(L: int, k: int, n: int) -> float:
    return float(_lib.shgo_host_eri_eps(L, k, n))


def host_boys(nmax: int, T: float) -> np.ndarray:
    F = np.zeros(nmax + 1)
    _check(_lib.shgo_host_boys(int(nmax), float(T), _ptr(F, ctypes.c_double)))
    return F


# ------------------------------------------------------------------ batches of molecules
class Batch:
    """Owns a batch handle (shgo_batch_create) over a list of (basis dict, n_nuclei)."""

    def __init__(self, molecules, precision: int = SHGO_PREC_FP64, device: int = -1):
        mol_nshells = np.array([len(b["l"]) for b, _ in molecules], dtype=np.int32)
        mol_ncent = np.array([int(n) for _, n in molecules], dtype=np.int64)
        l = np.ascontiguousarray(np.concatenate([b["l"] for b, _ in molecules]), dtype=np.int32)
        nprim = np.ascontiguousarray(np.concatenate([b["nprim"] for b, _ in molecules]), dtype=np.int32)
        exps = np.ascontiguousarray(np.concatenate([b["exps"] for b, _ in molecules]), dtype=np.float64)
        coefs = np.ascontiguousarray(np.concatenate([b["coefs"] for b, _ in molecules]), dtype=np.float64)
        xyz = np.ascontiguousarray(np.concatenate([b["xyz"] for b, _ in molecules]), dtype=np.float64).reshape(-1)
        opt = shgo_options(int(precision), int(device), 0)
        handle = ctypes.c_void_p()
        _check(_lib.shgo_batch_create(len(molecules), _ptr(mol_nshells, ctypes.c_int32), _ptr(mol_ncent, ctypes.c_int64),
                                      len(l), _ptr(l, ctypes.c_int32), _ptr(nprim, ctypes.c_int32),
                                      _ptr(exps, ctypes.c_double), _ptr(coefs, ctypes.c_double),
                                      _ptr(xyz, ctypes.c_double), ctypes.byref(opt), ctypes.byref(handle)))
        self.handle = handle.value
        self.n_mol = len(molecules)
        self.mol_nbf = np.zeros(self.n_mol, dtype=np.int64)
        self.mol_off = np.zeros(self.n_mol, dtype=np.int64)
        _check(_lib.shgo_batch_layout(ctypes.c_void_p(self.handle), _ptr(self.mol_nbf, ctypes.c_int64),
                                      _ptr(self.mol_off, ctypes.c_int64)))
        self.out_size = int(_lib.shgo_batch_out_size(ctypes.c_void_p(self.handle)))
        self.n_centers = int(mol_ncent.sum())

    def block(self, out, m):
        """V of molecule m as an (nbf_m, nbf_m) view of the batched output."""
        n = int(self.mol_nbf[m])
        o = int(self.mol_off[m])
        return out[o:o + n * n].reshape(n, n)

    def close(self) -> None:
        if getattr(self, "handle", None):
            shgo_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def shgo_nuclear_attraction_batched(batch, centers_ptr, charges_ptr, out_ptr, stream=None):
    _check(_lib.shgo_nuclear_attraction_batched(ctypes.c_void_p(batch), ctypes.c_void_p(int(centers_ptr) or 0),
                                                ctypes.c_void_p(int(charges_ptr) or 0),
                                                ctypes.c_void_p(int(out_ptr) or 0), _stream_handle(stream)))


def nuclear_attraction_batched(batch: Batch, centers, charges, out=None, stream=None):
    """All molecules' V blocks, concatenated (see Batch.block).  centers [sum n, 3], charges [sum n]
    are CUDA float64 tensors in molecule order."""
    import torch
    centers = centers.contiguous()
    charges = charges.contiguous()
    if out is None:
        out = torch.empty(max(batch.out_size, 1), dtype=torch.float64, device=centers.device)
    shgo_nuclear_attraction_batched(batch.handle, centers.data_ptr() if centers.numel() else 0,
                                    charges.data_ptr() if charges.numel() else 0, out.data_ptr(), stream)
    return out


# ------------------------------------------------------------------ learned screening (shgo_mlp.h)
MLP_IN, MLP_HIDDEN = 16, 64
MLP_NPARAM = 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1


def _bind_mlp():
    f32p = ctypes.POINTER(ctypes.c_float)
    vp = ctypes.c_void_p
    L = _lib
    L.shgo_mlp_create.argtypes = [f32p, f32p, f32p, ctypes.POINTER(vp)]
    L.shgo_mlp_create.restype = ctypes.c_int
    L.shgo_mlp_free.argtypes = [vp]
    L.shgo_mlp_free.restype = None
    L.shgo_mlp_get_params.argtypes = [vp, f32p]
    L.shgo_mlp_get_params.restype = ctypes.c_int
    L.shgo_mlp_get_state.argtypes = [vp, f32p, f32p, f32p, ctypes.POINTER(ctypes.c_int64)]
    L.shgo_mlp_get_state.restype = ctypes.c_int
    L.shgo_mlp_set_state.argtypes = [vp, f32p, f32p, f32p, ctypes.c_int64]
    L.shgo_mlp_set_state.restype = ctypes.c_int
    L.shgo_mlp_forward.argtypes = [vp, vp, ctypes.c_int64, vp, vp]
    L.shgo_mlp_forward.restype = ctypes.c_int
    L.shgo_mlp_gradients.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.c_float, f32p, f32p]
    L.shgo_mlp_gradients.restype = ctypes.c_int
    L.shgo_mlp_train_step.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.c_float, ctypes.c_float, f32p, vp]
    L.shgo_mlp_train_step.restype = ctypes.c_int
    L.shgo_screen_features.argtypes = [vp, vp, vp, vp, ctypes.c_int64, vp, vp]
    L.shgo_screen_features.restype = ctypes.c_int
    L.shgo_pair_shells.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    L.shgo_pair_shells.restype = ctypes.c_int
    L.shgo_screen_build.argtypes = [vp, vp, vp, vp, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                    ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    L.shgo_screen_build.restype = ctypes.c_int
    L.shgo_screen_mask.argtypes = [vp, ctypes.POINTER(ctypes.c_uint8)]
    L.shgo_screen_mask.restype = ctypes.c_int
    L.shgo_nuclear_attraction_screened.argtypes = [vp, vp, vp, ctypes.c_int64, vp, vp]
    L.shgo_nuclear_attraction_screened.restype = ctypes.c_int


_bind_mlp()


class MLP:
    """The screening network on the current device (FP32 master weights, BF16 forward)."""

    def __init__(self, params, feature_mean, feature_sd):
        p = np.ascontiguousarray(params, dtype=np.float32)
        mu = np.ascontiguousarray(feature_mean, dtype=np.float32)
        sd = np.ascontiguousarray(feature_sd, dtype=np.float32)
        assert p.size == MLP_NPARAM and mu.size == MLP_IN and sd.size == MLP_IN
        h = ctypes.c_void_p()
        _check(_lib.shgo_mlp_create(_ptr(p, ctypes.c_float), _ptr(mu, ctypes.c_float), _ptr(sd, ctypes.c_float),
                                    ctypes.byref(h)))
        self.handle = h.value
        self.mean = mu
        self.sd = sd

    def state(self) -> dict:
        """Checkpoint: FP32 parameters, Adam moments and step count (host copies)."""
        p = np.zeros(MLP_NPARAM, dtype=np.float32)
        m = np.zeros(MLP_NPARAM, dtype=np.float32)
        v = np.zeros(MLP_NPARAM, dtype=np.float32)
        step = ctypes.c_int64()
        _check(_lib.shgo_mlp_get_state(ctypes.c_void_p(self.handle), _ptr(p, ctypes.c_float), _ptr(m, ctypes.c_float),
                                       _ptr(v, ctypes.c_float), ctypes.byref(step)))
        return {"params": p, "adam_m": m, "adam_v": v, "step": int(step.value)}

    def load_state(self, st: dict) -> None:
        p = np.ascontiguousarray(st["params"], dtype=np.float32)
        m = np.ascontiguousarray(st["adam_m"], dtype=np.float32)
        v = np.ascontiguousarray(st["adam_v"], dtype=np.float32)
        _check(_lib.shgo_mlp_set_state(ctypes.c_void_p(self.handle), _ptr(p, ctypes.c_float), _ptr(m, ctypes.c_float),
                                       _ptr(v, ctypes.c_float), int(st["step"])))

    def params(self) -> np.ndarray:
        p = np.zeros(MLP_NPARAM, dtype=np.float32)
        _check(_lib.shgo_mlp_get_params(ctypes.c_void_p(self.handle), _ptr(p, ctypes.c_float)))
        return p

    def forward(self, X, y=None, stream=None):
        import torch
        if y is None:
            y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        _check(_lib.shgo_mlp_forward(ctypes.c_void_p(self.handle), ctypes.c_void_p(X.data_ptr()), X.shape[0],
                                     ctypes.c_void_p(y.data_ptr()), _stream_handle(stream)))
        return y

    def gradients(self, X, T, under_weight=1.0):
        g = np.zeros(MLP_NPARAM, dtype=np.float32)
        loss = ctypes.c_float()
        _check(_lib.shgo_mlp_gradients(ctypes.c_void_p(self.handle), ctypes.c_void_p(X.data_ptr()),
                                       ctypes.c_void_p(T.data_ptr()), X.shape[0], float(under_weight),
                                       _ptr(g, ctypes.c_float), ctypes.byref(loss)))
        return g, float(loss.value)

    def train_step(self, X, T, under_weight, lr, want_loss=False, stream=None):
        loss = ctypes.c_float()
        _check(_lib.shgo_mlp_train_step(ctypes.c_void_p(self.handle), ctypes.c_void_p(X.data_ptr()),
                                        ctypes.c_void_p(T.data_ptr()), X.shape[0], float(under_weight), float(lr),
                                        ctypes.byref(loss) if want_loss else None, _stream_handle(stream)))
        return float(loss.value) if want_loss else None

    def close(self):
        if getattr(self, "handle", None):
            _lib.shgo_mlp_free(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pair_shells(handle, npairs):
    a = np.zeros(npairs, dtype=np.int32)
    b = np.zeros(npairs, dtype=np.int32)
    _check(_lib.shgo_pair_shells(ctypes.c_void_p(handle), _ptr(a, ctypes.c_int32), _ptr(b, ctypes.c_int32)))
    return a, b


def screen_features(handle, centers, charges, triples, stream=None):
    """Features [n, 16] (float32, device) of triples [n, 2] (int32 device: pair index, nucleus index)."""
    import torch
    n = triples.shape[0]
    X = torch.empty((n, MLP_IN), dtype=torch.float32, device=triples.device)
    _check(_lib.shgo_screen_features(ctypes.c_void_p(handle), ctypes.c_void_p(centers.data_ptr()),
                                     ctypes.c_void_p(charges.data_ptr()), ctypes.c_void_p(triples.data_ptr()), n,
                                     ctypes.c_void_p(X.data_ptr()), _stream_handle(stream)))
    return X


def screen_build(handle, mlp: MLP, centers, charges, n_centers, log10_threshold, log10_margin):
    kept = ctypes.c_int64()
    skipped = ctypes.c_int64()
    _check(_lib.shgo_screen_build(ctypes.c_void_p(handle), ctypes.c_void_p(mlp.handle),
                                  ctypes.c_void_p(centers.data_ptr() if centers.numel() else 0),
                                  ctypes.c_void_p(charges.data_ptr() if charges.numel() else 0), int(n_centers),
                                  float(log10_threshold), float(log10_margin), ctypes.byref(kept),
                                  ctypes.byref(skipped)))
    return int(kept.value), int(skipped.value)


def screen_mask(handle, n_triples) -> np.ndarray:
    m = np.zeros(max(n_triples, 1), dtype=np.uint8)
    _check(_lib.shgo_screen_mask(ctypes.c_void_p(handle), _ptr(m, ctypes.c_uint8)))
    return m[:n_triples]


def nuclear_attraction_screened(handle, centers, charges, n_centers, out, stream=None):
    _check(_lib.shgo_nuclear_attraction_screened(ctypes.c_void_p(handle),
                                                 ctypes.c_void_p(centers.data_ptr() if centers.numel() else 0),
                                                 ctypes.c_void_p(charges.data_ptr() if charges.numel() else 0),
                                                 int(n_centers), ctypes.c_void_p(out.data_ptr()),
                                                 _stream_handle(stream)))
    return out


def _batch_from_arrays(cls, mols: dict, mol_ncenters, precision: int = SHGO_PREC_FP64, device: int = -1):
    """A batch from concatenated arrays: mols["nshells"][m] shells per molecule and the shell
    arrays l, nprim, exps, coefs, xyz of all molecules back to back."""
    self = cls.__new__(cls)
    mol_nshells = np.ascontiguousarray(mols["nshells"], dtype=np.int32)
    mol_ncent = np.ascontiguousarray(mol_ncenters, dtype=np.int64)
    l = np.ascontiguousarray(mols["l"], dtype=np.int32)
    nprim = np.ascontiguousarray(mols["nprim"], dtype=np.int32)
    exps = np.ascontiguousarray(mols["exps"], dtype=np.float64)
    coefs = np.ascontiguousarray(mols["coefs"], dtype=np.float64)
    xyz = np.ascontiguousarray(mols["xyz"], dtype=np.float64).reshape(-1)
    opt = shgo_options(int(precision), int(device))
    handle = ctypes.c_void_p()
    _check(_lib.shgo_batch_create(len(mol_nshells), _ptr(mol_nshells, ctypes.c_int32),
                                  _ptr(mol_ncent, ctypes.c_int64), len(l), _ptr(l, ctypes.c_int32),
                                  _ptr(nprim, ctypes.c_int32), _ptr(exps, ctypes.c_double),
                                  _ptr(coefs, ctypes.c_double), _ptr(xyz, ctypes.c_double), ctypes.byref(opt),
                                  ctypes.byref(handle)))
    self.handle = handle.value
    self.n_mol = len(mol_nshells)
    self.mol_nbf = np.zeros(self.n_mol, dtype=np.int64)
    self.mol_off = np.zeros(self.n_mol, dtype=np.int64)
    _check(_lib.shgo_batch_layout(ctypes.c_void_p(self.handle), _ptr(self.mol_nbf, ctypes.c_int64),
                                  _ptr(self.mol_off, ctypes.c_int64)))
    self.out_size = int(_lib.shgo_batch_out_size(ctypes.c_void_p(self.handle)))
    self.n_centers = int(mol_ncent.sum())
    return self


Batch.from_arrays = classmethod(_batch_from_arrays)
