"""Plain CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use this
package.  The library never imports it, and it imports nothing from the library.

The arithmetic lives in ``shgo_oracle.c``: the plain definition
``V_ab = sum_C Z_C <phi_a|1/|r-C||phi_b>`` over the contracted solid-harmonic Gaussian
orbitals of Eq. 1, evaluated by the Cartesian McMurchie-Davidson route (the paper's comparison
route, Table 1 first column) followed by a Cartesian -> real solid-harmonic transform.  This
module only builds that C file with gcc and marshals arrays through ctypes.

Two builds exist: ``f64`` (double) and ``ld`` (long double: 80-bit on x86-64, IEEE binary128
on aarch64), used to certify the double oracle at high angular momentum.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "shgo_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIBS: dict[str, ctypes.CDLL] = {}
_LOCK = threading.Lock()

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def _lib_path(precision: str) -> str:
    return os.path.join(_BUILD, f"libshgo_oracle_{precision}.so")


def build(force: bool = False) -> None:
    """Compile both oracle builds with gcc (OpenMP over shell pairs)."""
    os.makedirs(_BUILD, exist_ok=True)
    for precision, extra in (("f64", []), ("ld", ["-DORACLE_LONG_DOUBLE"])):
        out = _lib_path(precision)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", *extra, "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)


def _lib(precision: str = "f64") -> ctypes.CDLL:
    with _LOCK:
        if precision in _LIBS:
            return _LIBS[precision]
        build()
        lib = ctypes.CDLL(_lib_path(precision))
        lib.oracle_boys.argtypes = [ctypes.c_int, ctypes.c_double, _f64p]
        lib.oracle_boys.restype = None
        lib.oracle_solid_harmonic_cart.argtypes = [ctypes.c_int, _f64p]
        lib.oracle_solid_harmonic_cart.restype = ctypes.c_int
        lib.oracle_solid_harmonic.argtypes = [ctypes.c_int, ctypes.c_long, _f64p, _f64p]
        lib.oracle_solid_harmonic.restype = ctypes.c_int
        lib.oracle_nuclear_attraction.argtypes = [
            ctypes.c_int, _i32p, _i32p, _f64p, _f64p, _f64p, ctypes.c_long, _f64p, _f64p, _f64p, ctypes.c_int]
        lib.oracle_nuclear_attraction.restype = ctypes.c_int
        lib.oracle_nuclear_field.argtypes = [
            ctypes.c_int, _i32p, _i32p, _f64p, _f64p, _f64p, ctypes.c_long, _f64p, _f64p, ctypes.c_int, _f64p,
            ctypes.c_int]
        lib.oracle_nuclear_field.restype = ctypes.c_int
        lib.oracle_nuclear_deriv.argtypes = [
            ctypes.c_int, _i32p, _i32p, _f64p, _f64p, _f64p, ctypes.c_long, _f64p, _f64p, ctypes.c_int, _f64p,
            ctypes.c_int]
        lib.oracle_nuclear_deriv.restype = ctypes.c_int
        lib.oracle_overlap.argtypes = [ctypes.c_int, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, ctypes.c_int]
        lib.oracle_coulomb_2c.argtypes = [ctypes.c_int, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, ctypes.c_int]
        lib.oracle_overlap.restype = ctypes.c_int
        lib.oracle_eri.argtypes = [ctypes.c_int, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, ctypes.c_int]
        lib.oracle_eri.restype = ctypes.c_int
        lib.oracle_prim_norm.argtypes = [ctypes.c_int, ctypes.c_double]
        lib.oracle_prim_norm.restype = ctypes.c_double
        lib.oracle_real_bits.argtypes = []
        lib.oracle_real_bits.restype = ctypes.c_int
        _LIBS[precision] = lib
        return lib


def _basis_arrays(basis):
    l = np.ascontiguousarray(basis["l"], dtype=np.int32)
    nprim = np.ascontiguousarray(basis["nprim"], dtype=np.int32)
    exps = np.ascontiguousarray(basis["exps"], dtype=np.float64)
    coefs = np.ascontiguousarray(basis["coefs"], dtype=np.float64)
    xyz = np.ascontiguousarray(basis["xyz"], dtype=np.float64).reshape(-1)
    return l, nprim, exps, coefs, xyz


def nbf(basis) -> int:
    return int(np.sum(2 * np.asarray(basis["l"]) + 1))


def nuclear_attraction(basis, centers, charges, threads: int = 1, precision: str = "f64") -> np.ndarray:
    """V_ab = sum_C Z_C <phi_a|1/|r-C||phi_b> (no minus sign), nbf x nbf."""
    l, nprim, exps, coefs, xyz = _basis_arrays(basis)
    C = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1)
    Z = np.ascontiguousarray(charges, dtype=np.float64).reshape(-1)
    n = nbf(basis)
    out = np.zeros(max(n * n, 1), dtype=np.float64)
    rc = _lib(precision).oracle_nuclear_attraction(len(l), l, nprim, exps, coefs, xyz, len(Z),
                                                   C if C.size else np.zeros(3), Z if Z.size else np.zeros(1),
                                                   out, threads)
    if rc != 0:
        raise ValueError(f"oracle rejected the basis (code {rc})")
    return out[: n * n].reshape(n, n)


def nuclear_field(basis, centers, charges, threads: int = 1, precision: str = "f64") -> np.ndarray:
    """dV/dC: [3, nbf, nbf], component c = sum_C Z_C d/dC_c <phi_a|1/|r-C||phi_b> (McMurchie-Davidson:
    d/dC_x R_tuv(P - C) = -R_{t+1,u,v})."""
    l, nprim, exps, coefs, xyz = _basis_arrays(basis)
    C = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1)
    Z = np.ascontiguousarray(charges, dtype=np.float64).reshape(-1)
    n = nbf(basis)
    res = np.zeros((3, n, n))
    for c in range(3):
        out = np.zeros(max(n * n, 1), dtype=np.float64)
        rc = _lib(precision).oracle_nuclear_field(len(l), l, nprim, exps, coefs, xyz, len(Z),
                                                  C if C.size else np.zeros(3), Z if Z.size else np.zeros(1), c,
                                                  out, threads)
        if rc != 0:
            raise ValueError(f"oracle rejected the basis (code {rc})")
        res[c] = out[: n * n].reshape(n, n)
    return res


def nuclear_deriv(basis, centers, charges, threads: int = 1, precision: str = "f64") -> np.ndarray:
    """d V / d (bra centre): [3, nbf, nbf], out[c][a][b] = d/dA_c sum_C Z_C <phi_a|1/|r-C||phi_b>, A the centre
    of a's shell (b's held fixed); the derivative with respect to b's centre is out[c][b][a].  Cartesian
    route: d/dA_x of x_A^i exp(-alpha r_A^2) = 2 alpha x_A^{i+1} exp(...) - i x_A^{i-1} exp(...)."""
    l, nprim, exps, coefs, xyz = _basis_arrays(basis)
    C = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1)
    Z = np.ascontiguousarray(charges, dtype=np.float64).reshape(-1)
    n = nbf(basis)
    res = np.zeros((3, n, n))
    for c in range(3):
        out = np.zeros(max(n * n, 1), dtype=np.float64)
        rc = _lib(precision).oracle_nuclear_deriv(len(l), l, nprim, exps, coefs, xyz, len(Z),
                                                  C if C.size else np.zeros(3), Z if Z.size else np.zeros(1), c,
                                                  out, threads)
        if rc != 0:
            raise ValueError(f"oracle rejected the basis (code {rc})")
        res[c] = out[: n * n].reshape(n, n)
    return res


def overlap(basis, threads: int = 1, precision: str = "f64") -> np.ndarray:
    """S_ab = <phi_a|phi_b> (Eq. 4 with real solid harmonics), nbf x nbf."""
    l, nprim, exps, coefs, xyz = _basis_arrays(basis)
    n = nbf(basis)
    out = np.zeros(max(n * n, 1), dtype=np.float64)
    rc = _lib(precision).oracle_overlap(len(l), l, nprim, exps, coefs, xyz, out, threads)
    if rc != 0:
        raise ValueError(f"oracle rejected the basis (code {rc})")
    return out[: n * n].reshape(n, n)


def coulomb_2c(basis, threads: int = 1, precision: str = "f64") -> np.ndarray:
    """(a|b) = int int phi_a(r1) phi_b(r2) / |r1 - r2| (two-centre electron repulsion), nbf x nbf."""
    l, nprim, exps, coefs, xyz = _basis_arrays(basis)
    n = nbf(basis)
    out = np.zeros(max(n * n, 1), dtype=np.float64)
    rc = _lib(precision).oracle_coulomb_2c(len(l), l, nprim, exps, coefs, xyz, out, threads)
    if rc != 0:
        raise ValueError(f"oracle rejected the basis (code {rc})")
    return out[: n * n].reshape(n, n)


def eri(basis, threads: int = 1, precision: str = "f64") -> np.ndarray:
    """(ij|kl) = int int phi_i(r1) phi_j(r1) phi_k(r2) phi_l(r2) / |r1 - r2| (four-centre electron
    repulsion, Eqs. 13-15), nbf x nbf x nbf x nbf."""
    l, nprim, exps, coefs, xyz = _basis_arrays(basis)
    n = nbf(basis)
    out = np.zeros(max(n ** 4, 1), dtype=np.float64)
    rc = _lib(precision).oracle_eri(len(l), l, nprim, exps, coefs, xyz, out, threads)
    if rc != 0:
        raise ValueError(f"oracle rejected the basis (code {rc})")
    return out[: n ** 4].reshape(n, n, n, n)


def boys(nmax: int, T: float, precision: str = "f64") -> np.ndarray:
    """F_n(T) for n = 0..nmax."""
    F = np.zeros(nmax + 1, dtype=np.float64)
    _lib(precision).oracle_boys(int(nmax), float(T), F)
    return F


def solid_harmonic(l: int, xyz) -> np.ndarray:
    """Real Racah-normalised solid harmonics S_lm(r), m = -l..l, at each row of xyz (n x 3)."""
    pts = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((pts.shape[0], 2 * l + 1), dtype=np.float64)
    if _lib().oracle_solid_harmonic(int(l), pts.shape[0], pts.reshape(-1), out.reshape(-1)) != 0:
        raise ValueError("l out of range")
    return out


def prim_norm(l: int, alpha: float) -> float:
    return float(_lib().oracle_prim_norm(int(l), float(alpha)))


def real_bits(precision: str = "f64") -> int:
    return int(_lib(precision).oracle_real_bits())
