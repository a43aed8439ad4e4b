"""CPU checks of the library's host side (no GPU): the C ABI exports, the real solid-harmonic
recursion, the coupling (Gaunt) and translation (Eq. 7-8) tables, and the Boys scheme the kernels
use.  A numpy restatement of the corrected method built from those tables is compared with the
oracle, which pins the readings of Eqs. 7, 11 and 12 before any kernel runs."""
import math
import os
import re

import numpy as np
import pytest
import scipy.special as sp

import oracle
from paper_2404_16245_gb300 import workloads as W
from tests import refmath as RM

shgo = pytest.importorskip("paper_2404_16245_gb300.shgo", reason="libshgo.so not built")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_abi_exports_every_declared_symbol():
    import ctypes
    lib = ctypes.CDLL(shgo._build.LIB)
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(shgo_[a-z0-9_]+)\s*\(", txt)
    assert "shgo_basis_create" in names and "shgo_nuclear_attraction" in names and "shgo_free" in names
    for n in set(names):
        assert hasattr(lib, n), n


def test_invalid_arguments_are_rejected_without_gpu_work():
    with pytest.raises(shgo.ShgoError) as e:
        shgo.shgo_basis_create(1, [9], [1], [1.0], [1.0], [0.0, 0.0, 0.0])
    assert e.value.status == 2
    with pytest.raises(shgo.ShgoError) as e:
        shgo.shgo_basis_create(1, [1], [1], [-1.0], [1.0], [0.0, 0.0, 0.0])
    assert e.value.status == 1
    with pytest.raises(shgo.ShgoError):
        shgo.shgo_basis_create(1, [1], [0], [], [], [0.0, 0.0, 0.0])


def test_non_finite_and_out_of_range_inputs_are_rejected_on_the_host():
    """Basis creation validates on the host before any device work: NaN or infinite exponents,
    coefficients or centres, zero or negative exponents and primitive counts outside 1..64."""
    bad = [
        ([1], [1], [float("nan")], [1.0], [0.0, 0.0, 0.0]),
        ([1], [1], [float("inf")], [1.0], [0.0, 0.0, 0.0]),
        ([1], [1], [0.0], [1.0], [0.0, 0.0, 0.0]),
        ([1], [1], [1.0], [float("nan")], [0.0, 0.0, 0.0]),
        ([1], [1], [1.0], [float("-inf")], [0.0, 0.0, 0.0]),
        ([1], [1], [1.0], [1.0], [0.0, float("nan"), 0.0]),
        ([0], [65], [1.0] * 65, [1.0] * 65, [0.0, 0.0, 0.0]),
    ]
    for l, npr, ex, co, xyz in bad:
        with pytest.raises(shgo.ShgoError) as e:
            shgo.shgo_basis_create(1, l, npr, ex, co, xyz)
        assert e.value.status == 1


def test_every_entry_point_rejects_null_handles_without_gpu_work():
    """Failure detection on the host: every call on a basis, batch or network handle returns
    SHGO_ERR_INVALID_ARG for a NULL handle before any device work; size queries answer -1 and the
    free calls accept NULL."""
    import ctypes
    lib = ctypes.CDLL(shgo._build.LIB)
    vp, i64, i32, f32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_double
    N = None
    calls = {
        "shgo_nuclear_attraction": ([vp] * 5, [N] * 5),
        "shgo_nuclear_attraction_timed": ([vp] * 6, [N] * 6),
        "shgo_nuclear_attraction_class_timed": ([vp] * 6, [N] * 6),
        "shgo_nuclear_attraction_batched": ([vp] * 5, [N] * 5),
        "shgo_esp": ([vp] * 5, [N] * 5),
        "shgo_esp_gradient": ([vp] * 5, [N] * 5),
        "shgo_overlap": ([vp] * 3, [N] * 3),
        "shgo_coulomb_2c": ([vp] * 3, [N] * 3),
        "shgo_eri": ([vp] * 3, [N] * 3),
        "shgo_eri_jk": ([vp] * 5, [N] * 5),
        "shgo_batch_layout": ([vp] * 3, [N] * 3),
        "shgo_pair_shells": ([vp] * 3, [N] * 3),
        "shgo_screen_mask": ([vp] * 2, [N] * 2),
        "shgo_basis_flops": ([vp, i64, vp, vp], [N, 4, N, N]),
        "shgo_basis_class_stats": ([vp, i64, i32, vp, vp], [N, 4, 0, N, N]),
        "shgo_screen_features": ([vp, vp, vp, vp, i64, vp, vp], [N, N, N, N, 0, N, N]),
        "shgo_screen_build": ([vp, vp, vp, vp, i64, f64, f64, vp, vp], [N, N, N, N, 0, -12.0, 0.0, N, N]),
        "shgo_nuclear_attraction_screened": ([vp, vp, vp, i64, vp, vp], [N, N, N, 0, N, N]),
        "shgo_mlp_get_params": ([vp] * 2, [N] * 2),
        "shgo_mlp_forward": ([vp, vp, i64, vp, vp], [N, N, 1, N, N]),
        "shgo_mlp_gradients": ([vp, vp, vp, i64, f32, vp, vp], [N, N, N, 1, 4.0, N, N]),
        "shgo_mlp_train_step": ([vp, vp, vp, i64, f32, f32, vp, vp], [N, N, N, 1, 4.0, 1e-3, N, N]),
    }
    for name, (types, args) in calls.items():
        f = getattr(lib, name)
        f.argtypes, f.restype = types, ctypes.c_int
        assert f(*args) == 1, name
    for name in ("shgo_basis_nbf", "shgo_basis_npairs", "shgo_basis_launches", "shgo_batch_out_size"):
        f = getattr(lib, name)
        f.argtypes, f.restype = [vp], i64
        assert f(N) == -1, name
    lib.shgo_basis_nclasses.argtypes, lib.shgo_basis_nclasses.restype = [vp], i32
    assert lib.shgo_basis_nclasses(N) == -1
    lib.shgo_free.argtypes, lib.shgo_free.restype = [vp], None
    lib.shgo_free(N)
    lib.shgo_mlp_free.argtypes, lib.shgo_mlp_free.restype = [vp], None
    lib.shgo_mlp_free(N)


@pytest.mark.parametrize("l", range(0, 18))
def test_host_harmonic_recursion_matches_scipy(l):
    rng = np.random.default_rng(l)
    pts = rng.normal(size=(30, 3))
    got = shgo.host_solid_harmonics(l, pts)
    ref = RM.solid_harmonics_scipy(l, pts)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("l1,l2", [(0, 0), (1, 1), (2, 1), (3, 3), (4, 2), (5, 5), (8, 7), (8, 8)])
def test_gaunt_product_rule(l1, l2):
    # S_{l1 m1} S_{l2 m2} = sum_{L,M} G r^{l1+l2-L} S_{LM} at random points (Supp. Eq. 4 product rule)
    rng = np.random.default_rng(10 * l1 + l2)
    pts = rng.normal(size=(12, 3))
    r = np.linalg.norm(pts, axis=1)
    S1 = RM.solid_harmonics_scipy(l1, pts)
    S2 = RM.solid_harmonics_scipy(l2, pts)
    SL = {L: RM.solid_harmonics_scipy(L, pts) for L in range(abs(l1 - l2), l1 + l2 + 1)}
    for m1 in range(-l1, l1 + 1):
        for m2 in range(-l2, l2 + 1):
            rhs = np.zeros(len(pts))
            for L in range(abs(l1 - l2), l1 + l2 + 1, 2):
                for M in range(-L, L + 1):
                    g = shgo.host_gaunt(l1, m1, l2, m2, L, M)
                    if g:
                        rhs += g * r ** (l1 + l2 - L) * SL[L][:, M + L]
            lhs = S1[:, m1 + l1] * S2[:, m2 + l2]
            assert np.allclose(lhs, rhs, rtol=1e-11, atol=1e-11 * np.max(np.abs(lhs) + 1))


@pytest.mark.parametrize("la", range(0, 9))
def test_translation_addition_theorem(la):
    # S_{la,ma}(x + y) = sum_{l1,m1,nu} E S_{l1,m1}(x) S_{la-l1,nu}(y)   (Eqs. 7-8, real basis)
    rng = np.random.default_rng(50 + la)
    x = rng.normal(size=(10, 3))
    y = rng.normal(size=(10, 3))
    lhs = RM.solid_harmonics_scipy(la, x + y)
    Sx = {l: RM.solid_harmonics_scipy(l, x) for l in range(la + 1)}
    Sy = {l: RM.solid_harmonics_scipy(l, y) for l in range(la + 1)}
    for ma in range(-la, la + 1):
        rhs = np.zeros(len(x))
        for l1 in range(la + 1):
            lr = la - l1
            for m1 in range(-l1, l1 + 1):
                for nu in range(-lr, lr + 1):
                    e = shgo.host_translation(la, ma, l1, m1, nu)
                    if e:
                        rhs += e * Sx[l1][:, m1 + l1] * Sy[lr][:, nu + lr]
        assert np.allclose(lhs[:, ma + la], rhs, rtol=1e-11, atol=1e-11 * (1 + np.max(np.abs(lhs))))


@pytest.mark.parametrize("T", [0.0, 1e-9, 0.01, 0.03124, 0.5, 3.3, 17.0, 39.97, 40.0, 55.5, 300.0, 1e5])
def test_boys_scheme(T):
    F = shgo.host_boys(17, T)
    for n in range(18):
        if T == 0:
            ref = 1.0 / (2 * n + 1)
        else:
            ref = sp.gamma(n + 0.5) * sp.gammainc(n + 0.5, T) / (2 * T ** (n + 0.5))
            if T < 1e-6:
                ref = 1.0 / (2 * n + 1) - T / (2 * n + 3)
        assert F[n] == pytest.approx(ref, rel=5e-14, abs=1e-300)


# ----------------------------------------------------------------- numpy model of the method
def _rlayout(lam):
    idx = {}
    e = 0
    for L in range(lam + 1):
        km = (lam - L) // 2
        for M in range(-L, L + 1):
            for k in range(km + 1):
                idx[(L, M, k)] = e
                e += 1
    return idx


def method_block(la, lb, A, B, alphas, betas, ca, cb, C, Z):
    """V block of one shell pair by Eq. 11 with the coupled one-centre integral (corrected Eq. 12)
    and the shift vectors b-a / a-b.  ca/cb are coefficients of normalised primitives already
    scaled for the contracted normalisation."""
    lam = la + lb
    AB = B - A
    V = np.zeros((2 * la + 1, 2 * lb + 1))
    Sab = {l: shgo.host_solid_harmonics(l, AB[None])[0] for l in range(max(la, lb) + 1)}
    TA = np.zeros((2 * la + 1, (la + 1) ** 2))
    TB = np.zeros((2 * lb + 1, (lb + 1) ** 2))
    for ma in range(-la, la + 1):
        for l1 in range(la + 1):
            for m1 in range(-l1, l1 + 1):
                TA[ma + la, l1 * l1 + l1 + m1] = sum(shgo.host_translation(la, ma, l1, m1, nu) * Sab[la - l1][nu + la - l1]
                                                     for nu in range(-(la - l1), la - l1 + 1))
    for mb in range(-lb, lb + 1):
        for l2 in range(lb + 1):
            for m2 in range(-l2, l2 + 1):
                TB[mb + lb, l2 * l2 + l2 + m2] = (-1) ** (lb - l2) * sum(
                    shgo.host_translation(lb, mb, l2, m2, nu) * Sab[lb - l2][nu + lb - l2] for nu in range(-(lb - l2), lb - l2 + 1))
    Wt = np.zeros(((la + 1) ** 2, (lb + 1) ** 2))
    for i, a in enumerate(alphas):
        for j, b in enumerate(betas):
            p = a + b
            P = (a * A + b * B) / p
            K = math.exp(-a * b / p * AB @ AB)
            R = {}
            for Cc, Zc in zip(C, Z):
                d = Cc - P
                s = d @ d
                T = p * s
                F = shgo.host_boys(lam, T)
                SL = {L: shgo.host_solid_harmonics(L, d[None])[0] for L in range(lam + 1)}
                for L in range(lam + 1):
                    for k in range((lam - L) // 2 + 1):
                        beta = sum(math.factorial(k) / math.factorial(jj) * T ** jj * F[L + jj] for jj in range(k + 1))
                        for M in range(-L, L + 1):
                            R[(L, M, k)] = R.get((L, M, k), 0.0) + Zc * SL[L][M + L] * beta
            for l1 in range(la + 1):
                for m1 in range(-l1, l1 + 1):
                    for l2 in range(lb + 1):
                        for m2 in range(-l2, l2 + 1):
                            acc = 0.0
                            for L in range(abs(l1 - l2), l1 + l2 + 1, 2):
                                k = (l1 + l2 - L) // 2
                                for M in range(-L, L + 1):
                                    g = shgo.host_gaunt(l1, m1, l2, m2, L, M)
                                    if g:
                                        acc += g * 2 * math.pi * p ** (-(k + 1)) * R[(L, M, k)]
                            Wt[l1 * l1 + l1 + m1, l2 * l2 + l2 + m2] += (
                                ca[i] * cb[j] * K * (b / p) ** (la - l1) * (a / p) ** (lb - l2) * acc)
    return TA @ Wt @ TB.T


def _norm_coefs(l, exps, coefs):
    d = np.array([c * oracle.prim_norm(l, e) for c, e in zip(coefs, exps)])
    basis = W.make_basis([l], [len(exps)], exps, coefs, [[0, 0, 0]])
    S = oracle.overlap(basis)
    return d  # oracle renormalises internally; the ratio is applied below


@pytest.mark.parametrize("la,lb", [(0, 0), (1, 0), (1, 1), (2, 1), (2, 2), (3, 2), (4, 3)])
def test_method_model_matches_oracle(la, lb):
    rng = np.random.default_rng(100 * la + lb)
    A = rng.uniform(-1, 1, 3)
    B = rng.uniform(-1, 1, 3) + np.array([0.7, 0.0, -0.4])
    alphas = np.exp(rng.uniform(-1, 1.5, 2))
    betas = np.exp(rng.uniform(-1, 1.5, 2))
    ca = rng.uniform(0.2, 1.0, 2)
    cb = rng.uniform(0.2, 1.0, 2)
    C = rng.uniform(-1.5, 1.5, (2, 3))
    Z = np.array([2.0, 5.0])
    basis = W.make_basis([la, lb], [2, 2], np.concatenate([alphas, betas]), np.concatenate([ca, cb]), [A, B])
    Vo = oracle.nuclear_attraction(basis, C, Z)[: 2 * la + 1, 2 * la + 1:]

    def contracted(l, ex, co):
        d = np.array([c * oracle.prim_norm(l, e) for c, e in zip(co, ex)])
        self = sum(co[i] * co[j] * (2 * math.sqrt(ex[i] * ex[j]) / (ex[i] + ex[j])) ** (l + 1.5)
                   for i in range(len(ex)) for j in range(len(ex)))
        return d / math.sqrt(self)

    Vm = method_block(la, lb, A, B, alphas, betas, contracted(la, alphas, ca), contracted(lb, betas, cb), C, Z)
    assert np.max(np.abs(Vm - Vo)) <= 1e-12 * max(1.0, np.max(np.abs(Vo)))


def test_printed_eq12_differs_from_the_coupled_form():
    # Eq. 12 as printed keeps only L = l1 + l2; for l1 = l2 = 1, m = 0 and C = P it gives 0,
    # while the integrand z^2 e^{-p r^2}/r is positive: the coupled form is required.
    basis = W.make_basis([1, 1], [1, 1], [0.6, 0.7], [1, 1], [[0, 0, 0], [0, 0, 0]])
    V = oracle.nuclear_attraction(basis, np.zeros((1, 3)), [1.0])
    assert V[1, 4] > 0.1  # (m = 0, m = 0) block element


@pytest.mark.parametrize("L", [0, 1, 3, 6])
def test_laplacian_and_eps_tables_by_symbolic_differentiation(L):
    """The library's a_{k,j}(L) and eps_{k,n}(L) tables against sympy.  With f(u) = exp(-p u) and
    Delta_L g = 4u g'' + (4L + 6) g' (the Laplacian of S_LM(R) g(|R|^2) divided by S_LM):
    Delta_L^k f = sum_j a_{k,j} u^j f^{(k+j)}, and u^k f = sum_n eps_{k,n} p^{-(k+n)} Delta_L^n f."""
    sympy = pytest.importorskip("sympy")
    u, p = sympy.symbols("u p", positive=True)
    f = sympy.exp(-p * u)

    def DL(g):
        return 4 * u * sympy.diff(g, u, 2) + (4 * L + 6) * sympy.diff(g, u)

    g = f
    for k in range(5):
        rhs = sum(sympy.Rational(shgo.host_laplacian_coef(L, k, j)) * u ** j * sympy.diff(f, u, k + j)
                  for j in range(k + 1))
        assert sympy.simplify(g - rhs) == 0, (L, k)
        g = DL(g)
    for k in range(5):
        tot, h = 0, f
        for n in range(k + 1):
            tot += sympy.Rational(shgo.host_eri_eps(L, k, n)) * p ** (-(k + n)) * h
            h = DL(h)
        assert sympy.simplify(tot - u ** k * f) == 0, (L, k)


def _eri_model(ls, exps, centres):
    """(ab|cd) of four normalised primitives by the route of the four-centre kernels, from the library's host
    tables: each pair translated to its product centre (Eq. 7, real addition theorem), its harmonics coupled
    there (Gaunt), r^{2k} S_LM e^{-pr^2} as Laplacian powers (eps table), and the two pairs applied as harmonic
    gradients to the s-s integral (product rule, Hobson's theorem, the a_{K,j} table, Boys values)."""
    import functools
    G = functools.lru_cache(None)(shgo.host_gaunt)
    T = functools.lru_cache(None)(shgo.host_translation)

    def S(l, v):
        return shgo.host_solid_harmonics(l, np.asarray(v, float).reshape(1, 3))[0]

    def entries(lam):
        return [(L, M, n) for L in range(lam + 1) for M in range(-L, L + 1) for n in range((lam - L) // 2 + 1)]

    def dist(la, lb, al, be, A, B, Na, Nb):
        p = al + be
        K = math.exp(-al * be / p * float(np.sum((A - B) ** 2)))
        sba, sab = {l: S(l, B - A) for l in range(la + 1)}, {l: S(l, A - B) for l in range(lb + 1)}
        EA = {(ma, l1, m1): (be / p) ** (la - l1) * sum(T(la, ma, l1, m1, nu) * sba[la - l1][nu + la - l1]
                                                         for nu in range(-(la - l1), la - l1 + 1))
              for ma in range(-la, la + 1) for l1 in range(la + 1) for m1 in range(-l1, l1 + 1)}
        EB = {(mb, l2, m2): (al / p) ** (lb - l2) * sum(T(lb, mb, l2, m2, nu) * sab[lb - l2][nu + lb - l2]
                                                         for nu in range(-(lb - l2), lb - l2 + 1))
              for mb in range(-lb, lb + 1) for l2 in range(lb + 1) for m2 in range(-l2, l2 + 1)}
        ks = entries(la + lb)
        D = np.zeros(((2 * la + 1) * (2 * lb + 1), len(ks)))
        for ia, ma in enumerate(range(-la, la + 1)):
            for ib, mb in enumerate(range(-lb, lb + 1)):
                Y = {}
                for l1 in range(la + 1):
                    for m1 in range(-l1, l1 + 1):
                        for l2 in range(lb + 1):
                            for m2 in range(-l2, l2 + 1):
                                w = EA[(ma, l1, m1)] * EB[(mb, l2, m2)]
                                for L1 in range(abs(l1 - l2), l1 + l2 + 1, 2):
                                    for M1 in range(-L1, L1 + 1):
                                        g = G(l1, m1, l2, m2, L1, M1)
                                        if g:
                                            key = (L1, M1, (l1 + l2 - L1) // 2)
                                            Y[key] = Y.get(key, 0.0) + g * w
                for c, (L1, M1, n1) in enumerate(ks):
                    v = sum(shgo.host_eri_eps(L1, k1, n1) * p ** (-(k1 + n1)) * Y.get((L1, M1, k1), 0.0)
                            for k1 in range(n1, (la + lb - L1) // 2 + 1))
                    D[ia * (2 * lb + 1) + ib, c] = Na * Nb * K * (2 * p) ** (-L1) * v
        return D, p, (al * A + be * B) / p, ks

    la, lb, lc, ld = ls
    A, B, C, Dd = [np.asarray(x, float) for x in centres]
    N = [oracle.prim_norm(l, e) for l, e in zip(ls, exps)]
    D1, p, P, k1 = dist(la, lb, exps[0], exps[1], A, B, N[0], N[1])
    D2, q, Q, k2 = dist(lc, ld, exps[2], exps[3], C, Dd, N[2], N[3])
    R = P - Q
    u, rho, lt = float(R @ R), p * q / (p + q), la + lb + lc + ld
    F = shgo.host_boys(lt, rho * u)
    g = [2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * (-rho) ** n * F[n] for n in range(lt + 1)]
    SR = {L: S(L, R) for L in range(lt + 1)}
    Im = np.zeros((len(k1), len(k2)))
    for i, (L1, M1, n1) in enumerate(k1):
        for j, (L2, M2, n2) in enumerate(k2):
            v = 0.0
            for L in range(abs(L1 - L2), L1 + L2 + 1, 2):
                K = (L1 + L2 - L) // 2 + n1 + n2
                rad = sum(shgo.host_laplacian_coef(L, K, jj) * u ** jj * g[L + K + jj] for jj in range(K + 1))
                for M in range(-L, L + 1):
                    gg = G(L1, M1, L2, M2, L, M)
                    if gg:
                        v += gg * 2 ** L * SR[L][M + L] * rad
            Im[i, j] = (-1) ** L2 * v
    return (D1 @ Im @ D2.T).reshape(2 * la + 1, 2 * lb + 1, 2 * lc + 1, 2 * ld + 1)


@pytest.mark.parametrize("ls", [(0, 0, 0, 0), (1, 0, 0, 0), (1, 1, 0, 0), (0, 0, 1, 1), (2, 1, 1, 0), (2, 2, 2, 1),
                                (3, 1, 2, 2)])
def test_eri_method_model_matches_oracle(ls):
    """The four-centre route of Eqs. 13-15 as re-derived (Laplacian powers for the r^{2k} factors), built from
    the library's own tables, equals the McMurchie-Davidson oracle on single quartets."""
    rng = np.random.default_rng(sum((i + 1) * l for i, l in enumerate(ls)))
    exps = np.exp(rng.uniform(np.log(0.3), np.log(5.0), 4))
    cen = rng.uniform(0, 2.5, (4, 3))
    basis = W.make_basis(list(ls), [1] * 4, exps, [1.0] * 4, cen)
    E = oracle.eri(basis, precision="ld")
    off = np.concatenate([[0], np.cumsum(2 * np.array(ls) + 1)])
    ref = E[off[0]:off[1], off[1]:off[2], off[2]:off[3], off[3]:off[4]]
    got = _eri_model(ls, exps, cen)
    assert np.max(np.abs(got - ref)) <= 1e-14 + 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("ls,exps,shared", [
    ((2, 2, 2, 2), (0.05, 0.1, 5000.0, 3000.0), "ket"),
    ((3, 1, 2, 2), (5000.0, 3000.0, 0.05, 0.1), "bra"),
    ((2, 1, 2, 1), (0.05, 4000.0, 0.08, 2500.0), "both"),
])
def test_eri_method_model_wide_exponent_ratios(ls, exps, shared):
    """The Laplacian-power form sums terms of alternating sign; with exponents 1e5 apart (tight pairs on one
    centre, so the Gaussian product factor stays 1) it still meets the parity bar against the oracle."""
    A, B, C = np.zeros(3), np.array([0.9, -0.4, 0.6]), np.array([1.7, 0.8, -0.5])
    cen = {"ket": (A, B, C, C), "bra": (A, A, B, C), "both": (A, A, C, C)}[shared]
    basis = W.make_basis(list(ls), [1] * 4, np.array(exps), [1.0] * 4, list(cen))
    E = oracle.eri(basis, precision="ld")
    off = np.concatenate([[0], np.cumsum(2 * np.array(ls) + 1)])
    ref = E[off[0]:off[1], off[1]:off[2], off[2]:off[3], off[3]:off[4]]
    got = _eri_model(ls, np.array(exps), cen)
    assert np.all(np.abs(got - ref) <= 1e-13 + 1e-11 * np.abs(ref))


def test_option_flags_are_validated_on_the_host():
    """Unknown option bits and a block-sparse batch are rejected before any device work."""
    import ctypes
    opt = shgo.shgo_options(0, -1, 64)
    h = ctypes.c_void_p()
    l = np.array([0], dtype=np.int32)
    npr = np.array([1], dtype=np.int32)
    one = np.array([1.0])
    xyz = np.zeros(3)
    st = shgo._lib.shgo_basis_create(1, shgo._ptr(l, ctypes.c_int32), shgo._ptr(npr, ctypes.c_int32),
                                     shgo._ptr(one, ctypes.c_double), shgo._ptr(one, ctypes.c_double),
                                     shgo._ptr(xyz, ctypes.c_double), ctypes.byref(opt), ctypes.byref(h))
    assert st == 1 and "flag" in shgo._lib.shgo_last_error().decode()
    opt = shgo.shgo_options(0, -1, shgo.SHGO_FLAG_BLOCK_SPARSE)
    nsh = np.array([1], dtype=np.int32)
    nc = np.array([1], dtype=np.int64)
    st = shgo._lib.shgo_batch_create(1, shgo._ptr(nsh, ctypes.c_int32), shgo._ptr(nc, ctypes.c_int64), 1,
                                     shgo._ptr(l, ctypes.c_int32), shgo._ptr(npr, ctypes.c_int32),
                                     shgo._ptr(one, ctypes.c_double), shgo._ptr(one, ctypes.c_double),
                                     shgo._ptr(xyz, ctypes.c_double), ctypes.byref(opt), ctypes.byref(h))
    assert st == 1 and "batch" in shgo._lib.shgo_last_error().decode()
    with pytest.raises(shgo.ShgoError):
        shgo.shgo_sparse_layout(0)


def _r_layout(lam):
    return [(L, M, k) for L in range(lam + 1) for M in range(-L, L + 1) for k in range((lam - L) // 2 + 1)]


def _one_centre_values(lam, x):
    # r^{2k} S_LM(x) for every entry of the layout of order lam (scipy's harmonics)
    r2 = float(np.dot(x, x))
    S = {L: RM.solid_harmonics_scipy(L, x[None, :])[0] for L in range(lam + 1)}
    return np.array([r2 ** k * S[L][M + L] for (L, M, k) in _r_layout(lam)])


@pytest.mark.parametrize("lam", [0, 1, 4, 9, 16])
def test_deriv_transform_raise_and_field(lam):
    # the tables behind the derivative integrals, applied to the integrand itself at a point: raising must
    # give x_c r^{2k} S_LM, the field step d/dx_c [r^{2k} S_LM e^{-p r^2}] e^{p r^2} (fourth-order differences)
    rng = np.random.default_rng(100 + lam)
    p = 0.7
    for _ in range(3):
        x = rng.uniform(-1.2, 1.2, 3)
        r1 = _one_centre_values(lam + 1, x)
        base = _one_centre_values(lam, x)
        lay = _r_layout(lam)
        for c in range(3):
            raised, field = shgo.host_deriv_transform(lam, c, p, r1)
            assert np.allclose(raised, x[c] * base, rtol=1e-12, atol=1e-12 * np.max(np.abs(base)))
            h = 1e-4

            def f(t):
                y = x.copy()
                y[c] += t
                return _one_centre_values(lam, y) * np.exp(-p * float(np.dot(y, y)))

            fd = (8 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12 * h) * np.exp(p * float(np.dot(x, x)))
            scale = np.max(np.abs(fd))
            assert np.max(np.abs(field - fd)) <= 1e-8 * scale, (lam, c, lay[int(np.argmax(np.abs(field - fd)))])


@pytest.mark.parametrize("l", [1, 2, 5, 8])
def test_deriv_lowering_is_the_gradient_of_the_harmonic(l):
    rng = np.random.default_rng(200 + l)
    x = rng.normal(size=3)
    Sl1 = RM.solid_harmonics_scipy(l - 1, x[None, :])[0]
    h = 1e-5
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        S = lambda y: RM.solid_harmonics_scipy(l, y[None, :])[0]  # noqa: E731
        fd = (8 * (S(x + e) - S(x - e)) - (S(x + 2 * e) - S(x - 2 * e))) / (12 * h)
        for m in range(-l, l + 1):
            w = shgo.host_deriv_lowering(l, c, m)
            assert abs(float(w @ Sl1) - fd[m + l]) <= 1e-8 * max(1.0, np.max(np.abs(fd)))


def test_deriv_entry_points_reject_bad_arguments():
    import ctypes
    c = shgo.shgo_centers(0, None)
    for fn in (shgo._lib.shgo_nuclear_attraction_deriv, shgo._lib.shgo_nuclear_field):
        assert fn(None, ctypes.byref(c), None, None, None) == 1  # SHGO_ERR_INVALID_ARG
    assert shgo._lib.shgo_nuclear_attraction_gradient(None, None, ctypes.byref(c), None, None, None) == 1
    with pytest.raises(shgo.ShgoError):
        shgo.host_deriv_transform(17, 0, 1.0, np.zeros(2000))
    with pytest.raises(shgo.ShgoError):
        shgo.host_deriv_lowering(0, 0, 0)
