"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test checks the oracle against something other than itself: closed forms (Eq. 5 product,
the s-s Boys form, F_0 = sqrt(pi/T) erf(sqrt T)/2), scipy's special functions and spherical
harmonics, brute-force 3-D quadrature, and invariances of the exact integral (hermiticity,
translation, rotation covariance by fitted Wigner-D blocks, linearity in the charges, far field).
"""
import math

import numpy as np
import pytest
import scipy.special as sp

import oracle
from paper_2404_16245_gb300 import workloads as W
from tests import refmath as RM


# ---------------------------------------------------------------- Boys function (after Eq. 12)
@pytest.mark.parametrize("T", [1e-12, 1e-6, 0.01, 0.5, 3.0, 11.0, 29.9, 30.1, 47.0, 60.0, 150.0, 2e3, 1e6])
def test_boys_f0_closed_form(T):
    ref = math.sqrt(math.pi / T) * math.erf(math.sqrt(T)) / 2
    assert oracle.boys(0, T)[0] == pytest.approx(ref, rel=2e-15)


def test_boys_zero_argument():
    F = oracle.boys(20, 0.0)
    assert np.allclose(F, 1.0 / (2 * np.arange(21) + 1), rtol=1e-15, atol=0)


@pytest.mark.parametrize("n", [1, 2, 5, 8, 12, 16, 20])
@pytest.mark.parametrize("T", [0.2, 1.7, 6.0, 19.0, 35.0, 55.0, 80.0, 300.0])
def test_boys_quadrature(n, T):
    # definition F_n(T) = int_0^1 u^{2n} exp(-T u^2) du by composite Gauss-Legendre
    u, w = [], []
    edges = np.linspace(0, 1, 41)
    for a, b in zip(edges[:-1], edges[1:]):
        x, ww = RM.gauss_legendre(40, a, b)
        u.append(x)
        w.append(ww)
    u = np.concatenate(u)
    w = np.concatenate(w)
    ref = np.sum(w * u ** (2 * n) * np.exp(-T * u * u))
    assert oracle.boys(n, T)[n] == pytest.approx(ref, rel=1e-13)


@pytest.mark.parametrize("T", [0.5, 4.0, 25.0, 41.0, 120.0])
def test_boys_incomplete_gamma(T):
    F = oracle.boys(16, T)
    for n in range(17):
        ref = sp.gamma(n + 0.5) * sp.gammainc(n + 0.5, T) / (2 * T ** (n + 0.5))
        assert F[n] == pytest.approx(ref, rel=1e-13)


@pytest.mark.parametrize("T", [0.01, 2.0, 33.0, 40.0, 77.0])
def test_boys_recursion_identity(T):
    F = oracle.boys(18, T)
    n = np.arange(18)
    lhs = 2 * T * F[1:]
    rhs = (2 * n + 1) * F[:-1] - math.exp(-T)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-300)


# ---------------------------------------------------------------- solid harmonics (Eq. 2)
@pytest.mark.parametrize("l", range(0, 11))
def test_solid_harmonics_match_scipy(l):
    rng = np.random.default_rng(100 + l)
    pts = rng.normal(size=(40, 3)) * 1.3
    got = oracle.solid_harmonic(l, pts)
    ref = RM.solid_harmonics_scipy(l, pts)
    scale = np.max(np.abs(ref)) + 1e-300
    assert np.max(np.abs(got - ref)) <= 1e-13 * scale


def test_solid_harmonics_low_order_explicit():
    x, y, z = 0.3, -1.1, 0.7
    S1 = oracle.solid_harmonic(1, [[x, y, z]])[0]
    assert np.allclose(S1, [y, z, x], rtol=0, atol=1e-15)
    S2 = oracle.solid_harmonic(2, [[x, y, z]])[0]
    r2 = x * x + y * y + z * z
    ref = [math.sqrt(3) * x * y, math.sqrt(3) * y * z, z * z - 0.5 * (x * x + y * y), math.sqrt(3) * x * z,
           math.sqrt(3) / 2 * (x * x - y * y)]
    assert np.allclose(S2, ref, rtol=0, atol=1e-15)
    assert abs(ref[2] - (1.5 * z * z - 0.5 * r2)) < 1e-15


# ---------------------------------------------------------------- normalisation (Eq. 1, Eq. 10)
@pytest.mark.parametrize("l", range(0, 9))
def test_primitive_norm_radial_quadrature(l):
    for a in (0.05, 1.0, 37.0):
        assert oracle.prim_norm(l, a) == pytest.approx(RM.radial_norm(l, a), rel=1e-12)


def test_self_overlap_is_identity_per_shell():
    basis = W.random_basis(7, 18, 8, max_prim=5)
    S = oracle.overlap(basis)
    off = np.concatenate([[0], np.cumsum(2 * basis["l"] + 1)])
    for s in range(len(basis["l"])):
        blk = S[off[s]:off[s + 1], off[s]:off[s + 1]]
        assert np.allclose(blk, np.eye(len(blk)), rtol=0, atol=1e-12)


def test_overlap_eq10_prefactor_one_centre():
    # Eq. 10 with a = b keeps only l1 = la = lb, where the epsilon factors are 1: the overlap of
    # two unnormalised primitives is 4 pi (pi/2)^{1/2} (2l-1)!!/[2p]^{l+3/2}, the Racah-normalised
    # angular integral 4 pi/(2l+1) times the radial moment int r^{2l+2} e^{-p r^2} dr
    for l in range(0, 7):
        a, b = 0.8, 2.3
        basis = W.make_basis([l, l], [1, 1], [a, b], [1.0, 1.0], [[0, 0, 0], [0, 0, 0]])
        S = oracle.overlap(basis)
        n = 2 * l + 1
        p = a + b
        dfact = float(np.prod(np.arange(2 * l - 1, 0, -2))) if l > 0 else 1.0
        eq10 = 4 * math.pi * math.sqrt(math.pi / 2) * dfact / (2 * p) ** (l + 1.5)
        ref = eq10 * RM.radial_norm(l, a) * RM.radial_norm(l, b)
        assert np.allclose(np.diag(S[:n, n:]), ref, rtol=1e-12)


def test_overlap_brute_force():
    basis = W.make_basis([1, 2], [2, 1], [0.9, 2.5, 1.4], [0.6, 0.4, 1.0], [[0, 0, 0], [0.4, -0.3, 0.8]])
    S = oracle.overlap(basis)
    # raw-normalised functions on a product grid about the first centre; renormalise numerically
    pts, w = RM.sphere_grid(60, 9.0, 40, 80, np.zeros(3))
    rho = np.linalg.norm(pts, axis=1)
    w = w * rho  # int f d^3r: restore the power of rho removed for 1/r kernels
    f0 = RM.shell_values(basis, 0, pts, [1.0, 1.0])
    n0 = np.sqrt(np.sum(w * f0[:, 0] ** 2))
    pts1, w1 = RM.sphere_grid(60, 9.0, 40, 80, basis["xyz"][1])
    w1 = w1 * np.linalg.norm(pts1 - basis["xyz"][1], axis=1)
    n1 = np.sqrt(np.sum(w1 * RM.shell_values(basis, 1, pts1, [1.0, 1.0])[:, 0] ** 2))
    fa = RM.shell_values(basis, 0, pts, [1 / n0, 1 / n1])
    fb = RM.shell_values(basis, 1, pts, [1 / n0, 1 / n1])
    ref = np.einsum("p,pi,pj->ij", w, fa, fb)
    assert np.allclose(S[:3, 3:], ref, rtol=0, atol=2e-11)


# ---------------------------------------------------------------- nuclear attraction
def test_ss_closed_form():
    # (2 pi / p) K_AB F_0(p |PC|^2) with K_AB and P of the Gaussian product rule (Eq. 5)
    rng = np.random.default_rng(3)
    for _ in range(5):
        a, b = np.exp(rng.uniform(-2, 3, 2))
        A, B, C = rng.uniform(-2, 2, (3, 3))
        Z = 3.0
        basis = W.make_basis([0, 0], [1, 1], [a, b], [1, 1], [A, B])
        V = oracle.nuclear_attraction(basis, C[None], [Z])
        p = a + b
        P = (a * A + b * B) / p
        K = math.exp(-a * b / p * np.sum((A - B) ** 2))
        T = p * np.sum((P - C) ** 2)
        F0 = math.sqrt(math.pi / T) * math.erf(math.sqrt(T)) / 2
        N = lambda x: (2 * x / math.pi) ** 0.75
        assert V[0, 1] == pytest.approx(Z * 2 * math.pi / p * K * F0 * N(a) * N(b), rel=1e-13)


def _brute_force_V(basis, centers, charges, n_rho=56, n_theta=48, n_phi=96, rho_max=10.0):
    n = len(basis["l"])
    # numerical contracted normalisation of every shell
    norms = []
    for s in range(n):
        pts, w = RM.sphere_grid(n_rho, rho_max, n_theta, n_phi, basis["xyz"][s])
        w = w * np.linalg.norm(pts - basis["xyz"][s], axis=1)
        f = RM.shell_values(basis, s, pts, np.ones(n))
        norms.append(1.0 / math.sqrt(np.sum(w * f[:, 0] ** 2)))
    nb = W.nbf(basis)
    V = np.zeros((nb, nb))
    off = np.concatenate([[0], np.cumsum(2 * basis["l"] + 1)])
    for C, Z in zip(centers, charges):
        pts, w = RM.sphere_grid(n_rho, rho_max, n_theta, n_phi, C)
        F = np.concatenate([RM.shell_values(basis, s, pts, norms) for s in range(n)], axis=1)
        V += Z * np.einsum("p,pi,pj->ij", w, F, F)
    return V


def test_brute_force_small_mixed():
    basis = W.make_basis([0, 1, 2, 1], [2, 1, 2, 1], [1.2, 0.4, 0.9, 1.5, 0.6, 2.0], [0.7, 0.5, 1.0, 0.3, 0.8, 1.0],
                         [[0, 0, 0], [0.0, 0.0, 0.0], [0.9, -0.4, 0.5], [-0.6, 0.7, -0.2]])
    centers = np.array([[0.3, -0.5, 0.8], [-0.4, 0.2, -0.3]])
    charges = np.array([2.0, 1.0])
    V = oracle.nuclear_attraction(basis, centers, charges)
    ref = _brute_force_V(basis, centers, charges)
    assert np.max(np.abs(V - ref)) < 1e-9 * np.max(np.abs(ref))


def test_brute_force_one_centre_l3():
    # both shells at P = 0, nucleus at (0.3, -0.5, 0.8): the one-centre integral of Eq. 11's last
    # line, including the coupled terms with L < l1 + l2 (l1 = 3, l2 = 2)
    basis = W.make_basis([3, 2], [1, 1], [0.6, 0.7], [1, 1], [[0, 0, 0], [0, 0, 0]])
    centers = np.array([[0.3, -0.5, 0.8]])
    V = oracle.nuclear_attraction(basis, centers, [1.0])
    ref = _brute_force_V(basis, centers, [1.0], n_rho=64, n_theta=56, n_phi=112)
    assert np.max(np.abs(V - ref)) < 1e-9 * np.max(np.abs(ref))


def test_hermitian():
    basis, pos, Z = W.config1()
    V = oracle.nuclear_attraction(basis, pos, Z)
    assert np.array_equal(V, V.T)


def test_translation_invariance():
    basis = W.random_basis(11, 10, 5, max_prim=3)
    C, Z = W.random_nuclei(12, 3)
    V = oracle.nuclear_attraction(basis, C, Z)
    shift = np.array([3.7, -11.2, 0.45])
    b2 = dict(basis)
    b2["xyz"] = basis["xyz"] + shift
    V2 = oracle.nuclear_attraction(b2, C + shift, Z)
    assert np.max(np.abs(V - V2)) < 1e-12 * np.max(np.abs(V))


@pytest.mark.parametrize("seed", [0, 1])
def test_rotation_covariance(seed):
    basis = W.random_basis(20 + seed, 9, 6, max_prim=2)
    C, Z = W.random_nuclei(30 + seed, 3)
    R = RM.rotation_matrix(seed)
    V = oracle.nuclear_attraction(basis, C, Z)
    b2 = dict(basis)
    b2["xyz"] = basis["xyz"] @ R.T
    V2 = oracle.nuclear_attraction(b2, C @ R.T, Z)
    off = np.concatenate([[0], np.cumsum(2 * basis["l"] + 1)])
    D = [RM.wigner_real(int(l), R) for l in basis["l"]]
    for a in range(len(basis["l"])):
        for b in range(len(basis["l"])):
            blk = V[off[a]:off[a + 1], off[b]:off[b + 1]]
            blk2 = V2[off[a]:off[a + 1], off[b]:off[b + 1]]
            assert np.allclose(D[a] @ blk @ D[b].T, blk2, rtol=0, atol=1e-11 * np.max(np.abs(V)))


def test_linear_in_charges_and_additive_over_nuclei():
    basis = W.random_basis(5, 8, 4, max_prim=3)
    C, Z = W.random_nuclei(6, 4)
    V = oracle.nuclear_attraction(basis, C, Z)
    parts = sum(oracle.nuclear_attraction(basis, C[i:i + 1], [1.0]) * Z[i] for i in range(4))
    assert np.allclose(V, parts, rtol=1e-13, atol=1e-14)


def test_far_field_limit():
    # V_ab -> Z S_ab / |C| as |C| -> infinity (monopole of the product distribution)
    basis = W.random_basis(8, 8, 4, max_prim=3, box=1.0)
    S = oracle.overlap(basis)
    R = 1e6
    C = np.array([[R, 0.3 * R, -0.2 * R]])
    dist = np.linalg.norm(C[0] - basis["xyz"].mean(axis=0))
    V = oracle.nuclear_attraction(basis, C, [2.0])
    assert np.allclose(V * dist / 2.0, S, rtol=0, atol=1e-5)


def test_degenerate_geometries():
    # nucleus at the product centre and coincident shell centres are valid inputs
    basis = W.make_basis([2, 2], [1, 1], [1.0, 1.0], [1, 1], [[0.5, 0.5, 0.5], [0.5, 0.5, 0.5]])
    V = oracle.nuclear_attraction(basis, np.array([[0.5, 0.5, 0.5]]), [1.0])
    assert np.all(np.isfinite(V))
    ref = _brute_force_V(basis, np.array([[0.5, 0.5, 0.5]]), [1.0])
    assert np.max(np.abs(V - ref)) < 1e-9 * np.max(np.abs(ref))


@pytest.mark.parametrize("la,lb", [(8, 8), (8, 5), (7, 7), (6, 3)])
def test_double_oracle_certified_by_extended_precision(la, lb):
    # the double build against the same code in long double (80-bit x86 / binary128 aarch64)
    tri = W.config5(12, replica=9)
    worst = 0.0
    for basis, C, Z in tri:
        b = dict(basis)
        b["l"] = np.array([la, lb], dtype=np.int32)
        V = oracle.nuclear_attraction(b, C, Z)
        Vl = oracle.nuclear_attraction(b, C, Z, precision="ld")
        scale = np.max(np.abs(Vl))
        if scale == 0:
            continue
        err = np.abs(V - Vl) / (1e-13 + 1e-11 * np.abs(Vl))
        worst = max(worst, float(np.max(err)))
    assert oracle.real_bits("ld") > 64
    assert worst <= 1.0


def test_field_integrals_are_the_position_derivative_of_V():
    # d V / d C from the shifted Hermite table against a fourth-order central difference of V itself
    basis = W.random_basis(7, 6, 4, max_prim=2, box=2.0, exp_lo=0.2, exp_hi=5.0)
    C, Z = np.array([[0.7, -0.3, 1.1], [1.9, 0.4, -0.6]]), np.array([1.0, -0.5])
    F = oracle.nuclear_field(basis, C, Z, precision="ld")
    h = 1e-3
    for c in range(3):
        e = np.zeros(3)
        e[c] = h

        def f(s):
            return oracle.nuclear_attraction(basis, C + s * e, Z, precision="ld")

        fd = (8 * (f(1) - f(-1)) - (f(2) - f(-2))) / (12 * h)
        assert np.max(np.abs(fd - F[c])) <= 1e-9 * np.max(np.abs(F[c]))


def test_field_ss_closed_form():
    # d/dC (2 pi / p) K_AB F_0(p |P - C|^2) N_a N_b = -(2 pi / p) K_AB N_a N_b F_1(T) 2 p (C - P)
    a, b = 0.8, 1.7
    A, B = np.array([0.0, 0.1, -0.2]), np.array([0.9, -0.4, 0.5])
    C = np.array([[0.3, 0.8, 0.2]])
    basis = W.make_basis([0, 0], [1, 1], [a, b], [1.0, 1.0], [A, B])
    p = a + b
    P = (a * A + b * B) / p
    K = math.exp(-a * b / p * float(np.sum((A - B) ** 2)))
    T = p * float(np.sum((P - C[0]) ** 2))
    F1 = sp.gamma(1.5) * sp.gammainc(1.5, T) / (2 * T ** 1.5)  # F_1(T) by the incomplete gamma function
    nn = oracle.prim_norm(0, a) * oracle.prim_norm(0, b)
    ref = -(2 * math.pi / p) * K * nn * F1 * 2 * p * (C[0] - P)
    F = oracle.nuclear_field(basis, C, np.ones(1))
    assert np.allclose(F[:, 0, 1], ref, rtol=1e-13, atol=1e-16)


# ---- two-centre Coulomb integrals (a|b) (the two-centre case of Eqs. 13-15) ----

def _norm_s(a):
    return (2 * a / math.pi) ** 0.75


@pytest.mark.parametrize("R", [0.0, 1.3, 7.5])
def test_coulomb2c_ss_closed_form(R):
    """(s|s) of normalised primitives: N_a N_b 2 pi^{5/2} / (a b sqrt(a + b)) F_0(rho R^2), rho = ab/(a+b),
    with F_0 from erf (the R = 0 limit 1 taken exactly)."""
    a, b = 0.7, 1.9
    basis = W.make_basis([0, 0], [1, 1], [a, b], [1.0, 1.0], [np.zeros(3), np.array([0.0, 0.0, R])])
    J = oracle.coulomb_2c(basis, precision="ld")
    T = a * b / (a + b) * R * R
    F0 = 1.0 if T == 0 else 0.5 * math.sqrt(math.pi / T) * sp.erf(math.sqrt(T))
    ref = _norm_s(a) * _norm_s(b) * 2 * math.pi ** 2.5 / (a * b * math.sqrt(a + b)) * F0
    assert J[0, 1] == pytest.approx(ref, rel=1e-14)
    self_ref = _norm_s(a) ** 2 * 2 * math.pi ** 2.5 / (a * a * math.sqrt(2 * a))
    assert J[0, 0] == pytest.approx(self_ref, rel=1e-14)


def test_coulomb2c_dipole_far_field():
    """Two p shells 400 bohr apart along z interact as point dipoles mu = int z phi_z: (z|z) -> -2 mu_a mu_b / R^3,
    (x|x) = (y|y) -> mu_a mu_b / R^3, mixed components -> 0 (relative corrections ~ (extent / R)^2)."""
    a, b, R = 0.9, 1.4, 400.0
    basis = W.make_basis([1, 1], [1, 1], [a, b], [1.0, 1.0], [np.zeros(3), np.array([0.0, 0.0, R])])
    J = oracle.coulomb_2c(basis, precision="ld")

    def mu(al):  # normalised primitive z exp(-al r^2): N^2 = 2 (2 al)^{5/2} / pi^{3/2}
        return math.sqrt(2 * (2 * al) ** 2.5 / math.pi ** 1.5) * (math.pi / al) ** 1.5 / (2 * al)

    d = mu(a) * mu(b) / R ** 3
    assert J[1, 4] == pytest.approx(-2 * d, rel=1e-8)   # m = 0 (z)
    assert J[0, 3] == pytest.approx(d, rel=1e-8)        # m = -1 (y)
    assert J[2, 5] == pytest.approx(d, rel=1e-8)        # m = +1 (x)
    assert abs(J[0, 4]) < 1e-12 * d and abs(J[1, 5]) < 1e-12 * d


@pytest.mark.parametrize("seed", [0, 1])
def test_coulomb2c_rotation_covariance_and_metric(seed):
    """(a|b) of a rotated basis is D^la (a|b) D^lb^T with fitted real Wigner blocks; the matrix is
    symmetric and positive definite (a Coulomb metric)."""
    basis = W.random_basis(40 + seed, 8, 4, max_prim=2)
    R = RM.rotation_matrix(seed)
    J = oracle.coulomb_2c(basis, precision="ld")
    b2 = dict(basis)
    b2["xyz"] = basis["xyz"] @ R.T
    J2 = oracle.coulomb_2c(b2, precision="ld")
    off = np.concatenate([[0], np.cumsum(2 * basis["l"] + 1)])
    D = [RM.wigner_real(int(l), R) for l in basis["l"]]
    for a in range(len(basis["l"])):
        for b in range(len(basis["l"])):
            blk = J[off[a]:off[a + 1], off[b]:off[b + 1]]
            blk2 = J2[off[a]:off[a + 1], off[b]:off[b + 1]]
            assert np.allclose(D[a] @ blk @ D[b].T, blk2, rtol=0, atol=1e-11 * np.max(np.abs(J)))
    assert np.array_equal(J, J.T)
    assert np.min(np.linalg.eigvalsh(J)) > 0


# ---- derivatives with respect to the basis-function centres ----

def _shift_shell(basis, s, delta):
    b = dict(basis)
    xyz = np.array(basis["xyz"], dtype=np.float64).reshape(-1, 3).copy()
    xyz[s] += delta
    b["xyz"] = xyz
    return b


def _shell_first(basis):
    l = np.asarray(basis["l"])
    return np.concatenate([[0], np.cumsum(2 * l + 1)]), l


@pytest.mark.parametrize("seed,lmax", [(11, 4), (12, 7)])
def test_centre_derivative_is_the_derivative_of_V(seed, lmax):
    # moving shell s moves the rows and the columns of its functions: dV/dX_s = D[s rows] + D[s rows]^T
    basis = W.random_basis(seed, 5, lmax, max_prim=2, box=2.5, exp_lo=0.2, exp_hi=4.0)
    C, Z = np.array([[0.4, -0.8, 0.3], [-1.0, 0.5, 0.9], [0.2, 0.2, -1.2]]), np.array([1.0, 2.5, -0.7])
    D = oracle.nuclear_deriv(basis, C, Z, precision="ld")
    first, l = _shell_first(basis)
    h = 1e-3
    for s in range(len(l)):
        rows = slice(first[s], first[s + 1])
        for c in range(3):
            e = np.zeros(3)
            e[c] = h

            def f(k):
                return oracle.nuclear_attraction(_shift_shell(basis, s, k * e), C, Z, precision="ld")

            fd = (8 * (f(1) - f(-1)) - (f(2) - f(-2))) / (12 * h)
            an = np.zeros_like(fd)
            an[rows, :] += D[c][rows, :]
            an[:, rows] += D[c][rows, :].T
            assert np.max(np.abs(fd - an)) <= 2e-9 * max(np.max(np.abs(an)), 1.0), (s, c)


def test_centre_derivatives_and_field_sum_to_zero():
    # translating the basis and the nuclei together leaves V unchanged: D + D^T + sum_C Z_C dV/dC = 0.
    # The two sides come from different recurrences (raised bra exponents against raised Hermite R).
    basis = W.random_basis(13, 9, 6, max_prim=3, box=3.0, exp_lo=0.1, exp_hi=30.0, n_sites=4)
    xyz = np.asarray(basis["xyz"]).reshape(-1, 3)
    C = np.vstack([xyz[0], np.array([[0.3, -0.2, 1.4], [-1.1, 0.6, 0.2]])])  # one nucleus on a basis centre
    Z = np.array([3.0, 1.0, -2.0])
    D = oracle.nuclear_deriv(basis, C, Z)
    F = oracle.nuclear_field(basis, C, Z)
    for c in range(3):
        scale = np.max(np.abs(F[c]))
        assert np.max(np.abs(D[c] + D[c].T + F[c])) <= 1e-12 * scale


def test_centre_derivative_ss_closed_form():
    # V = N_a N_b (2 pi / p) K F_0(T), K = exp(-mu |A - B|^2), T = p |P - C|^2, dP/dA = alpha / p:
    # dV/dA = N_a N_b (2 pi / p) K [-2 mu (A - B) F_0(T) - 2 alpha (P - C) F_1(T)]
    a, b = 0.9, 1.4
    A, B = np.array([0.2, -0.3, 0.4]), np.array([-0.7, 0.5, 1.1])
    C = np.array([[0.6, 0.9, -0.2]])
    basis = W.make_basis([0, 0], [1, 1], [a, b], [1.0, 1.0], [A, B])
    p, mu = a + b, a * b / (a + b)
    P = (a * A + b * B) / p
    K = math.exp(-mu * float(np.sum((A - B) ** 2)))
    T = p * float(np.sum((P - C[0]) ** 2))
    F0 = 0.5 * math.sqrt(math.pi / T) * sp.erf(math.sqrt(T))
    F1 = sp.gamma(1.5) * sp.gammainc(1.5, T) / (2 * T ** 1.5)
    nn = oracle.prim_norm(0, a) * oracle.prim_norm(0, b)
    ref = nn * (2 * math.pi / p) * K * (-2 * mu * (A - B) * F0 - 2 * a * (P - C[0]) * F1)
    D = oracle.nuclear_deriv(basis, C, np.ones(1))
    assert np.allclose(D[:, 0, 1], ref, rtol=1e-13, atol=1e-16)
    # the bra derivative of the (b, a) element moves B instead: swap the roles
    refB = nn * (2 * math.pi / p) * K * (-2 * mu * (B - A) * F0 - 2 * b * (P - C[0]) * F1)
    assert np.allclose(D[:, 1, 0], refB, rtol=1e-13, atol=1e-16)


def test_centre_derivative_one_centre_s_shell_vanishes_without_nuclei_offset():
    # a single s shell pair on one centre with the nucleus on that centre: V is stationary in A by symmetry
    basis = W.make_basis([0, 0], [1, 1], [0.8, 2.0], [1.0, 1.0], [np.zeros(3), np.zeros(3)])
    D = oracle.nuclear_deriv(basis, np.zeros((1, 3)), np.ones(1))
    assert np.max(np.abs(D)) <= 1e-14
