"""Pins of the oracle's four-centre electron-repulsion integrals (ab|cd) (Eqs. 13-15) against what
the mathematics fixes: the (ss|ss) closed form, covariance under reordering the shells and under a
rotation of the molecule, the point-charge limit of a tight ket (the pinned nuclear-attraction
integrals), the far-field limit (the pinned overlaps over the distance), the reduction of a pair
with a same-centre s function to the two-centre integrals, and positive semi-definiteness of the
Coulomb metric over orbital pairs."""
import math

import numpy as np
import pytest
from scipy import special as sp

import oracle
from paper_2404_16245_gb300 import workloads as W
from tests import refmath as RM


def _norm_s(a):
    return (2 * a / math.pi) ** 0.75


def _f0(T):
    return 1.0 if T == 0 else 0.5 * math.sqrt(math.pi / T) * sp.erf(math.sqrt(T))


@pytest.mark.parametrize("coincident", [False, True])
def test_eri_ssss_closed_form(coincident):
    """(ss|ss) of normalised primitives: N_a N_b N_c N_d K_AB K_CD 2 pi^{5/2} / (p q sqrt(p + q)) F_0(rho |PQ|^2)."""
    a, b, c, d = 0.7, 1.9, 0.4, 2.5
    A, B = np.zeros(3), np.array([0.3, -0.2, 1.1])
    if coincident:
        C, D = A.copy(), B.copy()
        c, d = a, b
    else:
        C, D = np.array([1.0, 0.5, -0.7]), np.array([-0.6, 1.2, 0.4])
    basis = W.make_basis([0] * 4, [1] * 4, [a, b, c, d], [1.0] * 4, [A, B, C, D])
    E = oracle.eri(basis, precision="ld")
    p, q = a + b, c + d
    P, Q = (a * A + b * B) / p, (c * C + d * D) / q
    K = math.exp(-a * b / p * np.sum((A - B) ** 2)) * math.exp(-c * d / q * np.sum((C - D) ** 2))
    ref = (_norm_s(a) * _norm_s(b) * _norm_s(c) * _norm_s(d) * K * 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q))
           * _f0(p * q / (p + q) * float(np.sum((P - Q) ** 2))))
    assert E[0, 1, 2, 3] == pytest.approx(ref, rel=1e-14)


def _reorder(basis, order):
    """The basis with its shells in `order`, and the function permutation that maps the new index to the old."""
    l, npr = basis["l"], basis["nprim"]
    poff = np.concatenate([[0], np.cumsum(npr)])
    foff = np.concatenate([[0], np.cumsum(2 * l + 1)])
    ex, co, fidx = [], [], []
    for s in order:
        ex.extend(basis["exps"][poff[s]:poff[s + 1]])
        co.extend(basis["coefs"][poff[s]:poff[s + 1]])
        fidx.extend(range(foff[s], foff[s + 1]))
    b2 = W.make_basis(l[order], npr[order], ex, co, basis["xyz"][order])
    return b2, np.array(fidx)


def test_eri_shell_order_covariance():
    """Reversing the shell order makes the oracle compute each quartet with its indices exchanged
    (b a | d c), (c d | a b), ...; the tensors must agree after relabelling.  A sign or index slip in the
    Hermite coefficients of either pair, or in the (-1)^{t'+u'+v'} of the ket, breaks this."""
    basis = W.random_basis(71, 5, 3, max_prim=2, box=2.5, n_sites=5)
    E = oracle.eri(basis, threads=4)
    b2, f = _reorder(basis, np.arange(len(basis["l"]))[::-1].copy())
    E2 = oracle.eri(b2, threads=4)
    assert np.allclose(E2, E[np.ix_(f, f, f, f)], rtol=1e-12, atol=1e-13)


def test_eri_tight_ket_is_the_point_charge_potential():
    """A ket of two s primitives on C with total exponent eta -> infinity is a point charge
    Q = N_g N_d (pi/eta)^{3/2} at C: (ab|cd) -> Q <a|1/|r - C||b>, with a relative error of order
    rho_ab(C) pi / eta / V (here below 1e-6)."""
    basis = W.random_basis(72, 4, 3, max_prim=2, box=2.0, n_sites=4)
    C = np.array([0.8, 1.1, 0.6])
    g, d = 4.0e7, 6.0e7
    nb = oracle.nbf(basis)
    big = W.make_basis(list(basis["l"]) + [0, 0], list(basis["nprim"]) + [1, 1],
                       list(basis["exps"]) + [g, d], list(basis["coefs"]) + [1.0, 1.0],
                       np.vstack([basis["xyz"], C, C]))
    E = oracle.eri(big, threads=4)
    eta = g + d
    Q = _norm_s(g) * _norm_s(d) * (math.pi / eta) ** 1.5
    V = oracle.nuclear_attraction(basis, C[None, :], np.ones(1))
    got = E[:nb, :nb, nb, nb + 1]
    assert np.allclose(got, Q * V, rtol=2e-6, atol=2e-6 * Q * np.max(np.abs(V)))


def test_eri_far_field_is_the_product_of_overlaps_over_the_distance():
    """Bra and ket 5e4 bohr apart: (ab|cd) = S_ab S_cd / R + O(multipoles / R^2)."""
    bra = W.random_basis(73, 3, 2, max_prim=2, box=1.5, n_sites=3)
    ket = W.random_basis(74, 3, 2, max_prim=2, box=1.5, n_sites=3)
    Rv = np.array([3.0e4, -2.0e4, 3.0e4])
    R = float(np.linalg.norm(Rv))
    both = W.make_basis(list(bra["l"]) + list(ket["l"]), list(bra["nprim"]) + list(ket["nprim"]),
                        list(bra["exps"]) + list(ket["exps"]), list(bra["coefs"]) + list(ket["coefs"]),
                        np.vstack([bra["xyz"], ket["xyz"] + Rv]))
    E = oracle.eri(both, threads=4, precision="ld")
    n1 = oracle.nbf(bra)
    S1, S2 = oracle.overlap(bra, precision="ld"), oracle.overlap(ket, precision="ld")
    ref = np.einsum("ab,cd->abcd", S1, S2) / R
    assert np.allclose(E[:n1, :n1, n1:, n1:], ref, rtol=0, atol=1e-3 / R)
    assert np.max(np.abs(ref)) > 0.5 / R


def test_eri_same_centre_s_partner_reduces_to_two_centre():
    """With s primitives of exponent e, f sitting on the centres of a and b, phi_a phi_s is an la function of
    exponent alpha + e up to normalisation, so (a s | b s') = N_e N_f N(la, alpha) / N(la, alpha + e)
    N(lb, beta) / N(lb, beta + f) (a' | b') with the two-centre integrals of the shifted exponents."""
    la, lb, al, be, e, f = 3, 2, 0.8, 1.3, 0.45, 2.2
    A, B = np.array([0.1, -0.3, 0.2]), np.array([1.2, 0.7, -0.9])
    basis = W.make_basis([la, 0, lb, 0], [1] * 4, [al, e, be, f], [1.0] * 4, [A, A, B, B])
    E = oracle.eri(basis, precision="ld")
    shifted = W.make_basis([la, lb], [1, 1], [al + e, be + f], [1.0, 1.0], [A, B])
    J = oracle.coulomb_2c(shifted, precision="ld")
    na = 2 * la + 1
    scale = (_norm_s(e) * _norm_s(f) * oracle.prim_norm(la, al) / oracle.prim_norm(la, al + e)
             * oracle.prim_norm(lb, be) / oracle.prim_norm(lb, be + f))
    got = E[:na, na, na + 1:na + 1 + 2 * lb + 1, na + 1 + 2 * lb + 1]
    assert np.allclose(got, scale * J[:na, na:], rtol=1e-12, atol=1e-14)


def test_eri_rotation_covariance():
    """(ab|cd) of the rotated molecule is the original contracted with the real Wigner blocks of all four shells."""
    basis = W.random_basis(75, 4, 2, max_prim=2, box=2.0, n_sites=4)
    R = RM.rotation_matrix(5)
    E = oracle.eri(basis, threads=4)
    b2 = dict(basis)
    b2["xyz"] = basis["xyz"] @ R.T
    E2 = oracle.eri(b2, threads=4)
    n = oracle.nbf(basis)
    D = np.zeros((n, n))
    off = np.concatenate([[0], np.cumsum(2 * basis["l"] + 1)])
    for s, l in enumerate(basis["l"]):
        D[off[s]:off[s + 1], off[s]:off[s + 1]] = RM.wigner_real(int(l), R)
    rot = np.einsum("ia,jb,kc,ld,abcd->ijkl", D, D, D, D, E, optimize=True)
    assert np.allclose(rot, E2, rtol=0, atol=1e-11 * np.max(np.abs(E)))


def test_eri_coulomb_metric_is_positive_semidefinite():
    """(ab|cd) as a matrix over orbital pairs (ab), (cd) is symmetric and positive semi-definite."""
    basis = W.random_basis(76, 5, 2, max_prim=2, box=2.5, n_sites=5)
    E = oracle.eri(basis, threads=4)
    n = oracle.nbf(basis)
    M = E.reshape(n * n, n * n)
    assert np.allclose(M, M.T, rtol=0, atol=1e-14 * np.max(np.abs(M)))
    ev = np.linalg.eigvalsh(M)
    assert ev.min() > -1e-12 * ev.max()


@pytest.mark.parametrize("ls", [(4, 3, 4, 2), (3, 3, 3, 3)])
def test_eri_double_oracle_certified_by_extended_precision(ls):
    """The double build against the long-double build on one high-l quartet."""
    rng = np.random.default_rng(sum(ls))
    basis = W.make_basis(list(ls), [2] * 4, np.exp(rng.uniform(np.log(0.2), np.log(20.0), 8)),
                         rng.uniform(0.2, 1.0, 8), rng.uniform(0.0, 3.0, (4, 3)))
    E = oracle.eri(basis)
    El = oracle.eri(basis, precision="ld")
    assert np.max(np.abs(E - El)) < 1e-13 + 1e-12 * np.max(np.abs(El))
