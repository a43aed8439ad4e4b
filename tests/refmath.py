"""Independent helpers for the tests: solid harmonics from scipy's spherical harmonics, numerical
Wigner-D fits and brute-force quadrature.  Nothing here comes from the oracle or the library."""
import numpy as np
import scipy.special as sp
from scipy import integrate


def solid_harmonics_scipy(l, xyz):
    """Real Racah-normalised solid harmonics S_lm, m = -l..l (Eq. 2 with Condon-Shortley phase;
    S_l0 = Y_l^0, S_{l,m>0} = (-1)^m sqrt2 Re, S_{l,-m} = (-1)^m sqrt2 Im), from scipy.special."""
    xyz = np.atleast_2d(np.asarray(xyz, dtype=np.float64))
    r = np.linalg.norm(xyz, axis=1)
    safe = np.where(r > 0, r, 1.0)
    th = np.arccos(np.clip(xyz[:, 2] / safe, -1.0, 1.0))
    ph = np.arctan2(xyz[:, 1], xyz[:, 0])
    out = np.zeros((xyz.shape[0], 2 * l + 1))
    fac = np.sqrt(4 * np.pi / (2 * l + 1)) * r ** l
    for m in range(-l, l + 1):
        am = abs(m)
        Y = sp.sph_harm_y(l, am, th, ph)
        if m == 0:
            v = Y.real
        elif m > 0:
            v = (-1) ** am * np.sqrt(2) * Y.real
        else:
            v = (-1) ** am * np.sqrt(2) * Y.imag
        out[:, m + l] = fac * v
    if l == 0:
        out[:, 0] = 1.0
    return out


def rotation_matrix(seed):
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def wigner_real(l, R, seed=0):
    """D with S_lm(R x) = sum_m' D[m, m'] S_lm'(x), fitted by least squares at random points."""
    rng = np.random.default_rng(seed + 17 * l)
    x = rng.normal(size=(8 * (2 * l + 1) + 16, 3))
    S = solid_harmonics_scipy(l, x)
    SR = solid_harmonics_scipy(l, x @ R.T)
    D, *_ = np.linalg.lstsq(S, SR, rcond=None)
    return D.T


def radial_norm(l, alpha):
    """N(l, alpha) with int (N S_lm e^{-alpha r^2})^2 d^3r = 1, by 1-D quadrature of
    4 pi/(2l+1) int r^{2l+2} e^{-2 alpha r^2} dr (the angular integral of S_lm^2 is 4 pi/(2l+1))."""
    val, _ = integrate.quad(lambda r: r ** (2 * l + 2) * np.exp(-2 * alpha * r * r), 0, np.inf,
                            epsabs=0, epsrel=2e-14, limit=200)
    return 1.0 / np.sqrt(4 * np.pi / (2 * l + 1) * val)


def gauss_legendre(n, a, b):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def shell_values(basis, s, pts, norms):
    """Values of the 2l+1 functions of shell s at pts (n x 3): sum_i c_i N_i S_lm(r-A) e^{-a_i|r-A|^2},
    times the contracted scale norms[s]."""
    off = int(np.sum(basis["nprim"][:s]))
    k = int(basis["nprim"][s])
    l = int(basis["l"][s])
    A = basis["xyz"][s]
    d = pts - A
    r2 = np.sum(d * d, axis=1)
    radial = np.zeros(len(pts))
    for i in range(k):
        a = basis["exps"][off + i]
        radial += basis["coefs"][off + i] * radial_norm(l, a) * np.exp(-a * r2)
    return solid_harmonics_scipy(l, d) * radial[:, None] * norms[s]


def sphere_grid(n_rho, rho_max, n_theta, n_phi, centre):
    """Product grid about `centre`: Gauss-Legendre in rho (4 panels) and cos(theta), trapezoid in phi.
    Returns points and weights for int f d^3r / |r - centre| (the r^2 of the volume element
    cancels one power against 1/r, leaving rho)."""
    edges = np.array([0.0, 0.15, 0.4, 0.7, 1.0]) * rho_max
    rho, wr = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        x, w = gauss_legendre(n_rho, a, b)
        rho.append(x)
        wr.append(w)
    rho = np.concatenate(rho)
    wr = np.concatenate(wr)
    ct, wt = gauss_legendre(n_theta, -1.0, 1.0)
    ph = np.arange(n_phi) * (2 * np.pi / n_phi)
    wp = np.full(n_phi, 2 * np.pi / n_phi)
    R, CT, PH = np.meshgrid(rho, ct, ph, indexing="ij")
    st = np.sqrt(1 - CT ** 2)
    pts = np.stack([R * st * np.cos(PH), R * st * np.sin(PH), R * CT], axis=-1).reshape(-1, 3) + centre
    w = (wr[:, None, None] * wt[None, :, None] * wp[None, None, :] * R).reshape(-1)
    return pts, w
