/*
 * Plain CPU oracle for nuclear-attraction integrals over contracted real solid-harmonic
 * Gaussian orbitals (SHGOs).  TEST INFRASTRUCTURE ONLY: it is called by the tests, by the
 * smoke check and by the CPU-baseline leg of the benchmark, never by the library.
 *
 * It deliberately does NOT follow the paper's SHGO route.  It evaluates the plain definition
 *
 *     V_ab = sum_C Z_C < phi_a | 1/|r - C| | phi_b >                         (operator of Eq. 11)
 *
 * over the orbitals of Eq. 1 by the Cartesian route that the paper lists as its comparison
 * (Table 1, first column): Boys function -> Hermite Coulomb integrals -> Hermite expansion
 * coefficients -> Cartesian integrals -> primitive contraction -> solid harmonics.  The
 * Cartesian integrals follow McMurchie and Davidson (J. Comput. Phys. 26, 218 (1978)), in the
 * notation of Helgaker, Jorgensen and Olsen, "Molecular Electronic-Structure Theory", ch. 9.
 *
 * Conventions (readings of the paper, all stated in the design notes):
 *  - Solid harmonics are Racah-normalised, Condon-Shortley phase (Eq. 2); the output uses the
 *    real combination S_l0 = Y_l^0, S_{l,m>0} = (-1)^m sqrt2 Re Y_l^m,
 *    S_{l,-m} = (-1)^m sqrt2 Im Y_l^m, so S_11 = x, S_1,-1 = y, S_10 = z.
 *  - N(l, alpha) of Eq. 1 normalises each primitive; the contracted function is then
 *    renormalised to <phi|phi> = 1, using this file's own Cartesian overlap integrals.
 *  - V carries no minus sign.  Functions are ordered shell by shell, m = -l..l.
 *  - The same file holds the overlap (Eq. 10), the field integrals, and the two- and four-centre
 *    electron-repulsion integrals (Eqs. 13-15), each by the same Cartesian route.
 *
 * The scalar type is `real`: double by default, long double when compiled with
 * -DORACLE_LONG_DOUBLE (80-bit on x86-64, IEEE binary128 on aarch64).  All public entry
 * points take and return double.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifdef ORACLE_LONG_DOUBLE
typedef long double real;
#define RX(f) f##l
#define RPI 3.141592653589793238462643383279502884L
#else
typedef double real;
#define RX(f) f
#define RPI 3.141592653589793238462643383279502884
#endif

#define ORACLE_LMAX 10 /* largest shell l accepted (the library's limit is 8) */

/* ------------------------------------------------------------------------------------------ */
/* Boys function  F_n(T) = int_0^1 u^{2n} exp(-T u^2) du   (the third factor after Eq. 12).   */
/*                                                                                            */
/* T below the switch: the convergent series                                                  */
/*     F_n(T) = exp(-T) sum_{i>=0} (2T)^i / [(2n+1)(2n+3)...(2n+2i+1)]                        */
/* evaluated for n = nmax, then the downward recursion F_n = (2T F_{n+1} + exp(-T))/(2n+1).   */
/* T at or above it: F_0 = sqrt(pi/T) erf(sqrt T)/2 and the upward recursion                  */
/*     F_{n+1} = ((2n+1) F_n - exp(-T)) / (2T),                                               */
/* which loses nothing while 2n+1 < 2T.                                                        */
/* ------------------------------------------------------------------------------------------ */
static void boys_r(int nmax, real T, real* F) {
  const real ex = RX(exp)(-T);
  const real tsw = (real)(2 * nmax + 40);
  if (T < tsw) {
    real term = (real)1 / (real)(2 * nmax + 1);
    real sum = term;
    for (int i = 1; i < 100000; ++i) {
      term *= (2 * T) / (real)(2 * nmax + 2 * i + 1);
      sum += term;
      if (term < sum * (real)1e-40) break;
    }
    F[nmax] = ex * sum;
    for (int n = nmax - 1; n >= 0; --n) F[n] = (2 * T * F[n + 1] + ex) / (real)(2 * n + 1);
  } else {
    const real st = RX(sqrt)(T);
    F[0] = RX(sqrt)(RPI) * RX(erf)(st) / (2 * st);
    for (int n = 0; n < nmax; ++n) F[n + 1] = ((real)(2 * n + 1) * F[n] - ex) / (2 * T);
  }
}

void oracle_boys(int nmax, double T, double* F) {
  real Fr[64];
  if (nmax < 0 || nmax > 60) return;
  boys_r(nmax, (real)T, Fr);
  for (int n = 0; n <= nmax; ++n) F[n] = (double)Fr[n];
}

/* ------------------------------------------------------------------------------------------ */
/* Cartesian components of degree l, ordered i = l..0, j = l-i..0, k = l-i-j (x^i y^j z^k).   */
/* ------------------------------------------------------------------------------------------ */
static int ncart(int l) { return (l + 1) * (l + 2) / 2; }

static int cart_index(int l, int i, int j) {
  /* position of (i, j, l-i-j) in the order above */
  int idx = 0;
  for (int ii = l; ii > i; --ii) idx += l - ii + 1;
  return idx + (l - i - j);
}

static real factorial_r(int n) {
  real f = 1;
  for (int i = 2; i <= n; ++i) f *= (real)i;
  return f;
}

static real binom_r(int n, int k) {
  if (k < 0 || k > n) return 0;
  return factorial_r(n) / (factorial_r(k) * factorial_r(n - k));
}

/*
 * Cartesian expansion of the real Racah-normalised solid harmonic S_lm (Eq. 2 with the real
 * combination above).  Written out from the textbook closed form
 *     S_{l,|m|}  = sqrt((2 - d_m0) (l-|m|)!/(l+|m|)!) Pi_l^|m|(z, r) Re (x + i y)^|m|
 *     S_{l,-|m|} = sqrt( 2        (l-|m|)!/(l+|m|)!) Pi_l^|m|(z, r) Im (x + i y)^|m|
 *     Pi_l^m(z, r) = sum_k (-1)^k 2^-l C(l,k) C(2l-2k,l) (l-2k)!/(l-2k-m)! r^{2k} z^{l-2k-m}
 * with r^{2k} = (x^2 + y^2 + z^2)^k expanded by the multinomial theorem.
 * coef[(m + l) * ncart(l) + c] multiplies Cartesian component c.
 */
static void solid_harmonic_cart(int l, real* coef) {
  const int nc = ncart(l);
  memset(coef, 0, sizeof(real) * (size_t)(2 * l + 1) * nc);
  for (int m = -l; m <= l; ++m) {
    const int am = m < 0 ? -m : m;
    const real norm = RX(sqrt)((m == 0 ? (real)1 : (real)2) * factorial_r(l - am) / factorial_r(l + am));
    real* row = coef + (size_t)(m + l) * nc;
    for (int k = 0; 2 * k <= l - am; ++k) {
      const real pik = ((k & 1) ? -1 : 1) * RX(pow)((real)2, (real)(-l)) * binom_r(l, k) *
                       binom_r(2 * l - 2 * k, l) * factorial_r(l - 2 * k) / factorial_r(l - 2 * k - am);
      /* (x + i y)^am: term C(am, q) x^{am-q} (i y)^q; real part for q even, imaginary for q odd */
      for (int q = 0; q <= am; ++q) {
        real xy;
        if (m >= 0) {
          if (q & 1) continue;
          xy = binom_r(am, q) * ((q / 2) & 1 ? -1 : 1);
        } else {
          if (!(q & 1)) continue;
          xy = binom_r(am, q) * (((q - 1) / 2) & 1 ? -1 : 1);
        }
        /* multinomial expansion of (x^2+y^2+z^2)^k */
        for (int a = 0; a <= k; ++a)
          for (int b = 0; a + b <= k; ++b) {
            const int c = k - a - b;
            const real mult = factorial_r(k) / (factorial_r(a) * factorial_r(b) * factorial_r(c));
            const int px = am - q + 2 * a, py = q + 2 * b;
            row[cart_index(l, px, py)] += norm * pik * xy * mult;
          }
      }
    }
  }
}

int oracle_solid_harmonic_cart(int l, double* coef) {
  if (l < 0 || l > ORACLE_LMAX) return -1;
  const int n = (2 * l + 1) * ncart(l);
  real* c = (real*)malloc(sizeof(real) * (size_t)n);
  if (!c) return -2;
  solid_harmonic_cart(l, c);
  for (int i = 0; i < n; ++i) coef[i] = (double)c[i];
  free(c);
  return 0;
}

/* Evaluate S_lm at npts points from the Cartesian expansion above: out[p * (2l+1) + m + l]. */
int oracle_solid_harmonic(int l, long npts, const double* xyz, double* out) {
  if (l < 0 || l > ORACLE_LMAX) return -1;
  const int nc = ncart(l);
  real* c = (real*)malloc(sizeof(real) * (size_t)(2 * l + 1) * nc);
  if (!c) return -2;
  solid_harmonic_cart(l, c);
  for (long p = 0; p < npts; ++p) {
    const real x = xyz[3 * p], y = xyz[3 * p + 1], z = xyz[3 * p + 2];
    for (int m = 0; m < 2 * l + 1; ++m) {
      real s = 0;
      for (int i = l; i >= 0; --i)
        for (int j = l - i; j >= 0; --j) {
          const int k = l - i - j;
          s += c[(size_t)m * nc + cart_index(l, i, j)] * RX(pow)(x, (real)i) * RX(pow)(y, (real)j) *
               RX(pow)(z, (real)k);
        }
      out[p * (2 * l + 1) + m] = (double)s;
    }
  }
  free(c);
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* McMurchie-Davidson building blocks.                                                       */
/* ------------------------------------------------------------------------------------------ */

/* Hermite expansion coefficients of one Cartesian direction:
 *   E^{00}_0 = exp(-mu X_AB^2)
 *   E^{i+1,j}_t = E^{ij}_{t-1}/(2p) + X_PA E^{ij}_t + (t+1) E^{ij}_{t+1}
 *   E^{i,j+1}_t = E^{ij}_{t-1}/(2p) + X_PB E^{ij}_t + (t+1) E^{ij}_{t+1}
 * Stored E[(i * (jmax+1) + j) * (tdim) + t], tdim = imax + jmax + 1. */
static void hermite_E(int imax, int jmax, real p, real XPA, real XPB, real E00, real* E) {
  const int tdim = imax + jmax + 1;
#define EIDX(i, j, t) (((i) * (jmax + 1) + (j)) * tdim + (t))
  memset(E, 0, sizeof(real) * (size_t)(imax + 1) * (jmax + 1) * tdim);
  E[EIDX(0, 0, 0)] = E00;
  const real h = (real)1 / (2 * p);
  for (int i = 0; i <= imax; ++i) {
    if (i > 0) {
      for (int t = 0; t <= i; ++t) {
        real v = XPA * E[EIDX(i - 1, 0, t)];
        if (t > 0) v += h * E[EIDX(i - 1, 0, t - 1)];
        if (t + 1 <= i - 1) v += (real)(t + 1) * E[EIDX(i - 1, 0, t + 1)];
        E[EIDX(i, 0, t)] = v;
      }
    }
    for (int j = 1; j <= jmax; ++j) {
      for (int t = 0; t <= i + j; ++t) {
        real v = 0;
        if (t <= i + j - 1) v += XPB * E[EIDX(i, j - 1, t)];
        if (t > 0) v += h * E[EIDX(i, j - 1, t - 1)];
        if (t + 1 <= i + j - 1) v += (real)(t + 1) * E[EIDX(i, j - 1, t + 1)];
        E[EIDX(i, j, t)] = v;
      }
    }
  }
#undef EIDX
}

/* Hermite Coulomb integrals R^0_{tuv}(p, P - C) for t + u + v <= L:
 *   R^n_{000} = (-2p)^n F_n(p |PC|^2)
 *   R^n_{t+1,u,v} = t R^{n+1}_{t-1,u,v} + X_PC R^{n+1}_{t,u,v}   (and likewise in y, z)
 * work holds (L+1)^4 reals; out[(t * (L+1) + u) * (L+1) + v] receives R^0_{tuv}. */
static void hermite_R(int L, real p, real XPC, real YPC, real ZPC, real* work, real* out) {
  const int d = L + 1;
#define RIDX(n, t, u, v) ((((n) * d + (t)) * d + (u)) * d + (v))
  real F[80];
  boys_r(L, p * (XPC * XPC + YPC * YPC + ZPC * ZPC), F);
  real m2p = 1;
  for (int n = 0; n <= L; ++n) {
    work[RIDX(n, 0, 0, 0)] = m2p * F[n];
    m2p *= -2 * p;
  }
  for (int n = L - 1; n >= 0; --n) {
    for (int s = 1; s <= L - n; ++s)
      for (int t = s; t >= 0; --t)
        for (int u = s - t; u >= 0; --u) {
          const int v = s - t - u;
          real r;
          if (t > 0) {
            r = XPC * work[RIDX(n + 1, t - 1, u, v)];
            if (t > 1) r += (real)(t - 1) * work[RIDX(n + 1, t - 2, u, v)];
          } else if (u > 0) {
            r = YPC * work[RIDX(n + 1, t, u - 1, v)];
            if (u > 1) r += (real)(u - 1) * work[RIDX(n + 1, t, u - 2, v)];
          } else {
            r = ZPC * work[RIDX(n + 1, t, u, v - 1)];
            if (v > 1) r += (real)(v - 1) * work[RIDX(n + 1, t, u, v - 2)];
          }
          work[RIDX(n, t, u, v)] = r;
        }
  }
  for (int t = 0; t <= L; ++t)
    for (int u = 0; u + t <= L; ++u)
      for (int v = 0; v + u + t <= L; ++v) out[(t * d + u) * d + v] = work[RIDX(0, t, u, v)];
#undef RIDX
}

/* ------------------------------------------------------------------------------------------ */
/* Basis handling.                                                                            */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  int l, nprim;
  const double* alpha;
  real coef[64]; /* contraction coefficient x primitive normalisation x contracted renormalisation */
  real A[3];
} shell_t;

/* N(l, alpha)^-2 = pi^{3/2} (2l-1)!! / (2^l (2 alpha)^{l + 3/2})   (normalisation of Eq. 1) */
static real prim_norm(int l, real a) {
  real dfact = 1;
  for (int k = 2 * l - 1; k > 1; k -= 2) dfact *= (real)k;
  const real n2 = RX(pow)(RPI, (real)1.5) * dfact / (RX(pow)((real)2, (real)l) * RX(pow)(2 * a, (real)l + (real)1.5));
  return 1 / RX(sqrt)(n2);
}

/* Cartesian overlap block of two contracted shells, transformed to real solid harmonics:
 * out[ma * (2lb+1) + mb].  (pi/p)^{3/2} E^{ij}_0 E^{kl}_0 E^{mn}_0 per primitive pair. */
static void overlap_block(const shell_t* a, const shell_t* b, const real* ca, const real* cb, real* out) {
  const int la = a->l, lb = b->l, nca = ncart(la), ncb = ncart(lb);
  const int tdim = la + lb + 1;
  real* Ex = (real*)malloc(sizeof(real) * 3 * (size_t)(la + 1) * (lb + 1) * tdim);
  real* Ey = Ex + (size_t)(la + 1) * (lb + 1) * tdim;
  real* Ez = Ey + (size_t)(la + 1) * (lb + 1) * tdim;
  real* Sc = (real*)calloc((size_t)nca * ncb, sizeof(real));
  for (int i = 0; i < a->nprim; ++i)
    for (int j = 0; j < b->nprim; ++j) {
      const real al = a->alpha[i], be = b->alpha[j], p = al + be, mu = al * be / p;
      real P[3], E00[3];
      for (int c = 0; c < 3; ++c) {
        P[c] = (al * a->A[c] + be * b->A[c]) / p;
        const real X = a->A[c] - b->A[c];
        E00[c] = RX(exp)(-mu * X * X);
      }
      hermite_E(la, lb, p, P[0] - a->A[0], P[0] - b->A[0], E00[0], Ex);
      hermite_E(la, lb, p, P[1] - a->A[1], P[1] - b->A[1], E00[1], Ey);
      hermite_E(la, lb, p, P[2] - a->A[2], P[2] - b->A[2], E00[2], Ez);
      const real pre = a->coef[i] * b->coef[j] * RX(pow)(RPI / p, (real)1.5);
      for (int ix = la; ix >= 0; --ix)
        for (int iy = la - ix; iy >= 0; --iy) {
          const int iz = la - ix - iy, ia = cart_index(la, ix, iy);
          for (int jx = lb; jx >= 0; --jx)
            for (int jy = lb - jx; jy >= 0; --jy) {
              const int jz = lb - jx - jy, ib = cart_index(lb, jx, jy);
              Sc[ia * ncb + ib] += pre * Ex[(ix * (lb + 1) + jx) * tdim] * Ey[(iy * (lb + 1) + jy) * tdim] *
                                   Ez[(iz * (lb + 1) + jz) * tdim];
            }
        }
    }
  for (int ma = 0; ma < 2 * la + 1; ++ma)
    for (int mb = 0; mb < 2 * lb + 1; ++mb) {
      real s = 0;
      for (int ia = 0; ia < nca; ++ia)
        for (int ib = 0; ib < ncb; ++ib) s += ca[ma * nca + ia] * cb[mb * ncb + ib] * Sc[ia * ncb + ib];
      out[ma * (2 * lb + 1) + mb] = s;
    }
  free(Sc);
  free(Ex);
}

/* Fill the shells: coef = c_i N(l, alpha_i) / sqrt(<phi|phi>), the self-overlap taken from
 * overlap_block (the m = -l diagonal element; all 2l+1 agree). */
static int setup_shells(int n_shells, const int* l, const int* nprim, const double* exps, const double* coefs,
                        const double* xyz, shell_t* sh, real** cart) {
  long off = 0;
  for (int s = 0; s < n_shells; ++s) {
    if (l[s] < 0 || l[s] > ORACLE_LMAX || nprim[s] < 1 || nprim[s] > 64) return -1;
    sh[s].l = l[s];
    sh[s].nprim = nprim[s];
    sh[s].alpha = exps + off;
    for (int c = 0; c < 3; ++c) sh[s].A[c] = xyz[3 * s + c];
    for (int i = 0; i < nprim[s]; ++i) sh[s].coef[i] = (real)coefs[off + i] * prim_norm(l[s], exps[off + i]);
    off += nprim[s];
  }
  for (int s = 0; s < n_shells; ++s) {
    const int ll = sh[s].l, nb = 2 * ll + 1;
    real* blk = (real*)malloc(sizeof(real) * (size_t)nb * nb);
    overlap_block(&sh[s], &sh[s], cart[ll], cart[ll], blk);
    const real scale = 1 / RX(sqrt)(blk[0]);
    for (int i = 0; i < sh[s].nprim; ++i) sh[s].coef[i] *= scale;
    free(blk);
  }
  return 0;
}

/* Nuclear-attraction block of one shell pair: out[ma * (2lb+1) + mb] =
 *   sum_C Z_C <a, ma | 1/|r-C| | b, mb>.
 * Per primitive pair: R^0_tuv is summed over nuclei weighted by Z_C (the operator of Eq. 11 is
 * the sum of the nuclear potentials), then contracted with E^x_t E^y_u E^z_v and (2 pi / p). */
/* dcomp < 0: the block of sum_C Z_C <a|1/|r-C||b>.  dcomp = 0, 1, 2: its derivative with respect to the
 * x, y or z coordinate of the nuclei, sum_C Z_C d/dC_c <a|1/|r-C||b>: R_tuv depends on C through P - C,
 * and d/dC_x R_tuv(P - C) = -R_{t+1,u,v}, so the same sum runs over the shifted R table. */
static void nuclear_block(const shell_t* a, const shell_t* b, const real* ca, const real* cb, long nC,
                          const double* C, const double* Z, real* out, int dcomp) {
  const int la = a->l, lb = b->l, L = la + lb, nca = ncart(la), ncb = ncart(lb);
  const int Lr = dcomp >= 0 ? L + 1 : L;  /* order of the R table */
  const int tdim = L + 1, d = Lr + 1;
  real* Ex = (real*)malloc(sizeof(real) * 3 * (size_t)(la + 1) * (lb + 1) * tdim);
  real* Ey = Ex + (size_t)(la + 1) * (lb + 1) * tdim;
  real* Ez = Ey + (size_t)(la + 1) * (lb + 1) * tdim;
  real* work = (real*)malloc(sizeof(real) * (size_t)d * d * d * d);
  real* Rc = (real*)malloc(sizeof(real) * (size_t)d * d * d);
  real* Rs = (real*)malloc(sizeof(real) * (size_t)d * d * d);
  real* Vc = (real*)calloc((size_t)nca * ncb, sizeof(real));
  for (int i = 0; i < a->nprim; ++i)
    for (int j = 0; j < b->nprim; ++j) {
      const real al = a->alpha[i], be = b->alpha[j], p = al + be, mu = al * be / p;
      real P[3], E00[3];
      for (int c = 0; c < 3; ++c) {
        P[c] = (al * a->A[c] + be * b->A[c]) / p;
        const real X = a->A[c] - b->A[c];
        E00[c] = RX(exp)(-mu * X * X);
      }
      hermite_E(la, lb, p, P[0] - a->A[0], P[0] - b->A[0], E00[0], Ex);
      hermite_E(la, lb, p, P[1] - a->A[1], P[1] - b->A[1], E00[1], Ey);
      hermite_E(la, lb, p, P[2] - a->A[2], P[2] - b->A[2], E00[2], Ez);
      memset(Rs, 0, sizeof(real) * (size_t)d * d * d);
      for (long c = 0; c < nC; ++c) {
        hermite_R(Lr, p, P[0] - (real)C[3 * c], P[1] - (real)C[3 * c + 1], P[2] - (real)C[3 * c + 2], work, Rc);
        for (int t = 0; t <= Lr; ++t)
          for (int u = 0; u + t <= Lr; ++u)
            for (int v = 0; v + u + t <= Lr; ++v) Rs[(t * d + u) * d + v] += (real)Z[c] * Rc[(t * d + u) * d + v];
      }
      const real pre = a->coef[i] * b->coef[j] * 2 * RPI / p;
      for (int ix = la; ix >= 0; --ix)
        for (int iy = la - ix; iy >= 0; --iy) {
          const int iz = la - ix - iy, ia = cart_index(la, ix, iy);
          for (int jx = lb; jx >= 0; --jx)
            for (int jy = lb - jx; jy >= 0; --jy) {
              const int jz = lb - jx - jy, ib = cart_index(lb, jx, jy);
              const real* ex = Ex + (ix * (lb + 1) + jx) * tdim;
              const real* ey = Ey + (iy * (lb + 1) + jy) * tdim;
              const real* ez = Ez + (iz * (lb + 1) + jz) * tdim;
              const int dt = dcomp == 0, du = dcomp == 1, dv = dcomp == 2;
              real s = 0;
              for (int t = 0; t <= ix + jx; ++t)
                for (int u = 0; u <= iy + jy; ++u)
                  for (int v = 0; v <= iz + jz; ++v)
                    s += ex[t] * ey[u] * ez[v] * Rs[((t + dt) * d + u + du) * d + v + dv];
              Vc[ia * ncb + ib] += (dcomp >= 0 ? -pre : pre) * s;
            }
        }
    }
  for (int ma = 0; ma < 2 * la + 1; ++ma)
    for (int mb = 0; mb < 2 * lb + 1; ++mb) {
      real s = 0;
      for (int ia = 0; ia < nca; ++ia)
        for (int ib = 0; ib < ncb; ++ib) s += ca[ma * nca + ia] * cb[mb * ncb + ib] * Vc[ia * ncb + ib];
      out[ma * (2 * lb + 1) + mb] = s;
    }
  free(Vc);
  free(Rs);
  free(Rc);
  free(work);
  free(Ex);
}

/* One primitive Cartesian nuclear-attraction integral (without the 2 pi / p prefactor) from the Hermite
 * expansion tables: sum_{t,u,v} E^x_{ix,jx;t} E^y_{iy,jy;u} E^z_{iz,jz;v} R_{tuv}, the E tables laid out
 * as hermite_E writes them (ket extent lb + 1, t extent tdim) and R as hermite_R writes it (extent d). */
static real hermite_cart(const real* Ex, const real* Ey, const real* Ez, int lb, int tdim, const real* R, int d,
                         int ix, int iy, int iz, int jx, int jy, int jz) {
  const real* ex = Ex + (ix * (lb + 1) + jx) * tdim;
  const real* ey = Ey + (iy * (lb + 1) + jy) * tdim;
  const real* ez = Ez + (iz * (lb + 1) + jz) * tdim;
  real s = 0;
  for (int t = 0; t <= ix + jx; ++t)
    for (int u = 0; u <= iy + jy; ++u)
      for (int v = 0; v <= iz + jz; ++v) s += ex[t] * ey[u] * ez[v] * R[(t * d + u) * d + v];
  return s;
}

/* Derivative of the nuclear-attraction block with respect to coordinate `comp` of the bra shell's centre
 * A (the ket's centre and the nuclei fixed): out[ma * (2lb+1) + mb] = d/dA_comp sum_C Z_C <a, ma|1/|r-C||b, mb>.
 * A Cartesian primitive x_A^i y_A^j z_A^k exp(-alpha r_A^2) has d/dA_x = 2 alpha x_A^{i+1} ... - i x_A^{i-1} ...,
 * so each Cartesian element is 2 alpha times the integral with the exponent of the differentiated
 * coordinate raised by one, minus that exponent times the integral with it lowered by one; the Hermite
 * tables run to la + 1 on the bra side and to order la + lb + 1 in R. */
static void nuclear_dA_block(const shell_t* a, const shell_t* b, const real* ca, const real* cb, long nC,
                             const double* C, const double* Z, real* out, int comp) {
  const int la = a->l, lb = b->l, nca = ncart(la), ncb = ncart(lb);
  const int ia1 = la + 1, L1 = la + lb + 1, tdim = ia1 + lb + 1, d = L1 + 1;
  real* Ex = (real*)malloc(sizeof(real) * 3 * (size_t)(ia1 + 1) * (lb + 1) * tdim);
  real* Ey = Ex + (size_t)(ia1 + 1) * (lb + 1) * tdim;
  real* Ez = Ey + (size_t)(ia1 + 1) * (lb + 1) * tdim;
  real* work = (real*)malloc(sizeof(real) * (size_t)d * d * d * d);
  real* Rc = (real*)malloc(sizeof(real) * (size_t)d * d * d);
  real* Rs = (real*)malloc(sizeof(real) * (size_t)d * d * d);
  real* Vc = (real*)calloc((size_t)nca * ncb, sizeof(real));
  for (int i = 0; i < a->nprim; ++i)
    for (int j = 0; j < b->nprim; ++j) {
      const real al = a->alpha[i], be = b->alpha[j], p = al + be, mu = al * be / p;
      real P[3], E00[3];
      for (int c = 0; c < 3; ++c) {
        P[c] = (al * a->A[c] + be * b->A[c]) / p;
        const real X = a->A[c] - b->A[c];
        E00[c] = RX(exp)(-mu * X * X);
      }
      hermite_E(ia1, lb, p, P[0] - a->A[0], P[0] - b->A[0], E00[0], Ex);
      hermite_E(ia1, lb, p, P[1] - a->A[1], P[1] - b->A[1], E00[1], Ey);
      hermite_E(ia1, lb, p, P[2] - a->A[2], P[2] - b->A[2], E00[2], Ez);
      memset(Rs, 0, sizeof(real) * (size_t)d * d * d);
      for (long c = 0; c < nC; ++c) {
        hermite_R(L1, p, P[0] - (real)C[3 * c], P[1] - (real)C[3 * c + 1], P[2] - (real)C[3 * c + 2], work, Rc);
        for (int t = 0; t <= L1; ++t)
          for (int u = 0; u + t <= L1; ++u)
            for (int v = 0; v + u + t <= L1; ++v) Rs[(t * d + u) * d + v] += (real)Z[c] * Rc[(t * d + u) * d + v];
      }
      const real pre = a->coef[i] * b->coef[j] * 2 * RPI / p;
      for (int ix = la; ix >= 0; --ix)
        for (int iy = la - ix; iy >= 0; --iy) {
          const int iz = la - ix - iy, ia = cart_index(la, ix, iy);
          const int e[3] = {ix, iy, iz};
          for (int jx = lb; jx >= 0; --jx)
            for (int jy = lb - jx; jy >= 0; --jy) {
              const int jz = lb - jx - jy, ib = cart_index(lb, jx, jy);
              const int up[3] = {ix + (comp == 0), iy + (comp == 1), iz + (comp == 2)};
              real v = 2 * al * hermite_cart(Ex, Ey, Ez, lb, tdim, Rs, d, up[0], up[1], up[2], jx, jy, jz);
              if (e[comp] > 0) {
                const int dn[3] = {ix - (comp == 0), iy - (comp == 1), iz - (comp == 2)};
                v -= (real)e[comp] * hermite_cart(Ex, Ey, Ez, lb, tdim, Rs, d, dn[0], dn[1], dn[2], jx, jy, jz);
              }
              Vc[ia * ncb + ib] += pre * v;
            }
        }
    }
  for (int ma = 0; ma < 2 * la + 1; ++ma)
    for (int mb = 0; mb < 2 * lb + 1; ++mb) {
      real s = 0;
      for (int ia = 0; ia < nca; ++ia)
        for (int ib = 0; ib < ncb; ++ib) s += ca[ma * nca + ia] * cb[mb * ncb + ib] * Vc[ia * ncb + ib];
      out[ma * (2 * lb + 1) + mb] = s;
    }
  free(Vc);
  free(Rs);
  free(Rc);
  free(work);
  free(Ex);
}

/* Two-centre Coulomb block of one shell pair: out[ma * (2lb+1) + mb] =
 *   (a, ma | b, mb) = int int phi_a(r1) phi_b(r2) / |r1 - r2| d3r1 d3r2.
 * McMurchie-Davidson with each orbital its own one-Gaussian "pair": per primitive pair,
 *   2 pi^{5/2} / (alpha beta sqrt(alpha + beta)) sum_{tuv} E^a_{tuv} sum_{t'u'v'} E^b_{t'u'v'} (-1)^{t'+u'+v'}
 *       R^0_{t+t', u+u', v+v'}(rho, A - B),   rho = alpha beta / (alpha + beta),
 * where the Hermite coefficients of x_A^i exp(-alpha x_A^2) follow from hermite_E with jmax = 0,
 * X_PA = 0 and E^{00}_0 = 1. */
static void coulomb2c_block(const shell_t* a, const shell_t* b, const real* ca, const real* cb, real* out) {
  const int la = a->l, lb = b->l, L = la + lb, nca = ncart(la), ncb = ncart(lb), d = L + 1;
  real* Ea = (real*)malloc(sizeof(real) * 3 * (size_t)(la + 1) * (la + 1));
  real* Eb = (real*)malloc(sizeof(real) * 3 * (size_t)(lb + 1) * (lb + 1));
  real* work = (real*)malloc(sizeof(real) * (size_t)d * d * d * d);
  real* R = (real*)malloc(sizeof(real) * (size_t)d * d * d);
  real* Vc = (real*)calloc((size_t)nca * ncb, sizeof(real));
  for (int i = 0; i < a->nprim; ++i)
    for (int j = 0; j < b->nprim; ++j) {
      const real al = a->alpha[i], be = b->alpha[j], rho = al * be / (al + be);
      for (int c = 0; c < 3; ++c) {
        hermite_E(la, 0, al, 0, 0, 1, Ea + (size_t)c * (la + 1) * (la + 1));
        hermite_E(lb, 0, be, 0, 0, 1, Eb + (size_t)c * (lb + 1) * (lb + 1));
      }
      hermite_R(L, rho, a->A[0] - b->A[0], a->A[1] - b->A[1], a->A[2] - b->A[2], work, R);
      const real pre = a->coef[i] * b->coef[j] * 2 * RX(pow)(RPI, (real)2.5) / (al * be * RX(sqrt)(al + be));
      for (int ix = la; ix >= 0; --ix)
        for (int iy = la - ix; iy >= 0; --iy) {
          const int iz = la - ix - iy, ia = cart_index(la, ix, iy);
          const real* ex = Ea + ix * (la + 1);
          const real* ey = Ea + (size_t)(la + 1) * (la + 1) + iy * (la + 1);
          const real* ez = Ea + (size_t)2 * (la + 1) * (la + 1) + iz * (la + 1);
          for (int jx = lb; jx >= 0; --jx)
            for (int jy = lb - jx; jy >= 0; --jy) {
              const int jz = lb - jx - jy, ib = cart_index(lb, jx, jy);
              const real* fx = Eb + jx * (lb + 1);
              const real* fy = Eb + (size_t)(lb + 1) * (lb + 1) + jy * (lb + 1);
              const real* fz = Eb + (size_t)2 * (lb + 1) * (lb + 1) + jz * (lb + 1);
              real sum = 0;
              for (int t = 0; t <= ix; ++t)
                for (int u = 0; u <= iy; ++u)
                  for (int v = 0; v <= iz; ++v) {
                    const real e = ex[t] * ey[u] * ez[v];
                    if (e == 0) continue;
                    for (int t2 = 0; t2 <= jx; ++t2)
                      for (int u2 = 0; u2 <= jy; ++u2)
                        for (int v2 = 0; v2 <= jz; ++v2) {
                          const real f = fx[t2] * fy[u2] * fz[v2];
                          if (f == 0) continue;
                          const real sg = ((t2 + u2 + v2) & 1) ? -1 : 1;
                          sum += e * f * sg * R[((t + t2) * d + u + u2) * d + v + v2];
                        }
                  }
              Vc[ia * ncb + ib] += pre * sum;
            }
        }
    }
  for (int ma = 0; ma < 2 * la + 1; ++ma)
    for (int mb = 0; mb < 2 * lb + 1; ++mb) {
      real s2 = 0;
      for (int ia = 0; ia < nca; ++ia)
        for (int ib = 0; ib < ncb; ++ib) s2 += ca[ma * nca + ia] * cb[mb * ncb + ib] * Vc[ia * ncb + ib];
      out[ma * (2 * lb + 1) + mb] = s2;
    }
  free(Vc);
  free(R);
  free(work);
  free(Eb);
  free(Ea);
}

/* Four-centre electron-repulsion block: out[((ma nb + mb) nc + mc) nd + md] =
 *   (a, ma b, mb | c, mc d, md) = int int phi_a(r1) phi_b(r1) phi_c(r2) phi_d(r2) / |r1 - r2| d3r1 d3r2,
 * the two-electron Coulomb integral whose SHGO form Eqs. 13-15 derive.  McMurchie-Davidson: per primitive
 * quartet, with p = alpha + beta, q = gamma + delta and the Hermite coefficients E^{ab} about P and E^{cd}
 * about Q,
 *   2 pi^{5/2} / (p q sqrt(p + q)) sum_{tuv} E^{ab}_{tuv} sum_{t'u'v'} (-1)^{t'+u'+v'} E^{cd}_{t'u'v'}
 *       R^0_{t+t', u+u', v+v'}(pq / (p + q), P - Q),
 * done as two passes: the ket sum for every bra Hermite index first, then the bra sum. */
static void eri_block(const shell_t* a, const shell_t* b, const shell_t* c, const shell_t* dd, const real* ca,
                      const real* cb, const real* cc, const real* cd, real* out) {
  const int la = a->l, lb = b->l, lc = c->l, ld = dd->l;
  const int L1 = la + lb, L2 = lc + ld, L = L1 + L2, d = L + 1;
  const int nca = ncart(la), ncb = ncart(lb), ncc = ncart(lc), ncd = ncart(ld);
  const int t1 = L1 + 1, t2 = L2 + 1;
  const size_t eab = (size_t)(la + 1) * (lb + 1) * t1, ecd = (size_t)(lc + 1) * (ld + 1) * t2;
  real* Eab = (real*)malloc(sizeof(real) * 3 * eab);
  real* Ecd = (real*)malloc(sizeof(real) * 3 * ecd);
  real* work = (real*)malloc(sizeof(real) * (size_t)d * d * d * d);
  real* R = (real*)malloc(sizeof(real) * (size_t)d * d * d);
  real* Wk = (real*)malloc(sizeof(real) * (size_t)t1 * t1 * t1);
  const size_t nabcd = (size_t)nca * ncb * ncc * ncd;
  real* G = (real*)calloc(nabcd, sizeof(real));
  for (int i = 0; i < a->nprim; ++i)
    for (int j = 0; j < b->nprim; ++j) {
      const real al = a->alpha[i], be = b->alpha[j], p = al + be, mu = al * be / p;
      real P[3];
      for (int x = 0; x < 3; ++x) {
        P[x] = (al * a->A[x] + be * b->A[x]) / p;
        const real X = a->A[x] - b->A[x];
        hermite_E(la, lb, p, P[x] - a->A[x], P[x] - b->A[x], RX(exp)(-mu * X * X), Eab + x * eab);
      }
      for (int k = 0; k < c->nprim; ++k)
        for (int l = 0; l < dd->nprim; ++l) {
          const real ga = c->alpha[k], de = dd->alpha[l], q = ga + de, nu = ga * de / q;
          real Q[3];
          for (int x = 0; x < 3; ++x) {
            Q[x] = (ga * c->A[x] + de * dd->A[x]) / q;
            const real X = c->A[x] - dd->A[x];
            hermite_E(lc, ld, q, Q[x] - c->A[x], Q[x] - dd->A[x], RX(exp)(-nu * X * X), Ecd + x * ecd);
          }
          hermite_R(L, p * q / (p + q), P[0] - Q[0], P[1] - Q[1], P[2] - Q[2], work, R);
          const real pre = a->coef[i] * b->coef[j] * c->coef[k] * dd->coef[l] * 2 * RX(pow)(RPI, (real)2.5) /
                           (p * q * RX(sqrt)(p + q));
          for (int kx = lc; kx >= 0; --kx)
            for (int ky = lc - kx; ky >= 0; --ky) {
              const int kz = lc - kx - ky, ic = cart_index(lc, kx, ky);
              for (int lx = ld; lx >= 0; --lx)
                for (int ly = ld - lx; ly >= 0; --ly) {
                  const int lz = ld - lx - ly, id = cart_index(ld, lx, ly);
                  const real* fx = Ecd + (kx * (ld + 1) + lx) * t2;
                  const real* fy = Ecd + ecd + (ky * (ld + 1) + ly) * t2;
                  const real* fz = Ecd + 2 * ecd + (kz * (ld + 1) + lz) * t2;
                  /* ket pass: W[t][u][v] for every bra Hermite index with t + u + v <= L1 */
                  for (int t = 0; t <= L1; ++t)
                    for (int u = 0; u + t <= L1; ++u)
                      for (int v = 0; v + u + t <= L1; ++v) {
                        real w = 0;
                        for (int tt = 0; tt <= kx + lx; ++tt)
                          for (int uu = 0; uu <= ky + ly; ++uu)
                            for (int vv = 0; vv <= kz + lz; ++vv) {
                              const real f = fx[tt] * fy[uu] * fz[vv];
                              const real sg = ((tt + uu + vv) & 1) ? -1 : 1;
                              w += sg * f * R[((t + tt) * d + u + uu) * d + v + vv];
                            }
                        Wk[(t * t1 + u) * t1 + v] = w;
                      }
                  /* bra pass */
                  for (int ix = la; ix >= 0; --ix)
                    for (int iy = la - ix; iy >= 0; --iy) {
                      const int iz = la - ix - iy, ia = cart_index(la, ix, iy);
                      for (int jx = lb; jx >= 0; --jx)
                        for (int jy = lb - jx; jy >= 0; --jy) {
                          const int jz = lb - jx - jy, ib = cart_index(lb, jx, jy);
                          const real* ex = Eab + (ix * (lb + 1) + jx) * t1;
                          const real* ey = Eab + eab + (iy * (lb + 1) + jy) * t1;
                          const real* ez = Eab + 2 * eab + (iz * (lb + 1) + jz) * t1;
                          real s = 0;
                          for (int t = 0; t <= ix + jx; ++t)
                            for (int u = 0; u <= iy + jy; ++u)
                              for (int v = 0; v <= iz + jz; ++v) s += ex[t] * ey[u] * ez[v] * Wk[(t * t1 + u) * t1 + v];
                          G[(((size_t)ia * ncb + ib) * ncc + ic) * ncd + id] += pre * s;
                        }
                    }
                }
            }
        }
    }
  /* Cartesian -> real solid harmonics, one index at a time */
  const int na = 2 * la + 1, nb = 2 * lb + 1, nc = 2 * lc + 1, nd = 2 * ld + 1;
  real* T1 = (real*)calloc((size_t)na * ncb * ncc * ncd, sizeof(real));
  real* T2 = (real*)calloc((size_t)na * nb * ncc * ncd, sizeof(real));
  real* T3 = (real*)calloc((size_t)na * nb * nc * ncd, sizeof(real));
  for (int ma = 0; ma < na; ++ma)
    for (int ia = 0; ia < nca; ++ia)
      for (size_t r = 0; r < (size_t)ncb * ncc * ncd; ++r)
        T1[(size_t)ma * ncb * ncc * ncd + r] += ca[ma * nca + ia] * G[(size_t)ia * ncb * ncc * ncd + r];
  for (int ma = 0; ma < na; ++ma)
    for (int mb = 0; mb < nb; ++mb)
      for (int ib = 0; ib < ncb; ++ib)
        for (size_t r = 0; r < (size_t)ncc * ncd; ++r)
          T2[((size_t)ma * nb + mb) * ncc * ncd + r] += cb[mb * ncb + ib] * T1[((size_t)ma * ncb + ib) * ncc * ncd + r];
  for (size_t ab = 0; ab < (size_t)na * nb; ++ab)
    for (int mc = 0; mc < nc; ++mc)
      for (int ic = 0; ic < ncc; ++ic)
        for (int id = 0; id < ncd; ++id)
          T3[(ab * nc + mc) * ncd + id] += cc[mc * ncc + ic] * T2[(ab * ncc + ic) * ncd + id];
  for (size_t abc = 0; abc < (size_t)na * nb * nc; ++abc)
    for (int md = 0; md < nd; ++md) {
      real s = 0;
      for (int id = 0; id < ncd; ++id) s += cd[md * ncd + id] * T3[abc * ncd + id];
      out[abc * nd + md] = s;
    }
  free(T3);
  free(T2);
  free(T1);
  free(G);
  free(Wk);
  free(R);
  free(work);
  free(Ecd);
  free(Eab);
}

/* ------------------------------------------------------------------------------------------ */
/* Public entry points.                                                                       */
/* ------------------------------------------------------------------------------------------ */
typedef enum { OP_OVERLAP = 0, OP_NUCLEAR = 1, OP_COULOMB2C = 2, OP_NUCLEAR_DA = 3 } op_t;

static int one_electron(op_t op, int n_shells, const int* l, const int* nprim, const double* exps,
                        const double* coefs, const double* xyz, long nC, const double* C, const double* Z,
                        double* out, int n_threads, int dcomp) {
  if (n_shells < 0) return -1;
  shell_t* sh = (shell_t*)calloc((size_t)(n_shells > 0 ? n_shells : 1), sizeof(shell_t));
  real* cart[ORACLE_LMAX + 1];
  for (int ll = 0; ll <= ORACLE_LMAX; ++ll) {
    cart[ll] = (real*)malloc(sizeof(real) * (size_t)(2 * ll + 1) * ncart(ll));
    solid_harmonic_cart(ll, cart[ll]);
  }
  int rc = setup_shells(n_shells, l, nprim, exps, coefs, xyz, sh, cart);
  long* off = (long*)malloc(sizeof(long) * (size_t)(n_shells + 1));
  off[0] = 0;
  for (int s = 0; s < n_shells; ++s) off[s + 1] = off[s] + (rc == 0 ? 2 * sh[s].l + 1 : 0);
  const long nbf = off[n_shells];
  if (rc == 0) {
    const long npairs = (long)n_shells * (n_shells + 1) / 2;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (long q = 0; q < npairs; ++q) {
      /* q enumerates pairs a >= b */
      long a = (long)((sqrt(8.0 * (double)q + 1.0) - 1.0) / 2.0);
      while (a * (a + 1) / 2 > q) --a;
      while ((a + 1) * (a + 2) / 2 <= q) ++a;
      const long b = q - a * (a + 1) / 2;
      const int na = 2 * sh[a].l + 1, nb = 2 * sh[b].l + 1;
      real* blk = (real*)malloc(sizeof(real) * (size_t)na * nb);
      if (op == OP_NUCLEAR_DA) {
        /* rows of shell a: the derivative with respect to a's centre; rows of shell b (a != b): with
         * respect to b's centre, the block with b as the bra */
        nuclear_dA_block(&sh[a], &sh[b], cart[sh[a].l], cart[sh[b].l], nC, C, Z, blk, dcomp);
        for (int i = 0; i < na; ++i)
          for (int j = 0; j < nb; ++j) out[(off[a] + i) * nbf + off[b] + j] = (double)blk[i * nb + j];
        if (a != b) {
          real* blk2 = (real*)malloc(sizeof(real) * (size_t)na * nb);
          nuclear_dA_block(&sh[b], &sh[a], cart[sh[b].l], cart[sh[a].l], nC, C, Z, blk2, dcomp);
          for (int j = 0; j < nb; ++j)
            for (int i = 0; i < na; ++i) out[(off[b] + j) * nbf + off[a] + i] = (double)blk2[j * na + i];
          free(blk2);
        }
        free(blk);
        continue;
      }
      if (op == OP_OVERLAP)
        overlap_block(&sh[a], &sh[b], cart[sh[a].l], cart[sh[b].l], blk);
      else if (op == OP_COULOMB2C)
        coulomb2c_block(&sh[a], &sh[b], cart[sh[a].l], cart[sh[b].l], blk);
      else
        nuclear_block(&sh[a], &sh[b], cart[sh[a].l], cart[sh[b].l], nC, C, Z, blk, dcomp);
      for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j) {
          out[(off[a] + i) * nbf + off[b] + j] = (double)blk[i * nb + j];
          out[(off[b] + j) * nbf + off[a] + i] = (double)blk[i * nb + j];
        }
      free(blk);
    }
  }
  free(off);
  for (int ll = 0; ll <= ORACLE_LMAX; ++ll) free(cart[ll]);
  free(sh);
  return rc;
}

/* V_ab = sum_C Z_C <phi_a | 1/|r - C| | phi_b>, written to out (nbf x nbf, row-major, both
 * triangles).  Shell s has l[s], nprim[s] primitives whose exponents and coefficients follow
 * those of shell s-1 in exps/coefs, and centre xyz[3s..3s+2] (bohr).  Returns 0, or -1 on bad
 * input.  n_threads > 0 sets the OpenMP thread count (shell pairs are independent). */
int oracle_nuclear_attraction(int n_shells, const int* l, const int* nprim, const double* exps,
                              const double* coefs, const double* xyz, long n_centers, const double* centers,
                              const double* charges, double* out, int n_threads) {
  return one_electron(OP_NUCLEAR, n_shells, l, nprim, exps, coefs, xyz, n_centers, centers, charges, out,
                      n_threads, -1);
}

/* Derivative of V with respect to coordinate `component` (0, 1, 2 = x, y, z) of the nuclei:
 * sum_C Z_C d/dC_component <phi_a | 1/|r - C| | phi_b> (for one nucleus, the field integrals of the
 * point C, up to sign).  Same layout and conventions as oracle_nuclear_attraction. */
int oracle_nuclear_field(int n_shells, const int* l, const int* nprim, const double* exps, const double* coefs,
                         const double* xyz, long n_centers, const double* centers, const double* charges,
                         int component, double* out, int n_threads) {
  if (component < 0 || component > 2) return -1;
  return one_electron(OP_NUCLEAR, n_shells, l, nprim, exps, coefs, xyz, n_centers, centers, charges, out,
                      n_threads, component);
}

/* Derivative of V with respect to coordinate `component` of the bra function's centre:
 * out[a][b] = d/dA_component sum_C Z_C <phi_a | 1/|r - C| | phi_b>, A the centre of a's shell, with the
 * centre of b's shell held fixed even where it coincides with A (so out is not symmetric; the derivative
 * with respect to b's centre is out[b][a]).  nbf x nbf row-major; returns 0, or -1 on bad input. */
int oracle_nuclear_deriv(int n_shells, const int* l, const int* nprim, const double* exps, const double* coefs,
                         const double* xyz, long n_centers, const double* centers, const double* charges,
                         int component, double* out, int n_threads) {
  if (component < 0 || component > 2) return -1;
  return one_electron(OP_NUCLEAR_DA, n_shells, l, nprim, exps, coefs, xyz, n_centers, centers, charges, out,
                      n_threads, component);
}

/* S_ab = <phi_a | phi_b> (Eq. 4) over the same basis; same layout and conventions. */
int oracle_overlap(int n_shells, const int* l, const int* nprim, const double* exps, const double* coefs,
                   const double* xyz, double* out, int n_threads) {
  return one_electron(OP_OVERLAP, n_shells, l, nprim, exps, coefs, xyz, 0, NULL, NULL, out, n_threads, -1);
}

/* Two-centre Coulomb integrals (a|b) = int int phi_a(r1) phi_b(r2) / |r1 - r2| over the same basis (the
 * metric of density fitting; the two-centre case of the electron-repulsion integrals of Eqs. 13-15);
 * same layout and conventions. */
int oracle_coulomb_2c(int n_shells, const int* l, const int* nprim, const double* exps, const double* coefs,
                      const double* xyz, double* out, int n_threads) {
  return one_electron(OP_COULOMB2C, n_shells, l, nprim, exps, coefs, xyz, 0, NULL, NULL, out, n_threads, -1);
}

/* Four-centre electron-repulsion integrals (ab|cd) over the same basis (Eqs. 13-15), written to out
 * (nbf^4 doubles, row-major: out[((i nbf + j) nbf + k) nbf + l] = (ij|kl)).  Each shell quartet with
 * pair index (a, b) >= (c, d), a >= b and c >= d is computed once and written to its eight
 * permutations (the integrals of real orbitals share one value).  Returns 0, or -1 on bad input. */
int oracle_eri(int n_shells, const int* l, const int* nprim, const double* exps, const double* coefs,
               const double* xyz, double* out, int n_threads) {
  if (n_shells < 0) return -1;
  shell_t* sh = (shell_t*)calloc((size_t)(n_shells > 0 ? n_shells : 1), sizeof(shell_t));
  real* cart[ORACLE_LMAX + 1];
  for (int ll = 0; ll <= ORACLE_LMAX; ++ll) {
    cart[ll] = (real*)malloc(sizeof(real) * (size_t)(2 * ll + 1) * ncart(ll));
    solid_harmonic_cart(ll, cart[ll]);
  }
  const int rc = setup_shells(n_shells, l, nprim, exps, coefs, xyz, sh, cart);
  long* off = (long*)malloc(sizeof(long) * (size_t)(n_shells + 1));
  off[0] = 0;
  for (int s = 0; s < n_shells; ++s) off[s + 1] = off[s] + (rc == 0 ? 2 * sh[s].l + 1 : 0);
  const long n = off[n_shells];
  if (rc == 0) {
    const long npairs = (long)n_shells * (n_shells + 1) / 2;
    long* pa = (long*)malloc(sizeof(long) * (size_t)(npairs > 0 ? npairs : 1));
    long* pb = (long*)malloc(sizeof(long) * (size_t)(npairs > 0 ? npairs : 1));
    for (long a = 0, q = 0; a < n_shells; ++a)
      for (long b = 0; b <= a; ++b, ++q) {
        pa[q] = a;
        pb[q] = b;
      }
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (long q1 = 0; q1 < npairs; ++q1)
      for (long q2 = 0; q2 <= q1; ++q2) {
        const long A = pa[q1], B = pb[q1], C = pa[q2], D = pb[q2];
        const int na = 2 * sh[A].l + 1, nb = 2 * sh[B].l + 1, nc = 2 * sh[C].l + 1, nd = 2 * sh[D].l + 1;
        real* blk = (real*)malloc(sizeof(real) * (size_t)na * nb * nc * nd);
        eri_block(&sh[A], &sh[B], &sh[C], &sh[D], cart[sh[A].l], cart[sh[B].l], cart[sh[C].l], cart[sh[D].l], blk);
        for (int i = 0; i < na; ++i)
          for (int j = 0; j < nb; ++j)
            for (int k = 0; k < nc; ++k)
              for (int m = 0; m < nd; ++m) {
                const double v = (double)blk[((i * nb + j) * nc + k) * nd + m];
                const long I = off[A] + i, J = off[B] + j, K = off[C] + k, M = off[D] + m;
                out[((I * n + J) * n + K) * n + M] = v;
                out[((J * n + I) * n + K) * n + M] = v;
                out[((I * n + J) * n + M) * n + K] = v;
                out[((J * n + I) * n + M) * n + K] = v;
                out[((K * n + M) * n + I) * n + J] = v;
                out[((M * n + K) * n + I) * n + J] = v;
                out[((K * n + M) * n + J) * n + I] = v;
                out[((M * n + K) * n + J) * n + I] = v;
              }
        free(blk);
      }
    free(pb);
    free(pa);
  }
  free(off);
  for (int ll = 0; ll <= ORACLE_LMAX; ++ll) free(cart[ll]);
  free(sh);
  return rc;
}

/* Primitive normalisation N(l, alpha) of Eq. 1, as used above. */
double oracle_prim_norm(int l, double alpha) { return (double)prim_norm(l, alpha); }

int oracle_real_bits(void) { return (int)(sizeof(real) * 8); }
