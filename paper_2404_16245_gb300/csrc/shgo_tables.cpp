// Host construction of the constant tables: recursion coefficients of the real solid
// harmonics, the real translation tensors (addition theorem, Eqs. 7-8), the real coupling
// (Gaunt) programs (Clebsch-Gordan product rule, Supp. Eq. 4), the packed layout of the
// per-primitive-pair coupling block, and the Boys grid.  Built once per process in long double.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include "shgo_internal.h"
#include "shgo_math.h"

namespace shgo {

using ld = long double;
using cld = std::complex<long double>;

namespace {

ld fact(int n) {
  ld f = 1;
  for (int i = 2; i <= n; ++i) f *= (ld)i;
  return f;
}

ld binom(int n, int k) {
  if (n < 0 || k < 0 || k > n) return 0;
  return fact(n) / (fact(k) * fact(n - k));
}

// Clebsch-Gordan coefficient <j1 m1 j2 m2 | J M> by Racah's closed formula.
ld clebsch_gordan(int j1, int m1, int j2, int m2, int J, int M) {
  if (M != m1 + m2 || J < std::abs(j1 - j2) || J > j1 + j2) return 0;
  if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(M) > J) return 0;
  const ld pre = std::sqrt((ld)(2 * J + 1) * fact(j1 + j2 - J) * fact(j1 - j2 + J) * fact(-j1 + j2 + J) /
                           fact(j1 + j2 + J + 1)) *
                 std::sqrt(fact(j1 + m1) * fact(j1 - m1) * fact(j2 + m2) * fact(j2 - m2) * fact(J + M) * fact(J - M));
  ld sum = 0;
  for (int k = 0; k <= j1 + j2 - J; ++k) {
    const int d1 = j1 + j2 - J - k, d2 = j1 - m1 - k, d3 = j2 + m2 - k, d4 = J - j2 + m1 + k, d5 = J - j1 - m2 + k;
    if (d1 < 0 || d2 < 0 || d3 < 0 || d4 < 0 || d5 < 0) continue;
    const ld term = 1 / (fact(k) * fact(d1) * fact(d2) * fact(d3) * fact(d4) * fact(d5));
    sum += (k & 1) ? -term : term;
  }
  return pre * sum;
}

// Unitary map from complex to real harmonics: S_{l,m} = sum_m' U[m][m'] Y_l^{m'} with
//   S_l0 = Y_l^0,  S_{l,m>0} = ((-1)^m Y^m + Y^-m)/sqrt2,  S_{l,-m} = ((-1)^m Y^m - Y^-m)/(i sqrt2).
cld umap(int m, int mp) {
  const ld r2 = std::sqrt((ld)0.5);
  if (m == 0) return mp == 0 ? cld(1, 0) : cld(0, 0);
  if (m > 0) {
    const ld sg = (m & 1) ? -1 : 1;
    if (mp == m) return cld(sg * r2, 0);
    if (mp == -m) return cld(r2, 0);
    return cld(0, 0);
  }
  const int mu = -m;
  const ld sg = (mu & 1) ? -1 : 1;
  if (mp == mu) return cld(0, -sg * r2);
  if (mp == -mu) return cld(0, r2);
  return cld(0, 0);
}

// The two complex indices that a real index m couples to (m and -m; one when m = 0).
int partners(int m, int* out) {
  if (m == 0) {
    out[0] = 0;
    return 1;
  }
  out[0] = std::abs(m);
  out[1] = -std::abs(m);
  return 2;
}

// Vector-coupling coefficient of Eq. 8: eps_{l1 l2 m1 m2} = sqrt(C(l1+m1, l2+m2) C(l1-m1, l2-m2)).
ld epsilon(int l1, int l2, int m1, int m2) { return std::sqrt(binom(l1 + m1, l2 + m2) * binom(l1 - m1, l2 - m2)); }

}  // namespace

double gaunt_real(int l1, int m1, int l2, int m2, int L, int M) {
  if (std::abs(m1) > l1 || std::abs(m2) > l2 || std::abs(M) > L) return 0;
  if (((l1 + l2 + L) & 1) || L < std::abs(l1 - l2) || L > l1 + l2) return 0;
  const ld cg0 = clebsch_gordan(l1, 0, l2, 0, L, 0);
  int p1[2], p2[2];
  const int n1 = partners(m1, p1), n2 = partners(m2, p2);
  cld acc(0, 0);
  for (int a = 0; a < n1; ++a)
    for (int b = 0; b < n2; ++b) {
      const int Mp = p1[a] + p2[b];
      if (std::abs(Mp) > L) continue;
      const ld cg = clebsch_gordan(l1, p1[a], l2, p2[b], L, Mp);
      acc += umap(m1, p1[a]) * umap(m2, p2[b]) * cg0 * cg * std::conj(umap(M, Mp));
    }
  return (double)acc.real();
}

double translation_real(int la, int ma, int l1, int m1, int nu) {
  const int lr = la - l1;
  if (l1 < 0 || lr < 0 || std::abs(ma) > la || std::abs(m1) > l1 || std::abs(nu) > lr) return 0;
  int pa[2], p1[2], pr[2];
  const int na = partners(ma, pa), n1 = partners(m1, p1), nr = partners(nu, pr);
  cld acc(0, 0);
  for (int a = 0; a < na; ++a)
    for (int b = 0; b < n1; ++b)
      for (int c = 0; c < nr; ++c) {
        if (pa[a] != p1[b] + pr[c]) continue;
        acc += umap(ma, pa[a]) * epsilon(la, l1, pa[a], p1[b]) * std::conj(umap(m1, p1[b])) * std::conj(umap(nu, pr[c]));
      }
  return (double)acc.real();
}

int translation_offset(int la, int ma, int l1, int m1) {
  // Within the la block: (ma, l1, m1) in order, each followed by 2(la-l1)+1 nu values.
  int off = 0;
  const int per_ma = [&] {
    int s = 0;
    for (int k = 0; k <= la; ++k) s += (2 * k + 1) * (2 * (la - k) + 1);
    return s;
  }();
  off += (ma + la) * per_ma;
  for (int k = 0; k < l1; ++k) off += (2 * k + 1) * (2 * (la - k) + 1);
  off += (m1 + l1) * (2 * (la - l1) + 1);
  return off;
}

const HarmCoef& harm_coef_host() {
  static HarmCoef hc;
  static std::once_flag once;
  std::call_once(once, [] {
    std::memset(&hc, 0, sizeof(hc));
    for (int l = 0; l <= kHarmMax; ++l) {
      hc.c[l] = (double)std::sqrt((ld)(2 * l + 1) / (ld)(2 * l + 2));
      for (int m = -l; m <= l; ++m) {
        const int k = harm_index(l, m);
        hc.a[k] = (double)((ld)(2 * l + 1) / std::sqrt((ld)(l + m + 1) * (ld)(l - m + 1)));
        hc.b[k] = (double)std::sqrt((ld)(l + m) * (ld)(l - m) / ((ld)(l + m + 1) * (ld)(l - m + 1)));
      }
    }
    // N_lm follows the normalised recursion's constants: N_{l+1,m} = a_lm N_lm for |m| <= l,
    // N_{l+1,+-(l+1)} = c_l N_{l,l}; then gamma_lm = b_lm N_{l-1,m} / (a_lm N_lm)
    std::vector<ld> N((size_t)(kHarmMax + 1) * (kHarmMax + 1), 0.0L);
    N[0] = 1.0L;
    if (kHarmMax >= 1) N[1] = N[2] = N[3] = 1.0L;
    for (int l = 1; l < kHarmMax; ++l) {
      const ld cl = std::sqrt((ld)(2 * l + 1) / (ld)(2 * l + 2));
      N[harm_index(l + 1, l + 1)] = cl * N[harm_index(l, l)];
      N[harm_index(l + 1, -l - 1)] = cl * N[harm_index(l, -l)];
      for (int m = -l; m <= l; ++m) {
        const ld a = (ld)(2 * l + 1) / std::sqrt((ld)(l + m + 1) * (ld)(l - m + 1));
        const ld b = std::sqrt((ld)(l + m) * (ld)(l - m) / ((ld)(l + m + 1) * (ld)(l - m + 1)));
        N[harm_index(l + 1, m)] = a * N[harm_index(l, m)];
        if (m > -l && m < l) hc.ng[harm_index(l, m)] = (double)(-b * N[harm_index(l - 1, m)] / (a * N[harm_index(l, m)]));
      }
    }
    for (size_t k = 0; k < N.size(); ++k) hc.n[k] = (double)N[k];
  });
  return hc;
}

const BoysConst& boys_const_host() {
  static BoysConst bc;
  static std::once_flag once;
  std::call_once(once, [] {
    for (int k = 0; k <= kBoysK; ++k) bc.inv_fact[k] = (double)(1 / fact(k));
    for (int n = 0; n < kBoysNmax + 2; ++n) bc.inv_odd[n] = (double)(1 / (ld)(2 * n + 1));
    bc.inv_int[0] = 0.0;
    for (int k = 1; k < kLamMax + 2; ++k) bc.inv_int[k] = (double)(1 / (ld)k);
  });
  return bc;
}

namespace {

// F_n(T_g) for n = 0..nmax by the series F_nmax(T) = exp(-T) sum_i (2T)^i/[(2nmax+1)...(2nmax+2i+1)]
// followed by downward recursion, all in long double.
void boys_grid_row(ld T, int nmax, ld* F, ld* ex) {
  *ex = std::exp(-T);
  ld term = 1 / (ld)(2 * nmax + 1), sum = term;
  for (int i = 1; i < 4000; ++i) {
    term *= 2 * T / (ld)(2 * nmax + 2 * i + 1);
    sum += term;
    if (term < sum * (ld)1e-36) break;
  }
  F[nmax] = *ex * sum;
  for (int n = nmax - 1; n >= 0; --n) F[n] = (2 * T * F[n + 1] + *ex) / (ld)(2 * n + 1);
}

// Index of (L, M, k) in the packed R layout of Lambda (entries ordered by L, then M, then k).
int r_index(int lam, int L, int M, int k) {
  int e = 0;
  for (int l = 0; l < L; ++l) e += (2 * l + 1) * (kmax_of(lam, l) + 1);
  return e + (M + L) * (kmax_of(lam, L) + 1) + k;
}

// Tables::d_* (derivative integrals): index maps between R layouts, the x_c-raising and the
// derivative of the one-centre integrand per R entry, and the lowering d/dx_c S_lm.
void build_deriv_tables(Tables& t) {
  const int mc[3] = {1, -1, 0};
  t.d_map0_off.assign(kLamMax + 2, 0);
  t.d_mapm_off.assign(kLamMax + 2, 0);
  t.d_xoff.assign(kLamMax + 2, 0);
  t.d_map0.clear();
  t.d_mapm.clear();
  for (int lam = 0; lam <= kLamMax; ++lam) {
    t.d_map0_off[lam] = (int)t.d_map0.size();
    t.d_mapm_off[lam] = (int)t.d_mapm.size();
    t.d_xoff[lam + 1] = t.d_xoff[lam] + n_r(lam);
    for (int L = 0; L <= lam; ++L)
      for (int M = -L; M <= L; ++M)
        for (int k = 0; k <= kmax_of(lam, L); ++k) t.d_map0.push_back(r_index(lam + 1, L, M, k));
    if (lam >= 1)
      for (int L = 0; L <= lam - 1; ++L)
        for (int M = -L; M <= L; ++M)
          for (int k = 0; k <= kmax_of(lam - 1, L); ++k) t.d_mapm.push_back(r_index(lam + 1, L, M, k));
  }
  t.d_map0_off[kLamMax + 1] = (int)t.d_map0.size();
  t.d_mapm_off[kLamMax + 1] = (int)t.d_mapm.size();
  const size_t nx = (size_t)t.d_xoff[kLamMax + 1] * 3 * kDerivSlots;
  t.d_raise.assign(nx, GTerm{0.0, 0, 0});
  t.d_field.assign(nx, GTerm{0.0, 0, 0});
  for (int lam = 0; lam <= kLamMax; ++lam) {
    int e = 0;
    for (int L = 0; L <= lam; ++L)
      for (int M = -L; M <= L; ++M)
        for (int k = 0; k <= kmax_of(lam, L); ++k, ++e)
          for (int c = 0; c < 3; ++c) {
            GTerm* rs = &t.d_raise[((size_t)(t.d_xoff[lam] + e) * 3 + c) * kDerivSlots];
            GTerm* fs = &t.d_field[((size_t)(t.d_xoff[lam] + e) * 3 + c) * kDerivSlots];
            int nr = 0, nf = 0;
            auto put = [](GTerm* slots, int& n, double coef, int idx) {
              if (n >= kDerivSlots) throw std::logic_error("derivative table: more terms than slots");
              slots[n++] = GTerm{coef, idx, 0};
            };
            for (int Mp = -(L + 1); Mp <= L + 1; ++Mp) {
              const double rho = gaunt_real(1, mc[c], L, M, L + 1, Mp);
              if (std::fabs(rho) <= 1e-15) continue;
              put(rs, nr, rho, r_index(lam + 1, L + 1, Mp, k));
              if (k >= 1) put(fs, nf, 2.0 * k * rho, r_index(lam + 1, L + 1, Mp, k - 1));
            }
            for (int Mp = -(L - 1); L >= 1 && Mp <= L - 1; ++Mp) {
              const double g = gaunt_real(1, mc[c], L, M, L - 1, Mp);
              if (std::fabs(g) <= 1e-15) continue;
              put(rs, nr, g, r_index(lam + 1, L - 1, Mp, k + 1));
              put(fs, nf, (double)(2 * k + 2 * L + 1) * g, r_index(lam + 1, L - 1, Mp, k));
            }
          }
  }
  t.d_low_off.assign(kLmax + 2, 0);
  t.d_low.clear();
  for (int l = 0; l <= kLmax; ++l) {
    t.d_low_off[l] = (int)t.d_low.size();
    if (l == 0) continue;
    for (int c = 0; c < 3; ++c)
      for (int m = -l; m <= l; ++m)
        for (int Mp = -(l - 1); Mp <= l - 1; ++Mp)
          t.d_low.push_back((double)(2 * l + 1) * gaunt_real(1, mc[c], l, m, l - 1, Mp));
  }
  t.d_low_off[kLmax + 1] = (int)t.d_low.size();
}

void build_tables(Tables& t) {
  // Boys grid
  t.boys.assign((size_t)kBoysNg * kBoysStride, 0.0);
  for (int g = 0; g < kBoysNg; ++g) {
    ld F[kBoysNmax + 1], ex;
    boys_grid_row((ld)g / (ld)kBoysInvH, kBoysNmax, F, &ex);
    t.boys[(size_t)g * kBoysStride] = (double)ex;
    for (int n = 0; n <= kBoysNmax; ++n) t.boys[(size_t)g * kBoysStride + 1 + n] = (double)F[n];
  }
  // Translation tensors
  t.eoff.assign(kLmax + 2, 0);
  for (int la = 0; la <= kLmax; ++la) {
    int per_ma = 0;
    for (int k = 0; k <= la; ++k) per_ma += (2 * k + 1) * (2 * (la - k) + 1);
    t.eoff[la + 1] = t.eoff[la] + (2 * la + 1) * per_ma;
  }
  t.etab.assign(t.eoff[kLmax + 1], 0.0);
  for (int la = 0; la <= kLmax; ++la)
    for (int ma = -la; ma <= la; ++ma)
      for (int l1 = 0; l1 <= la; ++l1)
        for (int m1 = -l1; m1 <= l1; ++m1) {
          const int base = t.eoff[la] + translation_offset(la, ma, l1, m1);
          for (int nu = -(la - l1); nu <= la - l1; ++nu)
            t.etab[base + nu + (la - l1)] = translation_real(la, ma, l1, m1, nu);
        }
  // Packed R layout per Lambda: harm index | beta index << 12 | k << 24
  t.rmap_off.assign(kLamDer + 2, 0);
  for (int lam = 0; lam <= kLamDer; ++lam) t.rmap_off[lam + 1] = t.rmap_off[lam] + n_r(lam);
  t.rmap.assign(t.rmap_off[kLamDer + 1], 0);
  for (int lam = 0; lam <= kLamDer; ++lam) {
    int e = t.rmap_off[lam], boff = 0;
    for (int L = 0; L <= lam; ++L) {
      const int km = kmax_of(lam, L);
      for (int M = -L; M <= L; ++M)
        for (int k = 0; k <= km; ++k) t.rmap[e++] = harm_index(L, M) | ((boff + k) << 12) | (k << 24);
      boff += km + 1;
    }
  }
  t.rnorm.resize(t.rmap.size());
  for (size_t e = 0; e < t.rmap.size(); ++e) t.rnorm[e] = harm_coef_host().n[t.rmap[e] & 0xfff];
  build_deriv_tables(t);
  // Rotation recursion lists: Cartesian component c = 0, 1, 2 (x, y, z) is S_{1, m(c)} with
  // m(x) = 1, m(y) = -1, m(z) = 0.
  t.rot_ptr.clear();
  t.rot_terms.clear();
  {
    const int mc[3] = {1, -1, 0};
    for (int l = 0; l < kLmax; ++l)
      for (int M = -(l + 1); M <= l + 1; ++M) {
        t.rot_ptr.push_back((int)t.rot_terms.size());
        for (int c = 0; c < 3; ++c)
          for (int mp = -l; mp <= l; ++mp) {
            const double g = gaunt_real(1, mc[c], l, mp, l + 1, M);
            if (std::fabs(g) > 1e-15) t.rot_terms.push_back(GTerm{g, c, mp});
          }
      }
    t.rot_ptr.push_back((int)t.rot_terms.size());
  }
  // two-centre Coulomb: product-rule terms per class and block entry, and the radial coefficients
  t.c2_ptr.clear();
  t.c2_terms.clear();
  t.c2_base.assign(kNumClasses, 0);
  for (int la = 0; la <= kLmax; ++la)
    for (int lb = 0; lb <= la; ++lb) {
      t.c2_base[class_id(la, lb)] = (int)t.c2_ptr.size();
      for (int ma = -la; ma <= la; ++ma)
        for (int mb = -lb; mb <= lb; ++mb) {
          t.c2_ptr.push_back((int)t.c2_terms.size());
          for (int L = la - lb; L <= la + lb; L += 2)
            for (int M = -L; M <= L; ++M) {
              const double g = gaunt_real(la, ma, lb, mb, L, M);
              if (std::fabs(g) > 1e-15) t.c2_terms.push_back(GTerm{g, L * L + L + M, L});
            }
        }
      t.c2_ptr.push_back((int)t.c2_terms.size());
    }
  t.c2_a.assign((size_t)(kLamMax + 1) * (kC2K + 1) * (kC2K + 1), 0.0);
  for (int L = 0; L <= kLamMax; ++L) {
    // a_{0,0} = 1; Delta_L (u^j f^{(n)}) = (4j^2 + (4L + 2) j) u^{j-1} f^{(n)} + (8j + 4L + 6) u^j f^{(n+1)}
    //                                     + 4 u^{j+1} f^{(n+2)}, with n = L + k + j
    std::vector<ld> cur(1, 1.0L);
    for (int k = 0; k <= kC2K; ++k) {
      for (int j = 0; j <= k; ++j) t.c2_a[((size_t)L * (kC2K + 1) + k) * (kC2K + 1) + j] = (double)cur[j];
      std::vector<ld> nxt(k + 2, 0.0L);
      for (int j = 0; j <= k; ++j) {
        if (j >= 1) nxt[j - 1] += cur[j] * (ld)(4 * j * j + (4 * L + 2) * j);
        nxt[j] += cur[j] * (ld)(8 * j + 4 * L + 6);
        nxt[j + 1] += cur[j] * 4.0L;
      }
      cur.swap(nxt);
    }
  }
  // eps_{k,n}(L): x^{k+1} S_L e^{-px} = [Delta + (8k + 4L + 6) p] (x^k S_L e^{-px}) / (4p^2)
  //               - (4k^2 + (4L + 2) k) x^{k-1} S_L e^{-px} / (4p^2), x = r^2, from
  // Delta (S_L f(x)) = S_L (4x f'' + (4L + 6) f'); the powers of p factor out as p^{-(k+n)}.
  t.eri_eps.assign((size_t)(kLamMax + 1) * (kC2K + 1) * (kC2K + 1), 0.0);
  for (int L = 0; L <= kLamMax; ++L) {
    std::vector<std::vector<ld>> e(kC2K + 1, std::vector<ld>(kC2K + 1, 0.0L));
    e[0][0] = 1.0L;
    for (int k = 0; k < kC2K; ++k)
      for (int n = 0; n <= k + 1; ++n) {
        ld v = (ld)(8 * k + 4 * L + 6) * (n <= k ? e[k][n] : 0.0L);
        if (n >= 1) v += e[k][n - 1];
        if (k >= 1 && n <= k - 1) v -= (ld)(4 * k * k + (4 * L + 2) * k) * e[k - 1][n];
        e[k + 1][n] = v / 4;
      }
    for (int k = 0; k <= kC2K; ++k)
      for (int n = 0; n <= k; ++n) t.eri_eps[((size_t)L * (kC2K + 1) + k) * (kC2K + 1) + n] = (double)e[k][n];
  }
  // Gaunt programs per class
  std::vector<std::vector<std::pair<int, double>>> terms;  // per (i1, i2) over all l <= kLmax
  const int nh = (kLmax + 1) * (kLmax + 1);
  terms.resize((size_t)nh * nh);
  for (int l1 = 0; l1 <= kLmax; ++l1)
    for (int m1 = -l1; m1 <= l1; ++m1)
      for (int l2 = 0; l2 <= kLmax; ++l2)
        for (int m2 = -l2; m2 <= l2; ++m2) {
          auto& v = terms[(size_t)harm_index(l1, m1) * nh + harm_index(l2, m2)];
          for (int L = std::abs(l1 - l2); L <= l1 + l2; L += 2)
            for (int M = -L; M <= L; ++M) {
              const double g = gaunt_real(l1, m1, l2, m2, L, M);
              if (std::fabs(g) > 1e-15) v.push_back({harm_index(L, M) | (((l1 + l2 - L) / 2) << 12), g});
            }
        }
  t.g_rowbase.assign(kNumClasses, 0);
  t.g_grpbase.assign(kNumClasses, 0);
  t.g_termbase.assign(kNumClasses, 0);
  t.g_nnz.assign(kNumClasses, 0);
  t.gt_base.assign(kNumClasses, 0);
  t.gt_termbase.assign(kNumClasses, 0);
  t.gt_ptr.clear();
  t.gt_terms.clear();
  t.g_rowinfo.clear();
  t.g_grp.clear();
  t.g_terms.clear();
  for (int la = 0; la <= kLmax; ++la)
    for (int lb = 0; lb <= la; ++lb) {
      const int cid = class_id(la, lb), lam = la + lb;
      t.g_rowbase[cid] = (int)t.g_rowinfo.size();
      t.g_grpbase[cid] = (int)t.g_grp.size() / 2;
      t.g_termbase[cid] = (int)t.g_terms.size();
      // R index of (L, M, k) in the Lambda layout
      auto ridx = [&](int L, int M, int k) {
        int off = 0;
        for (int Lp = 0; Lp < L; ++Lp) off += (2 * Lp + 1) * (kmax_of(lam, Lp) + 1);
        return off + (M + L) * (kmax_of(lam, L) + 1) + k;
      };
      const int nWa = (la + 1) * (la + 1), nWb = (lb + 1) * (lb + 1), nW = nWa * nWb, ws = w_stride(lb);
      std::vector<int> order;
      for (int i1 = 0; i1 < nWa; ++i1)
        for (int i2 = 0; i2 < nWb; ++i2) order.push_back(i1 * nWb + i2);
      auto row_terms = [&](int e) -> const std::vector<std::pair<int, double>>& {
        return terms[(size_t)(e / nWb) * nh + (e % nWb)];
      };
      std::stable_sort(order.begin(), order.end(),
                       [&](int x, int y) { return row_terms(x).size() > row_terms(y).size(); });
      const int nrp = (nW + 31) / 32 * 32;
      int local = 0;
      for (int g0 = 0; g0 < nrp; g0 += 32) {
        int K = 0;
        for (int i = 0; i < 32 && g0 + i < nW; ++i) K = std::max(K, (int)row_terms(order[g0 + i]).size());
        t.g_grp.push_back(local);
        t.g_grp.push_back(K);
        for (int j = 0; j < K; ++j)
          for (int i = 0; i < 32; ++i) {
            GTerm gt{0.0, 0, 0};
            if (g0 + i < nW) {
              const auto& v = row_terms(order[g0 + i]);
              if (j < (int)v.size()) {
                const int hi = v[j].first & 0xfff, k = v[j].first >> 12;
                int L = 0;
                while ((L + 1) * (L + 1) <= hi) ++L;
                gt = GTerm{v[j].second, ridx(L, hi - L * L - L, k), 0};
              }
            }
            t.g_terms.push_back(gt);
          }
        local += 32 * K;
        for (int i = 0; i < 32; ++i) {
          if (g0 + i >= nW) {
            t.g_rowinfo.push_back(-1);
            continue;
          }
          const int e = order[g0 + i], i1 = e / nWb, i2 = e % nWb;
          int l1 = 0, l2 = 0;
          while ((l1 + 1) * (l1 + 1) <= i1) ++l1;
          while ((l2 + 1) * (l2 + 1) <= i2) ++l2;
          t.g_rowinfo.push_back((i1 * ws + i2) | (l1 << 16) | (l2 << 20));
          t.g_nnz[cid] += (int)row_terms(e).size();
        }
      }
      // transposed program: for each R' entry, the (coefficient, W entry, l1 l2) pairs feeding it
      {
        const int nr = n_r(lam);
        std::vector<std::vector<GTerm>> byr(nr);
        for (int i1 = 0; i1 < nWa; ++i1)
          for (int i2 = 0; i2 < nWb; ++i2) {
            int l1 = 0, l2 = 0;
            while ((l1 + 1) * (l1 + 1) <= i1) ++l1;
            while ((l2 + 1) * (l2 + 1) <= i2) ++l2;
            for (const auto& v : row_terms(i1 * nWb + i2)) {
              const int hi = v.first & 0xfff, k = v.first >> 12;
              int L = 0;
              while ((L + 1) * (L + 1) <= hi) ++L;
              byr[ridx(L, hi - L * L - L, k)].push_back(GTerm{v.second, i1 * ws + i2, l1 * (lb + 1) + l2});
            }
          }
        t.gt_base[cid] = (int)t.gt_ptr.size();
        t.gt_termbase[cid] = (int)t.gt_terms.size();
        int loc = 0;
        for (int e = 0; e < nr; ++e) {
          t.gt_ptr.push_back(loc);
          for (const GTerm& g : byr[e]) t.gt_terms.push_back(g);
          loc += (int)byr[e].size();
        }
        t.gt_ptr.push_back(loc);
      }
    }
}

}  // namespace

void build_site_pairs(const double* shell_xyz, const std::vector<int>& pa, const std::vector<int>& pb,
                      std::vector<int>& pair_site, std::vector<int>& site_rep, std::vector<double>& site_rot) {
  // shells -> positions (bitwise-equal coordinates), then ordered position pairs
  int nsh = 0;
  for (size_t q = 0; q < pa.size(); ++q) nsh = std::max(nsh, std::max(pa[q], pb[q]) + 1);
  // positions keyed by the bits of their three coordinates
  struct Key {
    uint64_t x, y, z;
    bool operator==(const Key& o) const { return x == o.x && y == o.y && z == o.z; }
  };
  struct KeyHash {
    size_t operator()(const Key& k) const {
      uint64_t h = k.x * 0x9E3779B97F4A7C15ull;
      h ^= (k.y + 0x632BE59BD9B4E019ull + (h << 6) + (h >> 2)) * 0xBF58476D1CE4E5B9ull;
      h ^= (k.z + 0x94D049BB133111EBull + (h << 6) + (h >> 2)) * 0x9E3779B97F4A7C15ull;
      return (size_t)(h ^ (h >> 31));
    }
  };
  std::vector<int> shell_pos(nsh, -1);
  std::unordered_map<Key, int, KeyHash> pos;
  pos.reserve((size_t)nsh);
  for (int s = 0; s < nsh; ++s) {
    Key k{};
    std::memcpy(&k.x, shell_xyz + 3 * s, sizeof(double));
    std::memcpy(&k.y, shell_xyz + 3 * s + 1, sizeof(double));
    std::memcpy(&k.z, shell_xyz + 3 * s + 2, sizeof(double));
    shell_pos[s] = pos.emplace(k, (int)pos.size()).first->second;
  }
  const int64_t np = (int64_t)pos.size();
  pair_site.resize(pa.size());
  site_rep.clear();
  auto add = [&](size_t q) {
    site_rep.push_back((int)q);
    return (int)site_rep.size() - 1;
  };
  if (np * np <= ((int64_t)1 << 24)) {
    std::vector<int> table((size_t)(np * np), -1);
    for (size_t q = 0; q < pa.size(); ++q) {
      int& t = table[(size_t)(shell_pos[pa[q]] * np + shell_pos[pb[q]])];
      if (t < 0) t = add(q);
      pair_site[q] = t;
    }
  } else {
    std::unordered_map<int64_t, int> sp;
    for (size_t q = 0; q < pa.size(); ++q) {
      const int64_t key = (int64_t)shell_pos[pa[q]] * np + shell_pos[pb[q]];
      auto it = sp.find(key);
      if (it == sp.end()) it = sp.emplace(key, add(q)).first;
      pair_site[q] = it->second;
    }
  }
  site_rot.resize(9 * site_rep.size());
  for (size_t i = 0; i < site_rep.size(); ++i)
    pair_frame(shell_xyz + 3 * pa[site_rep[i]], shell_xyz + 3 * pb[site_rep[i]], &site_rot[9 * i]);
}

const Tables& tables_host() {
  static Tables t;
  static std::once_flag once;
  std::call_once(once, [] { build_tables(t); });
  return t;
}

void boys_host(int nmax, double T, double* F) { boys_eval(nmax, T, F, 1, tables_host().boys.data(), boys_const_host()); }

}  // namespace shgo
