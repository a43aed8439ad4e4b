// Per-nucleus device helpers of the FP64 nucleus loop (step S2), shared by the coupling kernel and the
// fused shell-pair kernel: Boys values and radial sums, unit-vector solid-harmonic columns and the
// pair-frame offset of a nucleus.  Each translation unit that includes this header gets its own copy of
// the recursion and Boys constants (k_harm, k_boys) and uploads them in its set-up function.
#pragma once

#include <cuda_runtime.h>

#include "shgo_internal.h"
#include "shgo_math.h"

namespace shgo {
namespace {

__constant__ HarmCoef k_harm;
__constant__ BoysConst k_boys;

constexpr double kTwoPiC = 6.283185307179586476925286766559;

__host__ __device__ constexpr int cn_harm(int lam) { return (lam + 1) * (lam + 1); }
__host__ __device__ constexpr int cn_beta(int lam) {
  int n = 0;
  for (int L = 0; L <= lam; ++L) n += ((lam - L) >> 1) + 1;
  return n;
}
__host__ __device__ constexpr int cn_r(int lam) { return (lam + 1) * (lam + 2) * (lam + 3) / 6; }

template <int LAM, int NCH>
struct CouplingShape {
  static constexpr int nS = cn_harm(LAM), nB = cn_beta(LAM), nR = cn_r(LAM);
  static constexpr int CS = NCH + 2;  // row stride of the nucleus tables (even: 16-byte rows)
  static constexpr size_t smem = sizeof(double) * ((size_t)(nS + nB) * CS + nR + 16);
};

// Harmonic columns: for fixed m the recursion U_{l+1,m} = z U_lm + ng_lm U_{l-1,m} (|m| < l),
// U_{|m|+1,m} = z U_{|m|,m}, runs on its own once the diagonal U_{|m|,+-|m|} is known, and the
// diagonal chain U_{l+1,l+1} = x U_ll - y U_{l,-l}, U_{l+1,-l-1} = y U_ll + x U_{l,-l} is two
// values per level.  Each entry is formed with the same operations as the level-by-level
// recursion, so a split of the columns between warps changes no result.
// Columns m in [M0, M1] of U_lm(u), l <= LAM, into col[h * CS] with h = l^2 + l + m.
template <int LAM, int CS, int M0, int M1>
__device__ __forceinline__ void harmonic_columns(double x, double y, double z, double* col) {
  double dp[LAM + 1], dm[LAM + 1];  // U_{l,l}, U_{l,-l}
  dp[0] = dm[0] = 1.0;
  if constexpr (LAM >= 1) {
    dp[1] = x;
    dm[1] = y;
#pragma unroll
    for (int l = 1; l < LAM; ++l) {
      dp[l + 1] = fma(x, dp[l], -y * dm[l]);
      dm[l + 1] = fma(y, dp[l], x * dm[l]);
    }
  }
#pragma unroll
  for (int m = M0; m <= M1; ++m) {
    const int am = m < 0 ? -m : m;
    double prv = m < 0 ? dm[am] : dp[am];
    col[(am * am + am + m) * CS] = prv;
    if (am + 1 <= LAM) {
      double cur = z * prv;
      col[((am + 1) * (am + 1) + am + 1 + m) * CS] = cur;
#pragma unroll
      for (int l = am + 1; l < LAM; ++l) {
        const double nxt = fma(k_harm.ng[l * l + l + m], prv, z * cur);
        col[((l + 1) * (l + 1) + l + 1 + m) * CS] = nxt;
        prv = cur;
        cur = nxt;
      }
    }
  }
}

// Split point of the harmonic columns between the two warps: warp 0 (which also evaluates the
// Boys values and radial sums) takes m < split, warp 1 takes m >= split, balancing FP64 operations.
__host__ __device__ constexpr int column_split(int lam) {
  const int radial = 5 * 7 + 1 + 3 * lam + 2 * lam + 1 + lam + 2 * (cn_beta(lam) - lam - 1);
  int best = -lam, best_gap = 1 << 30;
  for (int ms = -lam; ms <= lam + 1; ++ms) {
    int w0 = radial, w1 = 0;
    for (int m = -lam; m <= lam; ++m) (m < ms ? w0 : w1) += 2 * (lam - (m < 0 ? -m : m) + 1);
    const int gap = w0 > w1 ? w0 - w1 : w1 - w0;
    if (gap < best_gap) {
      best_gap = gap;
      best = ms;
    }
  }
  return best;
}

// Radial sums of one nucleus into its column bcol of the B table (row stride CS): with T = p |d|^2,
// G_n = Z |d|^n F_n(T) and tau_j = (p |d|)^j / j!, entry (L, k) is |d|^L beta_{L,k}(T) / k! =
// sum_{j<=k} tau_j G_{L+j}, rows in (L, k) order.  s2 = |d|^2, dn = |d|.
template <int LAM, int CS>
__device__ __forceinline__ void radial_column(double p, double s2, double dn, double z,
                                              const double* __restrict__ boys_tab, double* bcol) {
  const double T = p * s2;
  double F[LAM + 1];
  boys_eval(LAM, T, F, 1, boys_tab, k_boys);
  double zp = z;
#pragma unroll
  for (int n = 0; n <= LAM; ++n) {
    F[n] *= zp;
    zp *= dn;
  }
  double tau[LAM / 2 + 1];
  tau[0] = 1.0;
  const double pdn = p * dn;
#pragma unroll
  for (int k = 1; k <= LAM / 2; ++k) tau[k] = tau[k - 1] * pdn * k_boys.inv_int[k];
  int bo = 0;
#pragma unroll
  for (int L = 0; L <= LAM; ++L) {
    double acc = F[L];
    bcol[bo * CS] = acc;
#pragma unroll
    for (int k = 1; k <= (LAM - L) / 2; ++k) {
      acc = fma(tau[k], F[L + k], acc);
      bcol[(bo + k) * CS] = acc;
    }
    bo += (LAM - L) / 2 + 1;
  }
}

// Unit vector e = d/|d| and |d| of an offset d (d = 0 gives e = z and |d| = 0: only L = 0 survives,
// which any unit vector gives).
__device__ __forceinline__ void unit_offset(double dx, double dy, double dz, double& s2, double& dn, double& ex,
                                            double& ey, double& ez) {
  s2 = dx * dx + dy * dy + dz * dz;
  ex = 0.0;
  ey = 0.0;
  ez = 1.0;
  dn = 0.0;
  if (s2 > 0.0) {
    const double ri = rsqrt(s2);
    dn = s2 * ri;
    ex = dx * ri;
    ey = dy * ri;
    ez = dz * ri;
  }
}

// Tables of one nucleus (or point) for the chunk column `lane`: warp 0 writes the radial sums
// |d|^L beta_{L,k}/k! (times the charge z) into column lane of Btab and the harmonic columns m < MS of
// U_LM(d/|d|) into Stab, warp 1 the columns m >= MS.  d is C - P in the pair frame.
template <int LAM, int CS>
__device__ __forceinline__ void point_tables(int wid, int lane, double p, double dx, double dy, double dz, double z,
                                             const double* __restrict__ boys_tab, double* Stab, double* Btab) {
  constexpr int MS = column_split(LAM);
  double s2, dn, ex, ey, ez;
  unit_offset(dx, dy, dz, s2, dn, ex, ey, ez);
  if (wid == 0) {
    radial_column<LAM, CS>(p, s2, dn, z, boys_tab, Btab + lane);
    if constexpr (MS > -LAM) harmonic_columns<LAM, CS, -LAM, MS - 1>(ex, ey, ez, Stab + lane);
  } else {
    if constexpr (MS <= LAM) harmonic_columns<LAM, CS, MS, LAM>(ex, ey, ez, Stab + lane);
  }
}

// C - P in the pair frame for the nucleus at `c` (Q rows, A the a-shell centre, shift = |P - A|).
__device__ __forceinline__ void pair_frame_offset(const double* Q, double Ax, double Ay, double Az, double shift,
                                                  const double* c, double& dx, double& dy, double& dz) {
  const double ux = c[0] - Ax, uy = c[1] - Ay, uz = c[2] - Az;
  dx = Q[0] * ux + Q[1] * uy + Q[2] * uz;
  dy = Q[3] * ux + Q[4] * uy + Q[5] * uz;
  dz = Q[6] * ux + Q[7] * uy + Q[8] * uz - shift;
}

}  // namespace
}  // namespace shgo
