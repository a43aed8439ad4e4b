// FP32-bulk coupling kernel (step S2 in FP32 arithmetic), one instantiation per Lambda = la + lb and mode.
//
// The quantity is the FP64 kernel's, R'[L,M,k] = 2 pi k! p^{-(k+1)} sum_C Z_C S_LM(d) beta_{L,k}(T) / k!
// (d = C - P in the pair frame), written on dimensionless factors so that every intermediate stays
// inside FP32's exponent range:
//   S_LM(d) beta_{L,k} / k! = p^{-L/2} N_LM U_LM(e) sum_{j<=k} t_j Phi_{L+j},
//   e = d/|d|,  t_j = T^{j/2} / j!,  Phi_n = T^{n/2} F_n(T),
// with p^{-L/2}, N_LM and 2 pi k! p^{-(k+1)} applied in FP64 when the block is written.  The pair-frame
// geometry and the Boys grid stay FP64; everything per nucleus after them (the Boys Taylor step and
// recursions, Phi_n, t_j, the radial sums, the unit-vector harmonics U) and the nucleus sums run as
// FP32 instructions, 64 of which issue for each FP64 one on GB300 (sm_103a).
//
// FF = false (plain): each factor is one FP32 number and the nucleus sums are FMA chains.
// FF = true (compensated): each factor is an unevaluated pair hi + lo of FP32 numbers (48 significant
// bits), formed with error-free transformations -- Knuth's two-sum, Dekker's fast two-sum and the
// FMA two-product -- and the nucleus sums add the exact product hi*hi by two-sum into a (hi, lo)
// accumulator whose lo part also takes the cross terms (the Dot2 scheme of Ogita, Rump and Oishi,
// 2005, on pair inputs).  The Boys values come from the FP64 grid (split into pairs) by the same
// Taylor step and recursions as the FP64 path, run on pairs.
//
// Block = four warps on one primitive pair (two at Lambda <= 8), lane i of each owning nucleus i of a chunk
// of 32: warp 0 evaluates Phi for the nuclei with T < 40, warp 1 for those with T >= 40, and the harmonic
// columns and then the radial rows are split over the warps by a cost model.  Tables S[h][c] and B[b][c]
// (rows of 34 pairs or 36 floats: 16-byte multiples, rows 4 banks apart) feed the sums, where a thread
// takes the R' entries (L, M, k) and (L, M, k + 1) together (one S row, two B rows) or a lone (L, M, k).
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <utility>

#include "shgo_internal.h"
#include "shgo_math.h"

namespace shgo {

namespace {

constexpr int kNch = 32;        // nuclei per chunk
constexpr int kExpN = 2048;     // exp(-g/16) table: T < 128 (beyond, exp(-T) T^{n/2} is below 1e-30 of Phi_n)
constexpr double kTwoPiF = 6.283185307179586476925286766559;

__constant__ float2 f_ng[(kHarmMax + 1) * (kHarmMax + 1)];  // HarmCoef::ng as (hi, lo)
__constant__ float2 f_inv_odd[kBoysNmax + 2];               // 1/(2n+1)
__constant__ float2 f_inv_int[kLamMax + 2];                 // 1/k
__constant__ float2 f_half_sqrt_pi;                         // sqrt(pi)/2

// ------------------------------------------------------------------------------------------------
// Pair ("double-float") arithmetic.  The _rn intrinsics keep the compiler from fusing a product into
// a later sum, which would break the error-free transformations.
// ------------------------------------------------------------------------------------------------
struct ff {
  float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff vmul(ff a, ff b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  return fast_two_sum(p, e);
}
__device__ __forceinline__ ff vmulf(ff a, float b) {  // b exact
  const float p = __fmul_rn(a.h, b);
  const float e = fmaf(a.l, b, fmaf(a.h, b, -p));
  return fast_two_sum(p, e);
}
__device__ __forceinline__ ff vadd(ff a, ff b) {
  float s, t;
  two_sum(a.h, b.h, s, t);
  return fast_two_sum(s, __fadd_rn(t, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ ff vfma(ff a, ff b, ff c) {  // a b + c
  const float p = __fmul_rn(a.h, b.h);
  const float pe = fmaf(a.h, b.h, -p);
  float s, t;
  two_sum(p, c.h, s, t);
  const float lo = __fadd_rn(fmaf(a.h, b.l, fmaf(a.l, b.h, pe)), c.l);
  return fast_two_sum(s, __fadd_rn(t, lo));
}
__device__ __forceinline__ ff vdot2(ff a, ff b, ff c, ff d) {  // a b + c d
  const float p = __fmul_rn(a.h, b.h), q = __fmul_rn(c.h, d.h);
  const float pe = fmaf(a.h, b.h, -p), qe = fmaf(c.h, d.h, -q);
  float s, t;
  two_sum(p, q, s, t);
  const float lo = __fadd_rn(fmaf(a.h, b.l, fmaf(a.l, b.h, pe)), fmaf(c.h, d.l, fmaf(c.l, d.h, qe)));
  return fast_two_sum(s, __fadd_rn(t, lo));
}
__device__ __forceinline__ ff vneg(ff a) { return {-a.h, -a.l}; }
__device__ __forceinline__ ff vhalf(ff a) { return {0.5f * a.h, 0.5f * a.l}; }
__device__ __forceinline__ float vhi(ff a) { return a.h; }

__device__ __forceinline__ float vmul(float a, float b) { return a * b; }
__device__ __forceinline__ float vmulf(float a, float b) { return a * b; }
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float vdot2(float a, float b, float c, float d) { return fmaf(a, b, c * d); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float vhalf(float a) { return 0.5f * a; }
__device__ __forceinline__ float vhi(float a) { return a; }

// Conversions between FP64 and FP32 by integer operations (FP64-pipe conversions issue at the FP64
// rate).  double -> pair: hi is x with its low 29 fraction bits cleared, lo those bits rounded to a
// float, so hi + lo carries 48 significant bits; |x| below 2^-126 gives 0.  float -> double: exact
// for normal floats, zero and subnormals give (signed) 0.
__device__ __forceinline__ ff d2ff(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int ef = (int)((b >> 52) & 0x7ff) - 896;  // biased FP32 exponent
  if (ef <= 0) return {0.f, 0.f};
  if (ef >= 255) return {__uint_as_float(sign | 0x7f800000u), 0.f};
  const float h = __uint_as_float(sign | ((unsigned)ef << 23) | (unsigned)((b >> 29) & 0x7fffffu));
  const float scale = __uint_as_float((unsigned)ef << 23);  // 2^(ef - 127)
  const float l = __fmul_rn(__fmul_rn(__uint2float_rn((unsigned)(b & 0x1fffffffu)), 0x1p-52f), scale);
  return {h, __uint_as_float(__float_as_uint(l) | sign)};
}
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long e64 = ex == 0xffu ? 0x7ffull : (unsigned long long)(ex + 896u);
  const unsigned long long bits = sign | (e64 << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)(ex == 0 ? sign : bits));
}

template <typename V>
__device__ __forceinline__ V vfrom(double x);
template <>
__device__ __forceinline__ ff vfrom<ff>(double x) {
  return d2ff(x);
}
template <>
__device__ __forceinline__ float vfrom<float>(double x) {
  return __double2float_rn(x);
}
template <typename V>
__device__ __forceinline__ V vc(float2 c);
template <>
__device__ __forceinline__ ff vc<ff>(float2 c) {
  return {c.x, c.y};
}
template <>
__device__ __forceinline__ float vc<float>(float2 c) {
  return c.x;
}
template <typename V>
__device__ __forceinline__ V vf(float x) {
  return vc<V>(make_float2(x, 0.f));
}

// 1/x and sqrt(x), x > 0: the correctly rounded FP32 value refined by one Newton step on the pair.
__device__ __forceinline__ ff vrcp(ff x) {
  const float r = __frcp_rn(x.h);
  const float t = fmaf(-x.l, r, fmaf(-x.h, r, 1.0f));  // 1 - x r, small
  return fast_two_sum(r, r * t);
}
__device__ __forceinline__ float vrcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ ff vrsqrt(ff x) {
  const float r = __frsqrt_rn(x.h);
  const float yh = __fmul_rn(r, r), yl = fmaf(r, r, -yh);
  const float t = fmaf(-x.l, yh, fmaf(-x.h, yl, fmaf(-x.h, yh, 1.0f)));  // 1 - x r^2, small
  return fast_two_sum(r, 0.5f * r * t);
}
__device__ __forceinline__ float vrsqrt(float x) { return __frsqrt_rn(x); }
__device__ __forceinline__ ff vsqrt(ff x) {
  const float r = __frsqrt_rn(x.h);
  const float s = __fmul_rn(x.h, r);
  const float t = __fadd_rn(fmaf(-s, s, x.h), x.l);  // x - s^2, small
  return fast_two_sum(s, 0.5f * r * t);
}
__device__ __forceinline__ float vsqrt(float x) { return __fsqrt_rn(x); }

// Store into column `lane` of table row `row` (RS floats per row; a pair takes two floats).
__device__ __forceinline__ void vstore(float* tab, int rs, int row, int lane, ff v) {
  reinterpret_cast<float2*>(tab + row * rs)[lane] = make_float2(v.h, v.l);
}
__device__ __forceinline__ void vstore(float* tab, int rs, int row, int lane, float v) { tab[row * rs + lane] = v; }

// ------------------------------------------------------------------------------------------------
// Shapes
// ------------------------------------------------------------------------------------------------
__host__ __device__ constexpr int pair_items(int lam) {
  int n = 0;
  for (int L = 0; L <= lam; ++L) n += (2 * L + 1) * ((kmax_of(lam, L) + 1) / 2);
  return n;
}
__host__ __device__ constexpr int single_items(int lam) {
  int n = 0;
  for (int L = 0; L <= lam; ++L) n += (2 * L + 1) * ((kmax_of(lam, L) + 1) & 1);
  return n;
}

template <int LAM, bool FF>
struct F32Shape {
  static constexpr int nS = n_harm(LAM), nB = n_beta(LAM), nR = n_r(LAM);
  static constexpr int RS = FF ? 2 * (kNch + 2) : kNch + 4;  // floats per table row
  static constexpr int PER = FF ? 2 : 4;                     // nuclei per 16-byte load
  static constexpr int nPair = pair_items(LAM), nSingle = single_items(LAM);
  static constexpr int nScl = LAM / 2 + 1 + LAM + 1 + nB;
  static constexpr size_t smem = sizeof(float) * (size_t)(nS + nB + LAM + 1) * RS + sizeof(double) * nScl +
                                 sizeof(float2) * 14 + (FF ? 8 : 4) * (size_t)nR + 16;
};

// Work split of the table phase (costs in FP32 instructions per nucleus: a pair step about 20, a plain
// one 2).  Phase A: warp 0 evaluates Phi for the nuclei with T < 40, warp 1 for those with T >= 40,
// and the harmonic columns are split by |m| over the four warps so that the totals even out (warp w
// takes |m| in [col_bound(w), col_bound(w + 1))).  Phase B: the radial sums, rows L split over the
// four warps (warp w takes L in [row_bound(w), row_bound(w + 1))).
__host__ __device__ constexpr int col_cost(int lam, int a0, int a1, bool fp) {
  if (a1 <= a0) return 0;
  const int per = fp ? 20 : 2;
  int c = 2 * per * a1;  // the diagonal chain up to a1
  for (int am = a0; am < a1; ++am) c += per * (lam - am + 1) * (am > 0 ? 2 : 1);
  return c;
}
__host__ __device__ constexpr int col_bound(int lam, int w, bool fp) {
  if (w <= 0) return 0;
  if (w >= 4) return lam + 1;
  const int small = fp ? 300 + 37 * lam : 30 + 4 * lam;  // Phi for T < 40 (warp 0)
  const int large = fp ? 180 + 31 * lam : 20 + 4 * lam;  // Phi for T >= 40 (warp 1)
  int bb[4] = {0, 0, 0, 0}, best = 1 << 30;
  for (int b1 = 0; b1 <= lam + 1; ++b1)
    for (int b2 = b1; b2 <= lam + 1; ++b2)
      for (int b3 = b2; b3 <= lam + 1; ++b3) {
        const int c0 = small + col_cost(lam, 0, b1, fp), c1 = large + col_cost(lam, b1, b2, fp);
        const int c2 = col_cost(lam, b2, b3, fp), c3 = col_cost(lam, b3, lam + 1, fp);
        int mx = c0 > c1 ? c0 : c1;
        mx = mx > c2 ? mx : c2;
        mx = mx > c3 ? mx : c3;
        if (mx < best) {
          best = mx;
          bb[1] = b1;
          bb[2] = b2;
          bb[3] = b3;
        }
      }
  return bb[w];
}
// The same splits for two warps (small Lambda): warp 0 Phi for T < 40 and the columns below the bound,
// warp 1 Phi for T >= 40 and the rest; the radial rows halved.
__host__ __device__ constexpr int col_bound2(int lam, int w, bool fp) {
  if (w <= 0) return 0;
  if (w >= 2) return lam + 1;
  const int small = fp ? 300 + 37 * lam : 30 + 4 * lam;
  const int large = fp ? 180 + 31 * lam : 20 + 4 * lam;
  int best = 1 << 30, bb = 0;
  for (int b1 = 0; b1 <= lam + 1; ++b1) {
    const int c0 = small + col_cost(lam, 0, b1, fp), c1 = large + col_cost(lam, b1, lam + 1, fp);
    const int mx = c0 > c1 ? c0 : c1;
    if (mx < best) {
      best = mx;
      bb = b1;
    }
  }
  return bb;
}
__host__ __device__ constexpr int row_bound2(int lam, int w) {
  if (w <= 0) return 0;
  if (w >= 2) return lam + 1;
  const int total = n_beta(lam);
  int L = 0, acc = 0;
  while (L <= lam && 2 * (acc + kmax_of(lam, L) + 1) <= total + 1) acc += kmax_of(lam, L++) + 1;
  return L;
}
__host__ __device__ constexpr int row_bound(int lam, int w) {
  if (w <= 0) return 0;
  if (w >= 4) return lam + 1;
  const int total = n_beta(lam);
  int L = 0, acc = 0;
  while (L <= lam && 4 * (acc + kmax_of(lam, L) + 1) <= w * total + 2) acc += kmax_of(lam, L++) + 1;
  return L;
}

// Columns m = +-am, am in [A0, A1), of U_lm(e), l <= LAM (the FP64 kernel's recursion: U_{l+1,m} =
// z U_lm + ng_lm U_{l-1,m}, U_{|m|+1,m} = z U_{|m|,m}, diagonal U_{l+1,l+1} = x U_ll - y U_{l,-l},
// U_{l+1,-l-1} = y U_ll + x U_{l,-l}) into table rows h = l^2 + l + m, column lane.  The diagonal
// chain runs from am = 0; the two columns of one am advance together (two independent chains), as
// loops so that the code stays small.
template <typename V, int LAM, int RS>
__device__ __forceinline__ void harmonic_pairs(int A0, int A1, V x, V y, V z, float* tab, int lane) {
  V dp = vf<V>(1.0f), dm = vf<V>(0.0f);  // U_{am,am}, U_{am,-am}
  const V ny = vneg(y);
#pragma unroll 1
  for (int am = 0; am < A1; ++am) {
    if (am >= A0) {
      V pp = dp, pm = dm;
      vstore(tab, RS, am * am + 2 * am, lane, pp);
      if (am > 0) vstore(tab, RS, am * am, lane, pm);
      if (am + 1 <= LAM) {
        V cp = vmul(z, pp), cm = vmul(z, pm);
        const int h1 = (am + 1) * (am + 2);  // row of (am + 1, 0)
        vstore(tab, RS, h1 + am, lane, cp);
        if (am > 0) vstore(tab, RS, h1 - am, lane, cm);
#pragma unroll 2
        for (int l = am + 1; l < LAM; ++l) {
          const int h = l * l + l, hn = (l + 1) * (l + 2);
          const V np = vdot2(vc<V>(f_ng[h + am]), pp, z, cp);
          vstore(tab, RS, hn + am, lane, np);
          pp = cp;
          cp = np;
          if (am > 0) {
            const V nm = vdot2(vc<V>(f_ng[h - am]), pm, z, cm);
            vstore(tab, RS, hn - am, lane, nm);
            pm = cm;
            cm = nm;
          }
        }
      }
    }
    if (am == 0) {
      dp = x;
      dm = y;
    } else {
      const V t = vdot2(x, dp, ny, dm);
      dm = vdot2(y, dp, x, dm);
      dp = t;
    }
  }
}

// exp(dT) = sum_k dT^k / k! and, alongside, F_top(T) = sum_k F_{top+k}(T_g) dT^k / k! (dF_n/dT = -F_{n+1},
// dT = T_g - T), Horner with the weights dT/k; row[0] = exp(-T_g), row[1 + n] = F_n(T_g).
template <typename V, int TOP>
__device__ __forceinline__ void boys_taylor(V dT, const float2* __restrict__ row, V& ftop, V& ew) {
  ftop = vc<V>(__ldg(row + 1 + TOP + kBoysK));
  ew = vf<V>(1.0f);
#pragma unroll
  for (int k = kBoysK; k >= 1; --k) {
    const V q = vmul(dT, vc<V>(f_inv_int[k]));
    ftop = vfma(ftop, q, vc<V>(__ldg(row + TOP + k)));
    ew = vfma(ew, q, vf<V>(1.0f));
  }
}

// Phi_n = Z T^{n/2} F_n(T), n = 0..LAM, into row n of the Phi table (column lane).
//  T < 40: F_LAM and exp(-T) by the Taylor step about the nearest grid point, the downward recursion
//          F_n = (2T F_{n+1} + exp(-T)) / (2n+1), then the factor Z st^n (st = sqrt T < 6.33).
//  T >= 40: in scaled form, Phi_0 = Z sqrt(pi)/2 / st and the upward recursion
//          Phi_{n+1} = ((2n+1) Phi_n - E_n) / (2 st),  E_n = Z st^n exp(-T)
//          (F_{n+1} = ((2n+1) F_n - exp(-T)) / (2T) times T^{(n+1)/2}); exp(-T) = exp(-T_g) exp(dT)
//          from the table of exp(-g/16), zero past T = 128.
// Near T = 40 either form holds: the grid reaches T = 40 + 1/32 and the upward recursion is stable.
template <typename V, int LAM, int RS>
__device__ __forceinline__ void phi_small(V T, V st, V Z, const float2* __restrict__ boys_ff, float* Ptab,
                                          int lane) {
  const int g = __float2int_rn(vhi(T) * (float)kBoysInvH);
  const V dT = vadd(vf<V>((float)g * (float)(1.0 / kBoysInvH)), vneg(T));
  V ftop, ew;
  const float2* row = boys_ff + (size_t)g * kBoysStride;
  boys_taylor<V, LAM>(dT, row, ftop, ew);
  const V ex = vmul(vc<V>(__ldg(row)), ew);
  const V T2 = vmulf(T, 2.0f);
  V F[LAM + 1];
  F[LAM] = ftop;
#pragma unroll
  for (int n = LAM - 1; n >= 0; --n) F[n] = vmul(vfma(T2, F[n + 1], ex), vc<V>(f_inv_odd[n]));
  V P = Z;
#pragma unroll
  for (int n = 0; n <= LAM; ++n) {
    vstore(Ptab, RS, n, lane, vmul(F[n], P));
    if (n < LAM) P = vmul(P, st);
  }
}

template <typename V, int LAM, int RS>
__device__ __forceinline__ void phi_large(V T, V st, V Z, const float2* __restrict__ exp_ff, float* Ptab,
                                          int lane) {
  const int g = __float2int_rn(vhi(T) * (float)kBoysInvH);
  const V rst = vrcp(st);
  V phi = vmul(Z, vmul(vc<V>(f_half_sqrt_pi), rst));
  V E = vf<V>(0.0f);
  if (g < kExpN) {
    const V dT = vadd(vf<V>((float)g * (float)(1.0 / kBoysInvH)), vneg(T));
    V ew = vf<V>(1.0f);
#pragma unroll
    for (int k = kBoysK; k >= 1; --k) ew = vfma(ew, vmul(dT, vc<V>(f_inv_int[k])), vf<V>(1.0f));
    E = vmul(Z, vmul(vc<V>(__ldg(exp_ff + g)), ew));
  }
  const V h = vhalf(rst);
  vstore(Ptab, RS, 0, lane, phi);
#pragma unroll
  for (int n = 0; n < LAM; ++n) {
    phi = vmul(vadd(vmulf(phi, (float)(2 * n + 1)), vneg(E)), h);
    vstore(Ptab, RS, n + 1, lane, phi);
    E = vmul(E, st);
  }
}

template <typename V>
__device__ __forceinline__ V vload(const float* tab, int rs, int row, int lane);
template <>
__device__ __forceinline__ ff vload<ff>(const float* tab, int rs, int row, int lane) {
  const float2 v = reinterpret_cast<const float2*>(tab + row * rs)[lane];
  return {v.x, v.y};
}
template <>
__device__ __forceinline__ float vload<float>(const float* tab, int rs, int row, int lane) {
  return tab[row * rs + lane];
}

// Radial sums B[L,k] = sum_{j<=k} t_j Phi_{L+j} (t_j = st^j / j!) of rows L in [L0, L1) into Btab.
template <typename V, int LAM, int RS>
__device__ __forceinline__ void radial_rows(int L0, int L1, V st, const float* Ptab, float* Btab, int lane) {
  V tj[LAM / 2 + 1];
  tj[0] = vf<V>(1.0f);
#pragma unroll
  for (int j = 1; j <= LAM / 2; ++j) tj[j] = vmul(tj[j - 1], vmul(st, vc<V>(f_inv_int[j])));
  int bo = 0;
#pragma unroll
  for (int L = 0; L <= LAM; ++L) {
    if (L >= L0 && L < L1) {
      V acc = vload<V>(Ptab, RS, L, lane);
      vstore(Btab, RS, bo, lane, acc);
#pragma unroll
      for (int k = 1; k <= (LAM - L) / 2; ++k) {
        acc = vfma(tj[k], vload<V>(Ptab, RS, L + k, lane), acc);
        vstore(Btab, RS, bo + k, lane, acc);
      }
    }
    bo += (LAM - L) / 2 + 1;
  }
}

// Pair form of an FP64 value for the per-primitive-pair constants (plain: the rounded float).
template <bool FF>
__device__ __forceinline__ float2 to_pair(double x) {
  if constexpr (FF) {
    const ff v = d2ff(x);
    return make_float2(v.h, v.l);
  } else {
    return make_float2(__double2float_rn(x), 0.f);
  }
}

// ------------------------------------------------------------------------------------------------
// Nucleus sums
// ------------------------------------------------------------------------------------------------
// (ah, al) += (sh + sl)(bh + bl): the exact product of the high parts by FMA, added by two-sum; its
// rounding error, the cross terms and the sum's error go to al.
__device__ __forceinline__ void ff_acc(float2& a, float sh, float sl, float bh, float bl) {
  const float p = __fmul_rn(sh, bh);
  const float e = fmaf(sl, bh, fmaf(sh, bl, fmaf(sh, bh, -p)));
  float s, t;
  two_sum(a.x, p, s, t);
  a.y = __fadd_rn(a.y, __fadd_rn(t, e));
  a.x = s;
}
__device__ __forceinline__ void ff_merge(float2& a, float2 b) {
  float s, t;
  two_sum(a.x, b.x, s, t);
  a.y = __fadd_rn(a.y, __fadd_rn(t, b.y));
  a.x = s;
}

// Entries (e0, e0 + 1) = (L, M, k), (L, M, k + 1): one S row, B rows b and b + 1.
template <bool FF, int RS>
__device__ __forceinline__ void sum_pair(const float* S_, const float* B_, int nit, float2* racc2, float* racc1,
                                         int e0) {
  const float4* S = reinterpret_cast<const float4*>(S_);
  const float4* B0 = reinterpret_cast<const float4*>(B_);
  const float4* B1 = reinterpret_cast<const float4*>(B_ + RS);
  if constexpr (FF) {
    float2 a0 = racc2[e0], a1 = racc2[e0 + 1];
    auto step = [&](int c) {
      const float4 s = S[c], b0 = B0[c], b1 = B1[c];
      ff_acc(a0, s.x, s.y, b0.x, b0.y);
      ff_acc(a1, s.x, s.y, b1.x, b1.y);
      ff_acc(a0, s.z, s.w, b0.z, b0.w);
      ff_acc(a1, s.z, s.w, b1.z, b1.w);
    };
#pragma unroll 4
    for (int c = 0; c < nit; ++c) step(c);
    racc2[e0] = a0;
    racc2[e0 + 1] = a1;
  } else {
    float a0 = 0.f, a1 = 0.f, c0 = 0.f, c1 = 0.f;
    auto step = [&](int c) {
      const float4 s = S[c], b0 = B0[c], b1 = B1[c];
      a0 = fmaf(s.x, b0.x, fmaf(s.y, b0.y, a0));
      a1 = fmaf(s.x, b1.x, fmaf(s.y, b1.y, a1));
      c0 = fmaf(s.z, b0.z, fmaf(s.w, b0.w, c0));
      c1 = fmaf(s.z, b1.z, fmaf(s.w, b1.w, c1));
    };
#pragma unroll 4
    for (int c = 0; c < nit; ++c) step(c);
    racc1[e0] += a0 + c0;
    racc1[e0 + 1] += a1 + c1;
  }
}

template <bool FF>
__device__ __forceinline__ void sum_single(const float* S_, const float* B_, int nit, float2* racc2, float* racc1,
                                           int e0) {
  const float4* S = reinterpret_cast<const float4*>(S_);
  const float4* B0 = reinterpret_cast<const float4*>(B_);
  if constexpr (FF) {
    float2 a0 = racc2[e0], a1 = make_float2(0.f, 0.f);
    auto step = [&](int c) {
      const float4 s = S[c], b0 = B0[c];
      ff_acc(a0, s.x, s.y, b0.x, b0.y);
      ff_acc(a1, s.z, s.w, b0.z, b0.w);
    };
#pragma unroll 4
    for (int c = 0; c < nit; ++c) step(c);
    ff_merge(a0, a1);
    racc2[e0] = a0;
  } else {
    float a0 = 0.f, c0 = 0.f;
    auto step = [&](int c) {
      const float4 s = S[c], b0 = B0[c];
      a0 = fmaf(s.x, b0.x, fmaf(s.y, b0.y, a0));
      c0 = fmaf(s.z, b0.z, fmaf(s.w, b0.w, c0));
    };
#pragma unroll 4
    for (int c = 0; c < nit; ++c) step(c);
    racc1[e0] += a0 + c0;
  }
}

template <int LAM, bool FF, int NW>
__global__ void __launch_bounds__(32 * NW) k_coupling_f32(CouplingArgs A) {
  constexpr int NT = 32 * NW;  // four warps, or two at small Lambda (the same operations per entry)
  using Sh = F32Shape<LAM, FF>;
  using V = std::conditional_t<FF, ff, float>;
  constexpr int nS = Sh::nS, nB = Sh::nB, nR = Sh::nR, RS = Sh::RS;
  extern __shared__ __align__(16) float fsm[];
  float* Stab = fsm;                                            // [nS][RS] U_LM(e)
  float* Btab = Stab + nS * RS;                                 // [nB][RS] radial sums
  float* Ptab = Btab + nB * RS;                                 // [LAM + 1][RS] Phi_n
  double* sclk = reinterpret_cast<double*>(Ptab + (LAM + 1) * RS);  // [LAM/2 + 1] 2 pi k! p^{-(k+1)}
  double* sclL = sclk + LAM / 2 + 1;                            // [LAM + 1] p^{-L/2}
  double* sclb = sclL + LAM + 1;                                // [nB] their product for beta row b
  float2* geo = reinterpret_cast<float2*>(sclb + nB);           // [14] A, Q, |P - A|, p as pairs
  float2* racc2 = geo + 14;                                     // [nR] (FF)
  float* racc1 = reinterpret_cast<float*>(geo + 14);            // [nR] (plain)
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int cb1 = NW == 4 ? col_bound(LAM, 1, FF) : col_bound2(LAM, 1, FF);
  constexpr int cb2 = NW == 4 ? col_bound(LAM, 2, FF) : LAM + 1, cb3 = NW == 4 ? col_bound(LAM, 3, FF) : LAM + 1;
  constexpr int rb1 = NW == 4 ? row_bound(LAM, 1) : row_bound2(LAM, 1);
  constexpr int rb2 = NW == 4 ? row_bound(LAM, 2) : LAM + 1, rb3 = NW == 4 ? row_bound(LAM, 3) : LAM + 1;
  const int a0 = wid == 0 ? 0 : (wid == 1 ? cb1 : (wid == 2 ? cb2 : cb3));
  const int a1 = wid == 0 ? cb1 : (wid == 1 ? cb2 : (wid == 2 ? cb3 : LAM + 1));
  const int L0 = wid == 0 ? 0 : (wid == 1 ? rb1 : (wid == 2 ? rb2 : rb3));
  const int L1 = wid == 0 ? rb1 : (wid == 1 ? rb2 : (wid == 2 ? rb3 : LAM + 1));
  __shared__ long long s_next[2];
  __shared__ unsigned long long s_t0;
  wq_for_each(A.q, A.npp, s_next, &s_t0, [&](long long w) {
    const int64_t q = A.pp_base + w;
    const int pr = A.pp_pair[q];
    const PPData pd = A.ppd[q];
    // primitive pairs with a zero prefactor are skipped by the pair kernel too
    if (pd.pref == 0.0) return;
    __syncthreads();  // the previous primitive pair is done with racc, the scales and geo
    if (tid < 3) {
      geo[tid] = to_pair<FF>(A.shell_xyz[3 * A.pair_a[pr] + tid]);
    } else if (tid < 12) {
      geo[tid] = to_pair<FF>(A.site_rot[9 * A.pair_site[pr] + tid - 3]);
    } else if (tid == 12) {
      geo[12] = to_pair<FF>(pd.shift);
    } else if (tid == 13) {
      geo[13] = to_pair<FF>(pd.p);
    }
    for (int e = tid; e < nR; e += NT) {
      if constexpr (FF)
        racc2[e] = make_float2(0.f, 0.f);
      else
        racc1[e] = 0.f;
    }
    int64_t cbeg, ncen;
    mol_centers(A.mv, pr, cbeg, ncen);
    for (int64_t c0 = 0; c0 < ncen; c0 += kNch) {
      __syncthreads();  // the tables of the previous chunk are consumed; geo is written
      // Phase A: C - P in the pair frame, T, Phi (warps 0 and 1 by the size of T), harmonic columns
      V st;
      {
        V dx = vf<V>(0.0f), dy = dx, dz = dx, z = dx;
        if (c0 + lane < ncen) {
          const int64_t c = mol_center_index(A.mv, cbeg + c0 + lane);
          // C - P = Q (C - A) - |P - A| e_z: exact for a nucleus on the a-shell centre
          const V ux = vadd(vfrom<V>(A.centers[3 * c]), vneg(vc<V>(geo[0])));
          const V uy = vadd(vfrom<V>(A.centers[3 * c + 1]), vneg(vc<V>(geo[1])));
          const V uz = vadd(vfrom<V>(A.centers[3 * c + 2]), vneg(vc<V>(geo[2])));
          dx = vadd(vdot2(vc<V>(geo[3]), ux, vc<V>(geo[4]), uy), vmul(vc<V>(geo[5]), uz));
          dy = vadd(vdot2(vc<V>(geo[6]), ux, vc<V>(geo[7]), uy), vmul(vc<V>(geo[8]), uz));
          dz = vadd(vadd(vdot2(vc<V>(geo[9]), ux, vc<V>(geo[10]), uy), vmul(vc<V>(geo[11]), uz)),
                    vneg(vc<V>(geo[12])));
          z = vfrom<V>(A.charges[c]);
        }
        const V s2 = vfma(dx, dx, vfma(dy, dy, vmul(dz, dz)));
        const V T = vmul(vc<V>(geo[13]), s2);
        st = vhi(T) > 0.0f ? vsqrt(T) : vf<V>(0.0f);
        const bool small = vhi(T) < (float)kBoysTsw;
        if (wid == 0 && small) phi_small<V, LAM, RS>(T, st, z, A.boys_ff, Ptab, lane);
        if (wid == 1 && !small) phi_large<V, LAM, RS>(T, st, z, A.exp_ff, Ptab, lane);
        if (a1 > a0) {
          // unit vector of d; d = 0 gives (0, 0, 1), which only the L = 0 entry sees
          V ex = vf<V>(0.0f), ey = ex, ez = vf<V>(1.0f);
          if (vhi(s2) > 0.0f) {
            const V ri = vrsqrt(s2);
            ex = vmul(dx, ri);
            ey = vmul(dy, ri);
            ez = vmul(dz, ri);
          }
          harmonic_pairs<V, LAM, RS>(a0, a1, ex, ey, ez, Stab, lane);
        }
      }
      __syncthreads();
      // Phase B: radial sums
      radial_rows<V, LAM, RS>(L0, L1, st, Ptab, Btab, lane);
      __syncthreads();
      // Phase C: nucleus sums; a partial last chunk sums only its occupied columns (empty ones hold
      // Z = 0 radial sums)
      const int nv = ncen - c0 >= kNch ? kNch : (int)(ncen - c0);
      const int nit = (nv + Sh::PER - 1) / Sh::PER;
      for (int i = tid; i < Sh::nPair; i += NT) {
        const int e0 = __ldg(A.items + i);
        const int code = __ldg(A.rmap + e0);
        sum_pair<FF, RS>(Stab + (code & 0xfff) * RS, Btab + ((code >> 12) & 0xfff) * RS, nit, racc2, racc1, e0);
      }
      for (int i = Sh::nPair + tid; i < Sh::nPair + Sh::nSingle; i += NT) {
        const int e0 = __ldg(A.items + i);
        const int code = __ldg(A.rmap + e0);
        sum_single<FF>(Stab + (code & 0xfff) * RS, Btab + ((code >> 12) & 0xfff) * RS, nit, racc2, racc1, e0);
      }
    }
    // scales 2 pi k! p^{-(k+1)} and p^{-L/2} (FP64: their range exceeds FP32's), per beta row b = (L, k)
    if (wid == 1 && lane <= LAM / 2) {
      double s = kTwoPiF * pd.rp;
      for (int k = 1; k <= lane; ++k) s *= double(k) * pd.rp;
      sclk[lane] = s;
    }
    if (wid == 0 && lane <= LAM) {
      const double ip = pd.sp * pd.rp;  // p^{-1/2}
      double s = 1.0;
      for (int k = 0; k < lane; ++k) s *= ip;
      sclL[lane] = s;
    }
    __syncthreads();
    for (int b = tid; b < nB; b += NT) {
      int L = 0, bo = 0;
      while (bo + kmax_of(LAM, L) + 1 <= b) bo += kmax_of(LAM, L++) + 1;
      sclb[b] = sclk[b - bo] * sclL[L];
    }
    __syncthreads();
    // out = R' N_LM (pair product) x scale (FP64)
    double* out = A.rbuf + A.rbase + w * (int64_t)nR;
    for (int e = tid; e < nR; e += NT) {
      const int code = __ldg(A.rmap + e);
      double v;
      if constexpr (FF) {
        const ff r = vmul(ff{racc2[e].x, racc2[e].y}, vc<ff>(__ldg(A.rnorm_ff + e)));
        v = f2d(r.h) + f2d(r.l);
      } else {
        v = f2d(racc1[e] * __ldg(A.rnorm_ff + e).x);
      }
      out[e] = v * sclb[(code >> 12) & 0xfff];
    }
    });
}

using Kernel = void (*)(CouplingArgs);

template <bool FF, int NW, int... L>
constexpr Kernel kernel_at(int lam, std::integer_sequence<int, L...>) {
  Kernel k = nullptr;
  ((lam == L ? (k = &k_coupling_f32<L, FF, NW>, 0) : 0), ...);
  return k;
}

// Two warps per block up to Lambda = 8 (measured: the batched workload 6 % faster, the high-l molecule 1.5 %),
// for the bases that allow the smaller blocks (CouplingArgs::one_warp_ok).
constexpr int kTwoWarpLamMax = 8;
int f32_warps(int lam, bool small_ok) { return small_ok && lam <= kTwoWarpLamMax ? 2 : 4; }

template <bool FF, int... L>
constexpr size_t smem_at(int lam, std::integer_sequence<int, L...>) {
  size_t s = 0;
  ((lam == L ? (s = F32Shape<L, FF>::smem, 0) : 0), ...);
  return s;
}

using Lams = std::make_integer_sequence<int, kLamMax + 1>;

float2 split(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

}  // namespace

size_t coupling_f32_smem(int lam, bool compensated) {
  if (lam < 0 || lam > kLamMax) return 0;
  return compensated ? smem_at<true>(lam, Lams{}) : smem_at<false>(lam, Lams{});
}

std::vector<float2> boys_table_pairs(const std::vector<double>& boys) {
  std::vector<float2> out(boys.size());
  for (size_t i = 0; i < boys.size(); ++i) out[i] = split(boys[i]);
  return out;
}

std::vector<float2> pairs_of(const std::vector<double>& v) { return boys_table_pairs(v); }

std::vector<int> coupling_f32_items(const std::vector<int>& rmap_off) {
  std::vector<int> items(rmap_off.back(), 0);
  for (int lam = 0; lam <= kLamMax; ++lam) {
    int* it = items.data() + rmap_off[lam];
    int np = 0, ns = pair_items(lam), e = 0;
    for (int L = 0; L <= lam; ++L) {
      const int km = kmax_of(lam, L);
      for (int M = -L; M <= L; ++M) {
        for (int k = 0; k + 1 <= km; k += 2) it[np++] = e + k;
        if ((km + 1) & 1) it[ns++] = e + km;
        e += km + 1;
      }
    }
  }
  return items;
}

std::vector<float2> exp_table_pairs() {
  std::vector<float2> out(kExpN);
  for (int g = 0; g < kExpN; ++g) out[g] = split(std::exp(-(double)g / kBoysInvH));
  return out;
}

cudaError_t coupling_f32_setup() {
  const HarmCoef& hc = harm_coef_host();
  const BoysConst& bc = boys_const_host();
  float2 ng[(kHarmMax + 1) * (kHarmMax + 1)], io[kBoysNmax + 2], ii[kLamMax + 2];
  for (int i = 0; i < (kHarmMax + 1) * (kHarmMax + 1); ++i) ng[i] = split(hc.ng[i]);
  for (int i = 0; i < kBoysNmax + 2; ++i) io[i] = split(bc.inv_odd[i]);
  for (int i = 0; i < kLamMax + 2; ++i) ii[i] = split(i == 0 ? 0.0 : bc.inv_int[i]);
  const float2 hsp = split(0.88622692545275801364908374167057259);
  cudaError_t e = cudaMemcpyToSymbol(f_ng, ng, sizeof(ng));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(f_inv_odd, io, sizeof(io));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(f_inv_int, ii, sizeof(ii));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(f_half_sqrt_pi, &hsp, sizeof(hsp));
  for (int lam = 0; lam <= kLamMax && e == cudaSuccess; ++lam) {
    e = set_max_dynamic_smem((const void*)kernel_at<true, 4>(lam, Lams{}));
    if (e == cudaSuccess) e = set_max_dynamic_smem((const void*)kernel_at<false, 4>(lam, Lams{}));
    if (e == cudaSuccess) e = set_max_dynamic_smem((const void*)kernel_at<true, 2>(lam, Lams{}));
    if (e == cudaSuccess) e = set_max_dynamic_smem((const void*)kernel_at<false, 2>(lam, Lams{}));
  }
  return e;
}

cudaError_t launch_coupling_f32(int lam, bool compensated, const CouplingArgs& args, int grid, cudaStream_t stream) {
  if (lam < 0 || lam > kLamMax || !args.boys_ff || !args.exp_ff || !args.items || !args.rnorm_ff)
    return cudaErrorInvalidValue;
  const int nw = f32_warps(lam, args.one_warp_ok != 0);
  const Kernel k = nw == 2 ? (compensated ? kernel_at<true, 2>(lam, Lams{}) : kernel_at<false, 2>(lam, Lams{}))
                           : (compensated ? kernel_at<true, 4>(lam, Lams{}) : kernel_at<false, 4>(lam, Lams{}));
  // two-warp blocks: twice the blocks
  if (nw == 2) grid = (int)std::min<int64_t>(2 * (int64_t)grid, std::max<int64_t>(args.npp, 1));
  k<<<grid, 32 * nw, coupling_f32_smem(lam, compensated), stream>>>(args);
  return cudaGetLastError();
}

}  // namespace shgo
