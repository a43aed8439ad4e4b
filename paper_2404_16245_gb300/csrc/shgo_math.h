// Scalar building blocks compiled for both the host (table checks) and the device (kernels).
#pragma once

#include <cuda_runtime.h>

#include "shgo_internal.h"

namespace shgo {

// Real Racah-normalised solid harmonics S_lm(x, y, z) for l = 0..lmax (Eq. 2 with the real
// combination of the library's conventions), written to out[stride * harm_index(l, m)].
// ca/cb/cc are the recursion coefficients of HarmCoef.
template <typename T>
__host__ __device__ inline void solid_harmonics(int lmax, T x, T y, T z, T* out, int stride, const double* ca,
                                                const double* cb, const double* cc) {
  out[0] = T(1);
  if (lmax < 1) return;
  out[stride * 1] = y;
  out[stride * 2] = z;
  out[stride * 3] = x;
  const T r2 = x * x + y * y + z * z;
  for (int l = 1; l < lmax; ++l) {
    const int cur = l * l + l, prv = (l - 1) * (l - 1) + (l - 1), nxt = (l + 1) * (l + 1) + (l + 1);
    const T sll = out[stride * (cur + l)], slml = out[stride * (cur - l)];
    const T c = T(cc[l]);
    out[stride * (nxt + l + 1)] = c * (x * sll - y * slml);
    out[stride * (nxt - l - 1)] = c * (y * sll + x * slml);
    for (int m = -l; m <= l; ++m) {
      const int k = cur + m;
      T v = T(ca[k]) * (z * out[stride * (cur + m)]);
      if (m > -l && m < l) v -= T(cb[k]) * (r2 * out[stride * (prv + m)]);
      out[stride * (nxt + m)] = v;
    }
  }
}

// Unnormalised solid harmonics U_lm(u) = S_lm(u) / N_lm of a unit vector u (|u| = 1), l <= lmax,
// by the one-constant recursion documented with HarmCoef::ng.  Two FP64 operations per entry.
__host__ __device__ inline void solid_harmonics_unit(int lmax, double x, double y, double z, double* out, int stride,
                                                     const double* ng) {
  out[0] = 1.0;
  if (lmax < 1) return;
  out[stride * 1] = y;
  out[stride * 2] = z;
  out[stride * 3] = x;
  for (int l = 1; l < lmax; ++l) {
    const int cur = l * l + l, prv = (l - 1) * (l - 1) + (l - 1), nxt = (l + 1) * (l + 1) + (l + 1);
    const double sll = out[stride * (cur + l)], slml = out[stride * (cur - l)];
    out[stride * (nxt + l + 1)] = fma(x, sll, -y * slml);
    out[stride * (nxt - l - 1)] = fma(y, sll, x * slml);
    out[stride * (nxt - l)] = z * slml;
    out[stride * (nxt + l)] = z * sll;
    for (int m = -l + 1; m < l; ++m) out[stride * (nxt + m)] = fma(ng[cur + m], out[stride * (prv + m)], z * out[stride * (cur + m)]);
  }
}

// Constants of the Boys evaluation: 1/k! for the Taylor weights and 1/(2n+1).
struct BoysConst {
  double inv_fact[kBoysK + 1];
  double inv_odd[kBoysNmax + 2];
  double inv_int[kLamMax + 2];  // 1/k (entry 0 unused)
};

// F_n(T) = int_0^1 u^{2n} exp(-T u^2) du for n = 0..nmax (the Boys function of Eq. 12 and the
// text after it), written to F[n * stride].  Returns exp(-T).
//  T < 40: the grid row nearest to T gives F_{nmax}(T) = sum_k F_{nmax+k}(T_g) (-dT)^k / k!
//          (dF_n/dT = -F_{n+1}) and exp(-T) = exp(-T_g) sum_k (-dT)^k / k!; lower orders come
//          from the stable downward recursion F_n = (2T F_{n+1} + exp(-T)) / (2n+1).
//  T >= 40: F_0 = sqrt(pi/T)/2 (erf(sqrt 40) = 1 to 2e-19) and the upward recursion
//          F_{n+1} = ((2n+1) F_n - exp(-T)) / (2T), stable while 2n+1 < 2T.
__host__ __device__ inline double boys_eval(int nmax, double T, double* F, int stride, const double* tab,
                                            const BoysConst& bc) {
  if (T < kBoysTsw) {
#ifdef __CUDA_ARCH__
    const int g = __double2int_rn(T * kBoysInvH);
#else
    const int g = (int)(T * kBoysInvH + 0.5);
#endif
    const double dT = double(g) * (1.0 / kBoysInvH) - T;  // = -(T - T_g)
    const double* row = tab + (size_t)g * kBoysStride;
    // Horner in dT with the weights dT/k: sum_k c_k dT^k / k! = c_0 + dT/1 (c_1 + dT/2 (c_2 + ...))
    double ftop = row[1 + nmax + kBoysK], ew = 1.0;
#pragma unroll
    for (int k = kBoysK; k >= 1; --k) {
      const double q = dT * bc.inv_int[k];
      ftop = fma(ftop, q, row[nmax + k]);
      ew = fma(ew, q, 1.0);
    }
    const double ex = row[0] * ew;
    F[nmax * stride] = ftop;
    const double t2 = 2.0 * T;
    for (int n = nmax - 1; n >= 0; --n) F[n * stride] = (t2 * F[(n + 1) * stride] + ex) * bc.inv_odd[n];
    return ex;
  }
#ifdef __CUDA_ARCH__
  const double rt = rsqrt(T);
  const double half_rt = 0.5 * __drcp_rn(T);
#else
  const double rt = 1.0 / sqrt(T);
  const double half_rt = 0.5 / T;
#endif
  const double ex = exp(-T);
  F[0] = 0.88622692545275801364908374167057259 * rt;  // sqrt(pi)/2
  for (int n = 0; n < nmax; ++n) F[(n + 1) * stride] = (double(2 * n + 1) * F[n * stride] - ex) * half_rt;
  return ex;
}

const BoysConst& boys_const_host();

}  // namespace shgo
