// FP64 coupling kernel (step S2), one instantiation per Lambda = la + lb and nucleus-chunk size.
//
// For one primitive pair (one warp) and its nuclei C, in the pair frame with d = C - P:
//   R'[L,M,k] = 2 pi k! p^{-(k+1)} sum_C Z_C S_LM(d) beta_{L,k}(T) / k!,
//   beta_{L,k} / k! = sum_{j<=k} T^j / j! F_{L+j}(T),  T = p |d|^2,
// the radial part of the corrected one-centre integral (Eq. 12 with the same-centre coupling
// restored) before the Clebsch-Gordan coupling of the pair kernel.  S_LM(d) = |d|^L N_LM U_LM(u)
// with u = d/|d|; the |d|^L goes with the radial factors (sum_j tau_j G_{L+j}, tau_j = (p|d|)^j/j!,
// G_n = Z |d|^n F_n) and N_LM with the final scale.
//
// A block of two warps works on one primitive pair.  Lane i of both warps owns nucleus i of a chunk
// of NCH: warp 0 evaluates the Boys values, the radial sums and part of the unit-vector harmonic
// columns, warp 1 the other columns, every loop unrolled (Lambda is a template parameter, so the
// recursions run in registers with their constants as immediate operands); they write column i of
// two shared tables S[h][c] and B[b][c].  Then thread t owns R' entries e = t, t + 64, ...: their
// sums over the chunk's nuclei read both table rows with 16-byte loads at fixed offsets.  Row
// stride NCH + 2 doubles keeps those loads free of bank conflicts.  Two warps per block double
// the warps an SM holds for the same shared memory.  At small Lambda (few harmonic columns and R'
// entries for the second warp) one warp does both halves (NW = 1); every entry is formed by the same
// operations either way.
#include <cuda_runtime.h>

#include <utility>

#include "shgo_internal.h"
#include "shgo_math.h"
#include "shgo_point_tables.cuh"

namespace shgo {

namespace {

template <int NCH, int LAM, int NW>
__global__ void __launch_bounds__(32 * NW) k_coupling_fp64(CouplingArgs A) {
  constexpr int NT = 32 * NW;
  using Sh = CouplingShape<LAM, NCH>;
  constexpr int nS = Sh::nS, nR = Sh::nR, CS = Sh::CS;
  extern __shared__ __align__(16) double smem[];
  double* Stab = smem;             // [nS][CS]
  double* Btab = Stab + nS * CS;   // [nB][CS]
  double* racc = Btab + Sh::nB * CS;
  double* scl = racc + nR;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  __shared__ long long s_next[2];
  __shared__ unsigned long long s_t0;
  wq_for_each(A.q, A.npp, s_next, &s_t0, [&](long long w) {
    const int64_t q = A.pp_base + w;
    const int pr = A.pp_pair[q];
    const int a = A.pair_a[pr];
    const PPData pd = A.ppd[q];
    // primitive pairs with a zero prefactor (K_AB of Eq. 5 underflowed, or the pair is below the
    // per-basis bound) are skipped by the pair kernel too, so their coupling block is not needed
    if (pd.pref == 0.0) return;
    // C - P = (C - A) - (beta/p)(B - A), in the pair frame where B - A is along z
    const double Ax = A.shell_xyz[3 * a], Ay = A.shell_xyz[3 * a + 1], Az = A.shell_xyz[3 * a + 2];
    double Q[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Q[k] = A.site_rot[9 * A.pair_site[pr] + k];
    __syncthreads();  // the previous primitive pair is done with racc and scl
    for (int e = tid; e < nR; e += NT) racc[e] = 0.0;
    int64_t cbeg, ncen;
    mol_centers(A.mv, pr, cbeg, ncen);
    for (int64_t c0 = 0; c0 < ncen; c0 += NCH) {
      __syncthreads();  // the tables of the previous chunk are consumed
      if (lane < NCH) {
        double dx = 0.0, dy = 0.0, dz = 0.0, z = 0.0;
        if (c0 + lane < ncen) {
          const int64_t c = mol_center_index(A.mv, cbeg + c0 + lane);
          pair_frame_offset(Q, Ax, Ay, Az, pd.shift, A.centers + 3 * c, dx, dy, dz);
          z = A.charges[c];
        }
        if (NW == 2) {
          point_tables<LAM, CS>(wid, lane, pd.p, dx, dy, dz, z, A.boys_tab, Stab, Btab);
        } else {  // one warp takes both halves of the tables
          point_tables<LAM, CS>(0, lane, pd.p, dx, dy, dz, z, A.boys_tab, Stab, Btab);
          point_tables<LAM, CS>(1, lane, pd.p, dx, dy, dz, z, A.boys_tab, Stab, Btab);
        }
      }
      __syncthreads();
      // a partial last chunk sums only its occupied columns (rounded up to a pair; empty columns
      // carry Z = 0 and so add exact zeros)
      const int nv2 = ncen - c0 >= NCH ? NCH / 2 : (int)((ncen - c0 + 1) >> 1);
      for (int e = tid; e < nR; e += NT) {
        const int code = __ldg(A.rmap + e);
        const double2* S = reinterpret_cast<const double2*>(Stab + (code & 0xfff) * CS);
        const double2* B = reinterpret_cast<const double2*>(Btab + ((code >> 12) & 0xfff) * CS);
        double a0 = racc[e], a1 = 0.0;
        if (nv2 == NCH / 2) {
#pragma unroll
          for (int c = 0; c < NCH / 2; ++c) {
            const double2 s = S[c], b = B[c];
            a0 = fma(s.x, b.x, a0);
            a1 = fma(s.y, b.y, a1);
          }
        } else {
#pragma unroll 4
          for (int c = 0; c < nv2; ++c) {
            const double2 s = S[c], b = B[c];
            a0 = fma(s.x, b.x, a0);
            a1 = fma(s.y, b.y, a1);
          }
        }
        racc[e] = a0 + a1;
      }
    }
    // scale 2 pi k! p^{-(k+1)} N_LM (each thread scales the entries it accumulated)
    if (tid <= LAM / 2) {
      double s = kTwoPiC * pd.rp;
      for (int k = 1; k <= tid; ++k) s *= double(k) * pd.rp;
      scl[tid] = s;
    }
    __syncthreads();
    double* out = A.rbuf + A.rbase + w * (int64_t)nR;
    for (int e = tid; e < nR; e += NT) out[e] = racc[e] * (scl[(__ldg(A.rmap + e) >> 24) & 0xff] * __ldg(A.rnorm + e));
    });
}

// R' entries of Lambda are ordered by L, then M, then k (k <= (Lambda - L)/2); the harmonic row of (L, M) is
// L^2 + L + M and the radial row of (L, k) is the number of (L', k') with L' < L plus k.
// First radial group (in (L, k) order) of the second warp: the groups before it hold at least half the entries.
__host__ __device__ constexpr int esp_group_split(int lam) {
  const int half = cn_r(lam) / 2;
  int g = 0, cum = 0;
  for (int L = 0; L <= lam; ++L)
    for (int k = 0; k <= (lam - L) / 2; ++k, ++g) {
      if (cum >= half) return g;
      cum += 2 * L + 1;
    }
  return g;
}

// Per point: sum_e G'[e] S[h(e)] B[b(e)] grouped by the radial row, sum_{L,k} B_Lk (sum_M G'_{LMk} S_LM): one
// multiply-add per entry and one per radial row, instead of a product and a multiply-add per entry.  Radial
// groups g in [g0, g1); the walk from group 0 to g0 stops by L = Lambda + 1 (g0 <= number of radial rows).
// Loops run over runtime bounds: a fully unrolled form was slower (its code overflowed the instruction cache).
template <int LAM, int CS>
__device__ __forceinline__ double esp_point_sum(int g0, int g1, const double* __restrict__ gam,
                                                const double* __restrict__ S, const double* __restrict__ B) {
  int L = 0, rb = 0, bb = 0;
  while (bb + (LAM - L) / 2 + 1 <= g0) {
    rb += (2 * L + 1) * ((LAM - L) / 2 + 1);
    bb += (LAM - L) / 2 + 1;
    ++L;
  }
  int k = g0 - bb, nk = (LAM - L) / 2 + 1;
  double s0 = 0.0, s1 = 0.0;
  for (int g = g0; g < g1; ++g) {
    const double* gp = gam + rb + k;  // G'_{L,M,k}, M = -L..L, stride nk
    const double* sp = S + L * L * CS;
    const int n = 2 * L + 1;
    double t0 = 0.0, t1 = 0.0;
    int j = 0;
    for (; j + 1 < n; j += 2) {
      t0 = fma(gp[j * nk], sp[j * CS], t0);
      t1 = fma(gp[(j + 1) * nk], sp[(j + 1) * CS], t1);
    }
    t0 = fma(gp[j * nk], sp[j * CS], t0);  // n is odd
    if (g & 1)
      s1 = fma(t0 + t1, B[(bb + k) * CS], s1);
    else
      s0 = fma(t0 + t1, B[(bb + k) * CS], s0);
    if (++k == nk) {
      rb += (2 * L + 1) * nk;
      bb += nk;
      ++L;
      k = 0;
      nk = (LAM - L) / 2 + 1;
    }
  }
  return s0 + s1;
}

// Electrostatic potential (adjoint of the coupling): for a chunk of NCH points and a range of primitive
// pairs of one class, phi(C) += sum_e G'[e] U_{L(e)M(e)}(d/|d|) |d|^L beta_{L,k}/k! (d = C - P, unit
// charge), G' being the density-weighted adjoint block of the primitive pair (k_esp_adjoint).  Block
// (chunk, split): the splits divide the class's primitive pairs; each block adds its partial sums to
// phi once per point.  Point sums: warp 0 takes the radial groups before esp_group_split, warp 1 the rest.
template <int NCH, int LAM>
__global__ void __launch_bounds__(64) k_esp_fp64(EspArgs A) {
  using Sh = CouplingShape<LAM, NCH>;
  constexpr int nS = Sh::nS, nR = Sh::nR, CS = Sh::CS;
  extern __shared__ __align__(16) double smem[];
  double* Stab = smem;
  double* Btab = Stab + nS * CS;
  double* gam = Btab + Sh::nB * CS;  // [nR]
  double* part = gam + nR;           // [NCH] partial sums of warp 1
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int chunk = blockIdx.x % A.nchunks, split = blockIdx.x / A.nchunks;
  const int64_t per = (A.npp + A.nsplit - 1) / A.nsplit;
  const int64_t w0 = split * per, w1 = min(A.npp, w0 + per);
  const int64_t c = (int64_t)chunk * NCH + lane;
  const bool valid = lane < NCH && c < A.npoints;
  double acc = 0.0;
  constexpr int GS = esp_group_split(LAM);
  for (int64_t w = w0; w < w1; ++w) {
    const int64_t q = A.pp_base + w;
    const PPData pd = A.ppd[q];
    if (pd.pref == 0.0) continue;
    const int pr = A.pp_pair[q];
    const int a = A.pair_a[pr];
    const double Ax = A.shell_xyz[3 * a], Ay = A.shell_xyz[3 * a + 1], Az = A.shell_xyz[3 * a + 2];
    double Q[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Q[k] = A.site_rot[9 * A.pair_site[pr] + k];
    __syncthreads();  // the previous primitive pair is done with the tables and gam
    for (int e = tid; e < nR; e += 64) gam[e] = A.gam[w * (int64_t)nR + e];
    if (lane < NCH) {
      double dx = 0.0, dy = 0.0, dz = 0.0, z = 0.0;
      if (valid) {
        pair_frame_offset(Q, Ax, Ay, Az, pd.shift, A.points + 3 * c, dx, dy, dz);
        z = 1.0;
      }
      point_tables<LAM, CS>(wid, lane, pd.p, dx, dy, dz, z, A.boys_tab, Stab, Btab);
    }
    __syncthreads();
    if (lane < NCH)
      acc += esp_point_sum<LAM, CS>(wid == 0 ? 0 : GS, wid == 0 ? GS : Sh::nB, gam, Stab + lane, Btab + lane);
  }
  __syncthreads();
  if (wid == 1 && lane < NCH) part[lane] = acc;
  __syncthreads();
  if (wid == 0 && valid) atomicAdd(A.phi + c, acc + part[lane]);
}

// Solid-harmonic polynomials S~_lm(d) = |d|^l U_lm(d/|d|) (degree l, same constants as U) and their
// gradients, l <= LAM, into P, Gx, Gy, Gz at row h = l^2 + l + m (stride CS): forward-mode derivatives of
// S~_{l+1,m} = z S~_lm + ng_lm r^2 S~_{l-1,m}, S~_{|m|+1,m} = z S~_{|m|,m} and of the diagonal chain
// S~_{l+1,l+1} = x S~_ll - y S~_{l,-l}, S~_{l+1,-l-1} = y S~_ll + x S~_{l,-l} (which does not depend on z).
// The columns are split by the sign of m between the two half-warps: lanes of half `neg` take
// m = -|m| for |m| >= 1, the others m = +|m| for |m| >= 0.  The diagonal chain and the column
// recursions run as loops over |m| and l, so that both halves, whose columns of one |m| have equal
// lengths, advance in step.
template <int LAM, int CS>
__device__ __forceinline__ void harmonic_columns_grad_half(bool neg, double x, double y, double z, double* P,
                                                           double* Gx, double* Gy, double* Gz) {
  const double r2 = x * x + y * y + z * z;
  double dp = 1.0, dm = 1.0, dpx = 0.0, dpy = 0.0, dmx = 0.0, dmy = 0.0;  // U_{am,+-am} and gradients
#pragma unroll 1
  for (int am = 0; am <= LAM; ++am) {
    if (!(neg && am == 0)) {
      const int m = neg ? -am : am;
      double v0 = neg ? dm : dp, x0 = neg ? dmx : dpx, y0 = neg ? dmy : dpy, z0 = 0.0;
      int h = am * am + am + m;
      P[h * CS] = v0;
      Gx[h * CS] = x0;
      Gy[h * CS] = y0;
      Gz[h * CS] = z0;
      if (am + 1 <= LAM) {
        double v1 = z * v0, x1 = z * x0, y1 = z * y0, z1 = v0;
        h = (am + 1) * (am + 1) + am + 1 + m;
        P[h * CS] = v1;
        Gx[h * CS] = x1;
        Gy[h * CS] = y1;
        Gz[h * CS] = z1;
#pragma unroll 2
        for (int l = am + 1; l < LAM; ++l) {
          const double g = k_harm.ng[l * l + l + m];
          const double v2 = fma(g * r2, v0, z * v1);
          const double x2 = fma(g, fma(2.0 * x, v0, r2 * x0), z * x1);
          const double y2 = fma(g, fma(2.0 * y, v0, r2 * y0), z * y1);
          const double z2 = fma(g, fma(2.0 * z, v0, r2 * z0), fma(z, z1, v1));
          h = (l + 1) * (l + 1) + l + 1 + m;
          P[h * CS] = v2;
          Gx[h * CS] = x2;
          Gy[h * CS] = y2;
          Gz[h * CS] = z2;
          v0 = v1; x0 = x1; y0 = y1; z0 = z1;
          v1 = v2; x1 = x2; y1 = y2; z1 = z2;
        }
      }
    }
    // the diagonal chain one level up
    if (am == 0) {
      dp = x;
      dm = y;
      dpx = 1.0;
      dpy = 0.0;
      dmx = 0.0;
      dmy = 1.0;
    } else {
      const double np = fma(x, dp, -y * dm), nm = fma(y, dp, x * dm);
      const double npx = dp + fma(x, dpx, -y * dmx), npy = fma(x, dpy, -y * dmy) - dm;
      const double nmx = fma(y, dpx, x * dmx) + dm, nmy = fma(y, dpy, x * dmy) + dp;
      dp = np;
      dm = nm;
      dpx = npx;
      dpy = npy;
      dmx = nmx;
      dmy = nmy;
    }
  }
}

template <int LAM>
struct GradShape {
  static constexpr int NCH = 16, CS = NCH + 2;
  static constexpr int nS = cn_harm(LAM), nB = cn_beta(LAM), nR = cn_r(LAM);
  static constexpr size_t smem = sizeof(double) * ((size_t)(4 * nS + 2 * nB) * CS + nR + 3 * NCH + 4 * 64 + 16);
};

// Gradient of the electrostatic potential at each point: for a chunk of 16 points and a range of
// primitive pairs of one class, grad phi(C) += Q^T sum_e G'[e] d/dd [S~_{LM}(d) B_{L,k}(T)], d = C - P in the
// pair frame, B_{L,k} = sum_{j<=k} T^j/j! F_{L+j} and dB_{L,k}/dT = -T^k/k! F_{L+k+1}, so
// d/dd [S~ B] = B grad S~ - 2p T^k/k! F_{L+k+1} S~ d.  Threads: point c = t % 16; in the table phase
// warp 0 (16 lanes) evaluates the Boys values and radial factors, warp 1 the harmonic columns (its two
// halves the columns of m >= 0 and m < 0); in the sum phase the four groups of 16 threads take a quarter
// of the R' entries each.
template <int LAM>
__global__ void __launch_bounds__(64) k_esp_grad_fp64(EspArgs A) {
  using Sh = GradShape<LAM>;
  constexpr int NCH = Sh::NCH, CS = Sh::CS, nS = Sh::nS, nB = Sh::nB, nR = Sh::nR;
  extern __shared__ __align__(16) double smem[];
  double* Pt = smem;
  double* Gxt = Pt + nS * CS;
  double* Gyt = Gxt + nS * CS;
  double* Gzt = Gyt + nS * CS;
  double* Bt = Gzt + nS * CS;
  double* Bq = Bt + nB * CS;
  double* gam = Bq + nB * CS;
  double* dv = gam + nR;      // [3][NCH]
  double* red = dv + 3 * NCH; // [3][64]
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, pc = tid & 15, quarter = tid >> 4;
  const int chunk = blockIdx.x % A.nchunks, split = blockIdx.x / A.nchunks;
  const int64_t per = (A.npp + A.nsplit - 1) / A.nsplit;
  const int64_t w0 = split * per, w1 = min(A.npp, w0 + per);
  const int64_t c = (int64_t)chunk * NCH + pc;
  const bool valid = c < A.npoints;
  const int e0 = quarter * nR / 4, e1 = (quarter + 1) * nR / 4;
  double gm[3] = {0.0, 0.0, 0.0};
  for (int64_t w = w0; w < w1; ++w) {
    const int64_t q = A.pp_base + w;
    const PPData pd = A.ppd[q];
    if (pd.pref == 0.0) continue;
    const int pr = A.pp_pair[q];
    const int a = A.pair_a[pr];
    double Q[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Q[k] = A.site_rot[9 * A.pair_site[pr] + k];
    double dx = 0.0, dy = 0.0, dz = 0.0;
    if (valid)
      pair_frame_offset(Q, A.shell_xyz[3 * a], A.shell_xyz[3 * a + 1], A.shell_xyz[3 * a + 2], pd.shift,
                        A.points + 3 * c, dx, dy, dz);
    __syncthreads();  // the previous primitive pair is done with the tables
    for (int e = tid; e < nR; e += 64) gam[e] = A.gam[w * (int64_t)nR + e];
    if (lane < NCH) {
      if (wid == 0) {
        dv[pc] = dx;
        dv[NCH + pc] = dy;
        dv[2 * NCH + pc] = dz;
        const double T = pd.p * (dx * dx + dy * dy + dz * dz);
        double F[LAM + 2];
        boys_eval(LAM + 1, T, F, 1, A.boys_tab, k_boys);
        double tk[LAM / 2 + 1];  // T^k / k!
        tk[0] = 1.0;
#pragma unroll
        for (int k = 1; k <= LAM / 2; ++k) tk[k] = tk[k - 1] * T * k_boys.inv_int[k];
        const double m2p = -2.0 * pd.p;
        int bo = 0;
#pragma unroll
        for (int L = 0; L <= LAM; ++L) {
          double acc = 0.0;
#pragma unroll
          for (int k = 0; k <= (LAM - L) / 2; ++k) {
            acc = fma(tk[k], F[L + k], acc);
            Bt[(bo + k) * CS + pc] = valid ? acc : 0.0;
            Bq[(bo + k) * CS + pc] = valid ? m2p * tk[k] * F[L + k + 1] : 0.0;
          }
          bo += (LAM - L) / 2 + 1;
        }
      }
    }
    if (wid == 1) {
      // both half-warps: the columns of m >= 0 (lanes 0-15) and m < 0 (lanes 16-31) of the same points
      harmonic_columns_grad_half<LAM, CS>(lane >= NCH, dx, dy, dz, Pt + pc, Gxt + pc, Gyt + pc, Gzt + pc);
    }
    __syncthreads();
    double gx = 0.0, gy = 0.0, gz = 0.0, sb = 0.0;
    for (int e = e0; e < e1; ++e) {
      const int code = __ldg(A.rmap + e);
      const int si = (code & 0xfff) * CS + pc, bi = ((code >> 12) & 0xfff) * CS + pc;
      const double g = gam[e];
      const double ab = g * Bt[bi];
      gx = fma(ab, Gxt[si], gx);
      gy = fma(ab, Gyt[si], gy);
      gz = fma(ab, Gzt[si], gz);
      sb = fma(g * Pt[si], Bq[bi], sb);
    }
    gx = fma(sb, dv[pc], gx);
    gy = fma(sb, dv[NCH + pc], gy);
    gz = fma(sb, dv[2 * NCH + pc], gz);
    // back to the molecular frame: grad_C = Q^T grad_d
    gm[0] += Q[0] * gx + Q[3] * gy + Q[6] * gz;
    gm[1] += Q[1] * gx + Q[4] * gy + Q[7] * gz;
    gm[2] += Q[2] * gx + Q[5] * gy + Q[8] * gz;
  }
  __syncthreads();
  red[tid] = gm[0];
  red[64 + tid] = gm[1];
  red[128 + tid] = gm[2];
  __syncthreads();
  if (tid < NCH && valid)
    for (int k = 0; k < 3; ++k)
      atomicAdd(A.phi + 3 * c + k, red[k * 64 + tid] + red[k * 64 + tid + 16] + red[k * 64 + tid + 32] +
                                       red[k * 64 + tid + 48]);
}

using CouplingKernel = void (*)(CouplingArgs);
using EspKernel = void (*)(EspArgs);

template <int... L>
constexpr EspKernel esp_grad_kernel_at(int lam, std::integer_sequence<int, L...>) {
  EspKernel k = nullptr;
  ((lam == L ? (k = &k_esp_grad_fp64<L>, 0) : 0), ...);
  return k;
}

template <int... L>
constexpr size_t esp_grad_smem_at(int lam, std::integer_sequence<int, L...>) {
  size_t s = 0;
  ((lam == L ? (s = GradShape<L>::smem, 0) : 0), ...);
  return s;
}

template <int... L>
constexpr EspKernel esp_kernel_at(int lam, std::integer_sequence<int, L...>) {
  EspKernel k = nullptr;
  ((lam == L ? (k = &k_esp_fp64<32, L>, 0) : 0), ...);
  return k;
}

template <int NCH, int NW, int... L>
constexpr CouplingKernel kernel_at(int lam, std::integer_sequence<int, L...>) {
  CouplingKernel k = nullptr;
  ((lam == L ? (k = &k_coupling_fp64<NCH, L, NW>, 0) : 0), ...);
  return k;
}

template <int NCH, int... L>
constexpr size_t smem_at(int lam, std::integer_sequence<int, L...>) {
  size_t s = 0;
  ((lam == L ? (s = CouplingShape<L, NCH>::smem, 0) : 0), ...);
  return s;
}

using Lams = std::make_integer_sequence<int, kLamMax + 1>;
// the coupling kernel also runs at Lambda = la + lb + 1 (derivative integrals)
using LamsDer = std::make_integer_sequence<int, kLamDer + 1>;

// Small Lambda: one warp per block does both halves of the nucleus tables (the second warp of the two-warp
// form has little of its own there: a few harmonic columns and a few R' entries).
constexpr int kOneWarpLamMax = 8;
using LamsOneWarp = std::make_integer_sequence<int, kOneWarpLamMax + 1>;
int coupling_warps(int lam, bool one_warp_ok) { return one_warp_ok && lam <= kOneWarpLamMax ? 1 : 2; }

CouplingKernel coupling_kernel(int lam, int nch, int nw) {
  if (lam < 0 || lam > kLamDer) return nullptr;
  if (nw == 1)
    return lam > kOneWarpLamMax ? nullptr
                                : (nch == 16 ? kernel_at<16, 1>(lam, LamsOneWarp{}) : kernel_at<32, 1>(lam, LamsOneWarp{}));
  return nch == 16 ? kernel_at<16, 2>(lam, LamsDer{}) : kernel_at<32, 2>(lam, LamsDer{});
}

}  // namespace

size_t coupling_fp64_smem(int lam, int nch) {
  if (lam < 0 || lam > kLamDer) return 0;
  return nch == 16 ? smem_at<16>(lam, LamsDer{}) : smem_at<32>(lam, LamsDer{});
}

size_t esp_fp64_smem(int lam) { return coupling_fp64_smem(lam, 32) + sizeof(double) * 40; }

cudaError_t launch_esp_fp64(int lam, const EspArgs& args, cudaStream_t stream) {
  if (lam < 0 || lam > kLamMax) return cudaErrorInvalidValue;
  const EspKernel k = esp_kernel_at(lam, Lams{});
  k<<<args.nchunks * args.nsplit, 64, esp_fp64_smem(lam), stream>>>(args);
  return cudaGetLastError();
}

cudaError_t launch_esp_grad_fp64(int lam, const EspArgs& args, cudaStream_t stream) {
  if (lam < 0 || lam > kLamMax) return cudaErrorInvalidValue;
  const EspKernel k = esp_grad_kernel_at(lam, Lams{});
  k<<<args.nchunks * args.nsplit, 64, esp_grad_smem_at(lam, Lams{}), stream>>>(args);
  return cudaGetLastError();
}

cudaError_t coupling_fp64_setup() {
  cudaError_t e = cudaMemcpyToSymbol(k_harm, &harm_coef_host(), sizeof(HarmCoef));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(k_boys, &boys_const_host(), sizeof(BoysConst));
  for (int lam = 0; lam <= kLamDer && e == cudaSuccess; ++lam)
    for (int nch : {16, 32})
      for (int nw : {1, 2}) {
        const CouplingKernel k = coupling_kernel(lam, nch, nw);
        if (k) e = set_max_dynamic_smem((const void*)k);
        if (e != cudaSuccess) break;
      }
  for (int lam = 0; lam <= kLamMax && e == cudaSuccess; ++lam) {
    e = set_max_dynamic_smem((const void*)esp_kernel_at(lam, Lams{}));
    if (e == cudaSuccess)
      e = set_max_dynamic_smem((const void*)esp_grad_kernel_at(lam, Lams{}));
  }
  return e;
}

cudaError_t launch_coupling_fp64(int lam, int nch, const CouplingArgs& args, int grid, cudaStream_t stream) {
  const int nw = coupling_warps(lam, args.one_warp_ok != 0);
  const CouplingKernel k = coupling_kernel(lam, nch, nw);
  if (!k) return cudaErrorInvalidValue;
  // one-warp blocks: twice the blocks for the same warps per SM
  if (nw == 1) grid = (int)std::min<int64_t>(2 * (int64_t)grid, std::max<int64_t>(args.npp, 1));
  k<<<grid, 32 * nw, coupling_fp64_smem(lam, nch), stream>>>(args);
  return cudaGetLastError();
}

}  // namespace shgo
