// Derivative integrals of the nuclear attraction: dV_ab/dA and dV_ab/dB (A, B the centres of the two basis
// functions) and the field integrals sum_C Z_C dV_ab/dC, through the steps of V itself (nucleus sums S2,
// Gaunt coupling and primitive contraction S3, translation and rotation S4) with one extra order of the
// one-centre integral and the l +- 1 steps of Eq. 3.
//
// For a = N S_la(r - A) exp(-alpha |r - A|^2), b the same on B with beta, p = alpha + beta, P the product
// centre (Eq. 5) and mu = alpha beta / p, the derivative of exp(-alpha |r - A|^2) by A_X is
// 2 alpha (r - A)_X exp(...), and r - A = (r - P) + (beta / p)(B - A), so
//   d/dA_X [a b] = -(d_X S_la)(r - A) [...]  -  2 mu (A - B)_X a b  +  2 alpha (r - P)_X a b.
// Term 1 is a V block of the lowered class (la - 1, lb), combined with
// d_X S_la,ma = (2 la + 1) sum_M G(1 m(X), la ma; la - 1 M) S_{la-1,M}.  Terms 2 and 3 together are
// 2 alpha (r - A)_X a b.  In the pair frame (z along B - A) r - A = (r - P) + |P - A| z, so component c of
// them multiplies the one-centre integrand of Eq. 12 by 2 alpha (x_c + |P - A| delta_cz); x_c couples S_LM to
// L + 1 and (with r^2) to L - 1 as the product S_1 S_L of Eq. 3:
//   r^{2k} x_c S_LM = sum G(1 m(c), L M; L+1 M') r^{2k} S_{L+1,M'} + sum G(1 m(c), L M; L-1 M') r^{2k+2} S_{L-1,M'},
// so it reads the one-centre integrals R'[L, M, k] up to Lambda + 1 = la + lb + 1.  B is the same with beta,
// r - B = (r - P) - |P - B| z and the lowered class (la, lb - 1).  The field integrals move the nucleus: the
// integral of f(r - P) / |r - C| has d/dC_X equal to the integral of (d_X f)(r - P) / |r - C|, and
// d_c [r^{2k} S_LM e^{-p r^2}] is again a sum of R' terms of order Lambda + 1.
//
// The raised and differentiated terms live in the pair frame (component c of Q (r - A)); the molecular
// component X is sum_c Q[c][X] (component c), Q the frame rotation, applied to the rotated blocks.
//
// Launches per class, on the pool streams: the FP64 coupling kernel at Lambda + 1 (one block per primitive
// pair), k_deriv_block (one block per shell pair and variant, blockIdx.y: the blocks raised along pair-frame
// axis c, weighted by 2 alpha and by 2 beta in one pass over the Gaunt program where shared memory allows, the
// lowered classes, or the field blocks, each rotated to the molecular frame into a scratch array) and
// k_deriv_combine, which adds a shell pair's blocks in a fixed order into the output (no atomics: the result
// does not depend on the schedule).  The density-contracted gradient replaces the combine by k_deriv_contract
// (each pair's elements weighted by the density and summed per pair) and k_shell_gradient (per shell, its
// pairs' sums in pair order).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "shgo_internal.h"

namespace shgo {

namespace {

// Variants of k_deriv_block (blockIdx.y selects one from DerivArgs::kinds).
constexpr int kKindAB = 0;      // .. 2: raised along axis c, weights 2 alpha and 2 beta (two accumulators)
constexpr int kKindA = 3;       // .. 5: the same, 2 alpha only
constexpr int kKindB = 6;       // .. 8: the same, 2 beta only
constexpr int kKindLowA = 9;    // class (la - 1, lb)
constexpr int kKindLowB = 10;   // class (la, lb - 1)
constexpr int kKindField = 11;  // .. 13: d_c of the one-centre integrand
// Blocks of a shell pair's scratch, each (2 la + 1) x (2 lb + 1): A's raised blocks (3 pair-frame axes), B's,
// the lowered classes' terms for A and for B (3 molecular axes each), the field (3 pair-frame axes).
constexpr int kSlotA = 0, kSlotB = 3, kSlotLowA = 6, kSlotLowB = 9, kSlotField = 12, kSlots = 15;

__host__ __device__ inline void deriv_shape(int la, int lb, int kind, int& lbra, int& lket) {
  lbra = kind == kKindLowA ? la - 1 : la;
  lket = kind == kKindLowB ? lb - 1 : lb;
}
__host__ __device__ inline bool kind_raised(int kind) { return kind < kKindLowA; }
__host__ __device__ inline int kind_comp(int kind) { return kind >= kKindField ? kind - kKindField : kind % 3; }

// Shared memory of one k_deriv_block variant (doubles, the carve-up in the kernel).
__host__ __device__ inline size_t deriv_block_doubles(int la, int lb, int kind) {
  int lbra, lket;
  deriv_shape(la, lb, kind, lbra, lket);
  const int lhi = lbra > lket ? lbra : lket, llo = lbra > lket ? lket : lbra;
  const int na = 2 * lbra + 1, nb = 2 * lket + 1;
  const int nacc = kind < kKindA ? 2 : 1;
  const bool zoff = kind_raised(kind) && kind_comp(kind) == 2;
  return (size_t)nacc * (lhi + 1) * (lhi + 1) * w_stride(llo) + na * na + nb * nb + (lbra + 1) * na +
         (lket + 1) * nb + (size_t)(lbra + 1) * (lbra + 1) * nb + 2 * na * nb + 2 * (lhi + 1) * (llo + 1) +
         n_r(la + lb + 1) + n_r(lbra + lket) + (zoff ? n_r(lbra + lket) : 0) + 16 + 16;
}

struct DerivArgs {
  int la = 0, lb = 0, npairs = 0, pair_base = 0;
  int64_t pp_base = 0, rbase = 0;  // the class's first primitive pair; its coupling blocks at r1buf + rbase
  int nkind = 0;
  int kinds[8] = {};
  int64_t soff[kSlots] = {};  // offset of each block in a shell pair's scratch (doubles)
  int64_t per_pair = 0;       // scratch doubles per shell pair
  double* scratch = nullptr;  // the class's scratch
  const int* pair_a = nullptr;
  const int* pair_b = nullptr;
  const int64_t* pair_ppoff = nullptr;
  const int* pair_site = nullptr;
  int64_t rot_per = 0;
  const double* rotd = nullptr;
  const int* shell_poff = nullptr;
  const int* shell_nprim = nullptr;
  const double* prim_exp = nullptr;
  const int* pp_ij = nullptr;
  const double* etab = nullptr;
  const int* eoff = nullptr;
  const int* rowinfo[3] = {};  // Gaunt programs: the class, the class lowered on a, lowered on b
  const int* grp[3] = {};
  const GTerm* gterms[3] = {};
  const int* map0 = nullptr;       // Lambda layout -> Lambda + 1 layout
  const int* mapm = nullptr;       // Lambda - 1 layout -> Lambda + 1 layout
  const GTerm* raise = nullptr;    // Tables::d_raise of this Lambda
  const GTerm* fconst = nullptr;   // Tables::d_field of this Lambda
  const double* low_a = nullptr;   // Tables::d_low of la (nullptr for la = 0)
  const double* low_b = nullptr;   // of lb
  const PPData* ppd = nullptr;
  const double* r1buf = nullptr;
};

// Gaunt coupling of one primitive pair into W0 (and W1): rows of one warp form one group (equal trip counts,
// coalesced term loads).  acc = sum G Rv[.]; with ZOFF also acz = sum G Rz[.] (the unraised block), and the
// row adds fab0 (acc + s0 acz) to W0 and, with TWO, fab1 (acc + s1 acz) to W1.
template <bool ZOFF, bool TWO>
__device__ __forceinline__ void gaunt_pass(int nrp, const int* __restrict__ rowinfo, const int* __restrict__ grp,
                                           const GTerm* __restrict__ gterms, const double* Rv, const double* Rz,
                                           const double* fab0, const double* fab1, int lcols, double s0, double s1,
                                           double* W0, double* W1) {
  for (int r = threadIdx.x; r < nrp; r += blockDim.x) {
    const int info = rowinfo[r];
    const int gi = r >> 5, K = grp[2 * gi + 1];
    const GTerm* tp = gterms + grp[2 * gi] + (r & 31);
    double acc = 0.0, acc1 = 0.0, acz = 0.0, acz1 = 0.0;
    int j = 0;
    for (; j + 1 < K; j += 2) {
      const GTerm g0 = tp[32 * j], g1 = tp[32 * j + 32];
      acc = fma(g0.coef, Rv[g0.ridx], acc);
      acc1 = fma(g1.coef, Rv[g1.ridx], acc1);
      if (ZOFF) {
        acz = fma(g0.coef, Rz[g0.ridx], acz);
        acz1 = fma(g1.coef, Rz[g1.ridx], acz1);
      }
    }
    if (j < K) {
      const GTerm g0 = tp[32 * j];
      acc = fma(g0.coef, Rv[g0.ridx], acc);
      if (ZOFF) acz = fma(g0.coef, Rz[g0.ridx], acz);
    }
    acc += acc1;
    acz += acz1;
    if (info >= 0) {
      const int e = info & 0xffff, l1 = (info >> 16) & 15, l2 = (info >> 20) & 15;
      const int f = l1 * lcols + l2;
      W0[e] = fma(fab0[f], ZOFF ? fma(s0, acz, acc) : acc, W0[e]);
      if (TWO) W1[e] = fma(fab1[f], ZOFF ? fma(s1, acz, acc) : acc, W1[e]);
    }
  }
}

__global__ void __launch_bounds__(128, 8) k_deriv_block(DerivArgs A) {
  extern __shared__ double smem[];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int kind = A.kinds[blockIdx.y];
  int lbra, lket;
  deriv_shape(A.la, A.lb, kind, lbra, lket);
  // the lowered class (la - 1, la) has its Gaunt program stored as (la, la - 1): rows on the ket
  const bool swap = lbra < lket;
  const int lhi = swap ? lket : lbra, llo = swap ? lbra : lket;
  const int prog = kind == kKindLowA ? 1 : (kind == kKindLowB ? 2 : 0);
  const int* __restrict__ rowinfo = A.rowinfo[prog];
  const int* __restrict__ grp = A.grp[prog];
  const GTerm* __restrict__ gterms = A.gterms[prog];
  const bool raised = kind_raised(kind), field = kind >= kKindField;
  const bool lowered = kind == kKindLowA || kind == kKindLowB;
  const int NA = 2 * A.la + 1, NB = 2 * A.lb + 1;  // the class's block
  const int comp = kind_comp(kind);
  const bool zoff = raised && comp == 2;  // the pair-axis offsets |P - A|, |P - B| enter on z
  const int nacc = kind < kKindA ? 2 : 1;
  // slots written: the A (or only) block, then the B block
  const int slot0 = kind < kKindB ? kSlotA + comp
                                  : (kind < kKindLowA ? kSlotB + comp
                                                      : (kind == kKindLowA ? kSlotLowA
                                                                           : (kind == kKindLowB ? kSlotLowB : kSlotField + comp)));
  const int nR1 = n_r(A.la + A.lb + 1), nRv = n_r(lbra + lket);
  const int nWh = (lhi + 1) * (lhi + 1), nWl = (llo + 1) * (llo + 1), nW = nWh * nWl;
  const int ws = w_stride(llo), nWs = nWh * ws, nrp = (nW + 31) & ~31;
  const int nWa = (lbra + 1) * (lbra + 1);
  const int na = 2 * lbra + 1, nb = 2 * lket + 1;
  const int lm = lbra > lket ? lbra : lket;
  const int nDb = lbra != lket ? nb * nb : 0;
  const int nfab = (lhi + 1) * (llo + 1);
  double* W = smem;                          // nacc arrays [hi (l1 m1)][lo (l2 m2)], row stride ws
  double* Dm = W + nacc * nWs;               // D^{lbra}(Q^T), then D^{lket}(Q^T) when they differ
  double* tA = Dm + na * na + nb * nb;       // [l1][ma]
  double* tB = tA + (lbra + 1) * na;         // [l2][mb]
  double* Zb = tB + (lket + 1) * nb;         // [bra (l1 m1)][mb]
  double* Vp = Zb + nWa * nb;                // [ma][mb]
  double* Yb = Vp + na * nb;                 // [ma][mb]
  double* fab = Yb + na * nb;                // two arrays [hi l][lo l]: the weights of W0 and W1
  double* R1 = fab + 2 * nfab;               // coupling block of Lambda + 1 of one primitive pair
  double* Rv = R1 + nR1;                     // the variant's block in the layout its program reads
  double* Rz = Rv + nRv;                     // zoff: the unraised block
  double* scal = Rz + (zoff ? nRv : 0);      // prefactor, beta/p, alpha/p, 2 alpha, 2 beta, p, |P - A|, |P - B|
  double* dpow = scal + 16;                  // |b - a|^k
  for (int w = blockIdx.x; w < A.npairs; w += gridDim.x) {
    const int pr = A.pair_base + w;
    const int a = A.pair_a[pr], b = A.pair_b[pr];
    const double* rd = A.rotd + (int64_t)A.pair_site[pr] * A.rot_per;
    __syncthreads();
    if (tid == 0) {
      const double dist = rd[0];
      double v = 1.0;
      for (int k = 0; k <= lm; ++k) {
        dpow[k] = v;
        v *= dist;
      }
    }
    for (int e = tid; e < na * na; e += nth) Dm[e] = rd[1 + rot_doff(lbra) + e];
    for (int e = tid; e < nDb; e += nth) Dm[na * na + e] = rd[1 + rot_doff(lket) + e];
    for (int e = tid; e < nacc * nWs; e += nth) W[e] = 0.0;
    __syncthreads();
    // translation along the pair axis (Eqs. 7-8, only nu = 0 survives), as in the V pair kernel
    for (int e = tid; e < (lbra + 1) * na; e += nth) {
      const int l1 = e / na, ma = e % na - lbra, lr = lbra - l1;
      double v = 0.0;
      if (l1 >= (ma < 0 ? -ma : ma)) v = A.etab[A.eoff[lbra] + translation_offset_dev(lbra, ma, l1, ma) + lr] * dpow[lr];
      tA[e] = v;
    }
    for (int e = tid; e < (lket + 1) * nb; e += nth) {
      const int l2 = e / nb, mb = e % nb - lket, lr = lket - l2;
      double v = 0.0;
      if (l2 >= (mb < 0 ? -mb : mb))
        v = A.etab[A.eoff[lket] + translation_offset_dev(lket, mb, l2, mb) + lr] * ((lr & 1) ? -dpow[lr] : dpow[lr]);
      tB[e] = v;
    }
    const int npa = A.shell_nprim[a], npb = A.shell_nprim[b];
    const int64_t q0 = A.pair_ppoff[pr];
    bool live = false;  // uniform over the block
    for (int ij = 0; ij < npa * npb; ++ij) {
      __syncthreads();  // the previous primitive pair is done with R1, Rv, Rz, fab and scal
      if (tid == 0) {
        const PPData pd = A.ppd[q0 + ij];
        const int pij = A.pp_ij[q0 + ij];
        const double al = A.prim_exp[A.shell_poff[a] + (pij >> 8)], be = A.prim_exp[A.shell_poff[b] + (pij & 0xff)];
        scal[0] = pd.pref;
        scal[1] = pd.ra;
        scal[2] = pd.rb;
        scal[3] = 2.0 * al;
        scal[4] = 2.0 * be;
        scal[5] = pd.p;
        scal[6] = pd.ra * rd[0];   // |P - A| = (beta / p) |B - A|
        scal[7] = -pd.rb * rd[0];  // P - B along the axis: -(alpha / p) |B - A|
      }
      __syncthreads();
      if (scal[0] == 0.0) continue;  // skipped by the coupling kernel too (uniform over the block)
      live = true;
      const double* R = A.r1buf + A.rbase + (q0 + ij - A.pp_base) * (int64_t)nR1;
      for (int e = tid; e < nR1; e += nth) R1[e] = R[e];
      if (tid < nfab) {
        const int l1 = tid / (llo + 1), l2 = tid % (llo + 1);
        const int lb_i = swap ? l2 : l1, lk_i = swap ? l1 : l2;  // the bra's and the ket's l of the row
        double v = scal[0];
        const double ra = scal[1], rb = scal[2];
        for (int k = 0; k < lbra - lb_i; ++k) v *= ra;
        for (int k = 0; k < lket - lk_i; ++k) v *= rb;
        // weights: 2 alpha (A, AB), 2 beta (B; the second array of AB), 1 (lowered, field)
        fab[tid] = raised ? v * (kind >= kKindB ? scal[4] : scal[3]) : v;
        fab[nfab + tid] = v * scal[4];
      }
      __syncthreads();
      if (raised || field) {
        const double m2p = -2.0 * scal[5];
        for (int e = tid; e < nRv; e += nth) {
          const GTerm* tr = A.raise + ((size_t)e * 3 + comp) * kDerivSlots;
          double s = 0.0;
#pragma unroll
          for (int t = 0; t < kDerivSlots; ++t) s = fma(tr[t].coef, R1[tr[t].ridx], s);
          if (field) {
            const GTerm* tf = A.fconst + ((size_t)e * 3 + comp) * kDerivSlots;
            double f = 0.0;
#pragma unroll
            for (int t = 0; t < kDerivSlots; ++t) f = fma(tf[t].coef, R1[tf[t].ridx], f);
            s = fma(m2p, s, f);
          }
          Rv[e] = s;
          if (zoff) Rz[e] = R1[A.map0[e]];
        }
      } else {
        for (int e = tid; e < nRv; e += nth) Rv[e] = R1[A.mapm[e]];
      }
      __syncthreads();
      const double s0 = kind >= kKindB ? scal[7] : scal[6];
      if (zoff) {
        if (nacc == 2)
          gaunt_pass<true, true>(nrp, rowinfo, grp, gterms, Rv, Rz, fab, fab + nfab, llo + 1, s0, scal[7], W, W + nWs);
        else
          gaunt_pass<true, false>(nrp, rowinfo, grp, gterms, Rv, Rz, fab, fab, llo + 1, s0, 0.0, W, W);
      } else if (nacc == 2) {
        gaunt_pass<false, true>(nrp, rowinfo, grp, gterms, Rv, Rv, fab, fab + nfab, llo + 1, 0.0, 0.0, W, W + nWs);
      } else {
        gaunt_pass<false, false>(nrp, rowinfo, grp, gterms, Rv, Rv, fab, fab, llo + 1, 0.0, 0.0, W, W);
      }
    }
    for (int t = 0; t < nacc; ++t) {
      __syncthreads();
      double* o = A.scratch + (int64_t)w * A.per_pair + A.soff[t == 0 ? slot0 : kSlotB + comp];
      if (!live) {
        for (int e = tid; e < (lowered ? 3 * NA * NB : na * nb); e += nth) o[e] = 0.0;
        continue;
      }
      const double* Wt = W + t * nWs;
      // V' = t_A W t_B in the pair frame (diagonal in m), first over the ket's l
      for (int e = tid; e < nWa * nb; e += nth) {
        const int q = e / nWa, i1 = e - q * nWa;
        const int amb = (q + 1) >> 1, mb = (q & 1) ? amb : -amb;
        double s = 0.0;
        for (int l2 = amb; l2 <= lket; ++l2) {
          const int i2 = l2 * l2 + l2 + mb;
          s = fma(tB[l2 * nb + mb + lket], swap ? Wt[i2 * ws + i1] : Wt[i1 * ws + i2], s);
        }
        Zb[i1 * nb + mb + lket] = s;
      }
      __syncthreads();
      for (int e = tid; e < na * nb; e += nth) {
        const int q = e / nb, mb = e - q * nb;
        const int ama = (q + 1) >> 1, ma = (q & 1) ? ama : -ama;
        double s = 0.0;
        for (int l1 = ama; l1 <= lbra; ++l1) s = fma(tA[l1 * na + ma + lbra], Zb[(l1 * l1 + l1 + ma) * nb + mb], s);
        Vp[(ma + lbra) * nb + mb] = s;
      }
      __syncthreads();
      // to the molecular frame: D^{lbra} V' (D^{lket})^T
      const double* Da = Dm;
      const double* Db = lbra != lket ? Dm + na * na : Dm;
      for (int e = tid; e < na * nb; e += nth) {
        const int ma = e / nb, mb = e % nb;
        double s = 0.0;
        for (int k = 0; k < nb; ++k) s = fma(Vp[ma * nb + k], Db[mb * nb + k], s);
        Yb[e] = s;
      }
      __syncthreads();
      double* fin = lowered ? Zb : o;  // a lowered block stays in shared memory for the lowering below
      for (int e = tid; e < na * nb; e += nth) {
        const int ma = e / nb, mb = e % nb;
        double s = 0.0;
        for (int k = 0; k < na; ++k) s = fma(Da[ma * na + k], Yb[k * nb + mb], s);
        fin[e] = s;
      }
      if (lowered) {
        // the lowered class's term of each molecular axis X: -(d_X S_la)-weighted rows (A) or columns (B)
        __syncthreads();
        for (int e = tid; e < 3 * NA * NB; e += nth) {
          const int X = e / (NA * NB), r = e - X * NA * NB, ma = r / NB, mb = r - ma * NB;
          double v = 0.0;
          if (kind == kKindLowA) {
            const int nl = 2 * A.la - 1;
            const double* lo = A.low_a + ((int64_t)X * NA + ma) * nl;
            for (int k = 0; k < nl; ++k) v = fma(-lo[k], Zb[k * NB + mb], v);
          } else {
            const int nl = 2 * A.lb - 1;
            const double* lo = A.low_b + ((int64_t)X * NB + mb) * nl;
            for (int k = 0; k < nl; ++k) v = fma(-lo[k], Zb[ma * nl + k], v);
          }
          o[e] = v;
        }
      }
    }
  }
}

struct CombineArgs {
  int la = 0, lb = 0, npairs = 0, pair_base = 0;
  bool field = false;
  int64_t nbf = 0;
  int64_t soff[kSlots] = {};
  int64_t per_pair = 0;
  const double* scratch = nullptr;
  const int* pair_a = nullptr;
  const int* pair_b = nullptr;
  const int* pair_site = nullptr;
  const double* site_rot = nullptr;
  const int64_t* shell_foff = nullptr;
  double* out = nullptr;  // [3][nbf][nbf]
};

// One thread per element of every shell pair of the class (pair-major): the pair's derivative (or field)
// elements from its scratch blocks, all three components, both orientations written.  Derivative:
// out[X][a][b] = sum_c Q[c][X] V_A,c + L_A,X and, for a != b, out[X][b][a] = sum_c Q[c][X] V_B,c + L_B,X (L the
// lowered classes' terms).  Field: out[X][a][b] = out[X][b][a] = sum_c Q[c][X] V_F,c (a diagonal shell block
// takes its upper triangle for both halves, as V does).  Every thread's loads are independent of one another.
__global__ void __launch_bounds__(256) k_deriv_combine(CombineArgs C) {
  const int na = 2 * C.la + 1, nb = 2 * C.lb + 1, nab = na * nb;
  const int64_t plane = C.nbf * C.nbf;
  const int64_t total = (int64_t)C.npairs * nab;
  double* __restrict__ out = C.out;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int w = (int)(i / nab), e = (int)(i - (int64_t)w * nab);
    const int pr = C.pair_base + w;
    const int a = C.pair_a[pr], b = C.pair_b[pr];
    const int64_t fa0 = C.shell_foff[a], fb0 = C.shell_foff[b];
    const double* __restrict__ s = C.scratch + (int64_t)w * C.per_pair;
    const double* __restrict__ Q = C.site_rot + 9 * (int64_t)C.pair_site[pr];
    double q[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) q[k] = __ldg(Q + k);
    const int ma = e / nb, mb = e % nb;
    const int64_t iab = (fa0 + ma) * C.nbf + fb0 + mb, iba = (fb0 + mb) * C.nbf + fa0 + ma;
    if (C.field) {
      const int ee = (a == b && ma > mb) ? mb * nb + ma : e;
      double v[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c] = s[C.soff[kSlotField + c] + ee];
#pragma unroll
      for (int X = 0; X < 3; ++X) {
        const double f = fma(q[6 + X], v[2], fma(q[3 + X], v[1], q[X] * v[0]));
        out[X * plane + iab] = f;
        if (a != b) out[X * plane + iba] = f;
      }
      continue;
    }
    const bool two = a != b;
    double va[3], vb[3], la[3], lb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      va[c] = s[C.soff[kSlotA + c] + e];
      la[c] = C.la > 0 ? s[C.soff[kSlotLowA] + c * nab + e] : 0.0;
      vb[c] = two ? s[C.soff[kSlotB + c] + e] : 0.0;
      lb[c] = two && C.lb > 0 ? s[C.soff[kSlotLowB] + c * nab + e] : 0.0;
    }
#pragma unroll
    for (int X = 0; X < 3; ++X) {
      out[X * plane + iab] = fma(q[6 + X], va[2], fma(q[3 + X], va[1], fma(q[X], va[0], la[X])));
      if (two) out[X * plane + iba] = fma(q[6 + X], vb[2], fma(q[3 + X], vb[1], fma(q[X], vb[0], lb[X])));
    }
  }
}

// Contraction of a class's derivative blocks with a density P: a group of lanes per shell pair writes
// partial[pr][0..2] = sum_{a, b} (P_ab + P_ba) dV_ab/dA_X over the pair's elements (the bra shell's centre) and,
// for two different shells, partial[pr][3..5] the same with dV_ab/dB_X (the ket shell's).  The element values
// are those k_deriv_combine writes; each lane sums its elements in index order and the group adds its lanes in
// a fixed butterfly, so the result does not depend on the schedule.
struct ContractArgs {
  int la = 0, lb = 0, npairs = 0, pair_base = 0;
  int64_t nbf = 0;
  int64_t soff[kSlots] = {};
  int64_t per_pair = 0;
  const double* scratch = nullptr;
  const int* pair_a = nullptr;
  const int* pair_b = nullptr;
  const int* pair_site = nullptr;
  const double* site_rot = nullptr;
  const int64_t* shell_foff = nullptr;
  const double* P = nullptr;  // nbf x nbf
  double* partial = nullptr;  // [npairs of the basis][6]
};

template <int G>
__global__ void __launch_bounds__(128) k_deriv_contract(ContractArgs C) {
  // G lanes per shell pair (a power of two up to 32, from the pair's element count); a warp takes 32 / G
  // consecutive pairs per round and keeps every lane in the round for the shuffles
  const int lane = threadIdx.x & 31, sub = lane / G, lg = lane % G;
  const int na = 2 * C.la + 1, nb = 2 * C.lb + 1, nab = na * nb;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  for (int64_t w0 = wid * (32 / G); w0 < C.npairs; w0 += warps * (32 / G)) {
    const int64_t w = w0 + sub;
    const bool active = w < C.npairs;
    const int pr = C.pair_base + (int)(active ? w : w0);
    const int a = C.pair_a[pr], b = C.pair_b[pr];
    const bool two = a != b;
    const int64_t fa0 = C.shell_foff[a], fb0 = C.shell_foff[b];
    const double* __restrict__ s = C.scratch + (int64_t)w * C.per_pair;
    const double* __restrict__ Q = C.site_rot + 9 * (int64_t)C.pair_site[pr];
    double q[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) q[k] = __ldg(Q + k);
    double ga[3] = {0.0, 0.0, 0.0}, gb[3] = {0.0, 0.0, 0.0};
    for (int e = lg; active && e < nab; e += G) {
      const int ma = e / nb, mb = e % nb;
      const int64_t iab = (fa0 + ma) * C.nbf + fb0 + mb, iba = (fb0 + mb) * C.nbf + fa0 + ma;
      const double pw = __ldg(C.P + iab) + __ldg(C.P + iba);
      double va[3], vb[3], la[3], lb[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        va[c] = s[C.soff[kSlotA + c] + e];
        la[c] = C.la > 0 ? s[C.soff[kSlotLowA] + c * nab + e] : 0.0;
        vb[c] = two ? s[C.soff[kSlotB + c] + e] : 0.0;
        lb[c] = two && C.lb > 0 ? s[C.soff[kSlotLowB] + c * nab + e] : 0.0;
      }
#pragma unroll
      for (int X = 0; X < 3; ++X) {
        ga[X] = fma(pw, fma(q[6 + X], va[2], fma(q[3 + X], va[1], fma(q[X], va[0], la[X]))), ga[X]);
        gb[X] = fma(pw, fma(q[6 + X], vb[2], fma(q[3 + X], vb[1], fma(q[X], vb[0], lb[X]))), gb[X]);
      }
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1)
#pragma unroll
      for (int X = 0; X < 3; ++X) {
        ga[X] += __shfl_xor_sync(0xffffffffu, ga[X], off);
        gb[X] += __shfl_xor_sync(0xffffffffu, gb[X], off);
      }
    if (active && lg == 0) {
      double* o = C.partial + 6 * (int64_t)pr;
#pragma unroll
      for (int X = 0; X < 3; ++X) {
        o[X] = ga[X];
        o[3 + X] = two ? gb[X] : 0.0;
      }
    }
  }
}

// grad[s][X] = the partials of the shell's pairs (entries pr * 2 + side of its list, in pair order) added up: one
// warp per shell, lane i taking entries i, i + 32, ... in order, then a fixed butterfly across the lanes.
__global__ void __launch_bounds__(128) k_shell_gradient(int n_shells, const int64_t* __restrict__ off,
                                                        const int64_t* __restrict__ list,
                                                        const double* __restrict__ partial, double* __restrict__ grad) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t sh = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); sh < n_shells; sh += warps) {
    double g[3] = {0.0, 0.0, 0.0};
    for (int64_t j = off[sh] + lane; j < off[sh + 1]; j += 32) {
      const int64_t e = list[j];
      const double* p = partial + 6 * (e >> 1) + 3 * (e & 1);
#pragma unroll
      for (int X = 0; X < 3; ++X) g[X] += p[X];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int X = 0; X < 3; ++X) g[X] += __shfl_xor_sync(0xffffffffu, g[X], o);
    if (lane == 0)
#pragma unroll
      for (int X = 0; X < 3; ++X) grad[3 * sh + X] = g[X];
  }
}

int class_of(int l1, int l2) { return l1 >= l2 ? class_id(l1, l2) : class_id(l2, l1); }

// Largest shared memory of a variant that raises for both centres in one pass: two blocks fit on an SM.
constexpr size_t kDualMaxBytes = 113 * 1024;

}  // namespace

shgo_status launch_nuclear_deriv(const DeviceBasis& db, const DeviceTables& dt, const std::vector<ClassWork>& work,
                                 int64_t nbf, int64_t ncenters, const double* centers, const double* charges,
                                 double* out, bool field, cudaStream_t stream, std::string* err,
                                 const DerivContraction* contract) {
  if (nbf == 0) return SHGO_OK;
  const size_t nout = contract ? (size_t)3 * (size_t)contract->n_shells : (size_t)3 * (size_t)nbf * (size_t)nbf;
  if (contract) out = contract->grad;
  if (ncenters == 0) {
    const cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * nout, stream);
    if (e != cudaSuccess) {
      *err = cudaGetErrorString(e);
      return SHGO_ERR_CUDA;
    }
    return SHGO_OK;
  }
  const Tables& th = tables_host();
  // per class: variants, scratch layout, coupling-block and scratch offsets
  struct Plan {
    DerivArgs d;
    CombineArgs c;
    size_t smem = 0;
    int threads = 32;
    int64_t r1 = 0, scr = 0;  // doubles
  };
  std::vector<Plan> plan(work.size());
  int64_t r1_total = 0, scr_total = 0;
  for (size_t ci = 0; ci < work.size(); ++ci) {
    const ClassWork& w = work[ci];
    Plan& P = plan[ci];
    DerivArgs& d = P.d;
    d.la = w.la;
    d.lb = w.lb;
    d.npairs = w.npairs;
    d.pair_base = w.pair_base;
    d.pp_base = w.pp_base;
    // variants: the three axes raised for both centres in one pass when two such blocks fit on an SM,
    // otherwise one pass per centre; the lowered classes; or the three field blocks
    std::vector<int> kinds;
    if (field) {
      kinds = {kKindField, kKindField + 1, kKindField + 2};
    } else {
      const bool dual = sizeof(double) * deriv_block_doubles(w.la, w.lb, kKindAB + 2) <= kDualMaxBytes;
      for (int c = 0; c < 3; ++c) {
        if (dual) {
          kinds.push_back(kKindAB + c);
        } else {
          kinds.push_back(kKindA + c);
          kinds.push_back(kKindB + c);
        }
      }
      if (w.la > 0) kinds.push_back(kKindLowA);
      if (w.lb > 0) kinds.push_back(kKindLowB);
    }
    d.nkind = (int)kinds.size();
    for (int k = 0; k < d.nkind; ++k) {
      d.kinds[k] = kinds[k];
      P.smem = std::max(P.smem, sizeof(double) * deriv_block_doubles(w.la, w.lb, kinds[k]));
    }
    // scratch blocks of a shell pair
    const int64_t nab = (int64_t)(2 * w.la + 1) * (2 * w.lb + 1);
    int64_t off = 0;
    auto place = [&](int slot, int64_t n) {
      d.soff[slot] = off;
      off += n;
    };
    if (field) {
      for (int c = 0; c < 3; ++c) place(kSlotField + c, nab);
    } else {
      for (int c = 0; c < 3; ++c) place(kSlotA + c, nab);
      for (int c = 0; c < 3; ++c) place(kSlotB + c, nab);
      if (w.la > 0) place(kSlotLowA, 3 * nab);
      if (w.lb > 0) place(kSlotLowB, 3 * nab);
    }
    d.per_pair = off;
    P.threads = (w.la + 1) * (w.la + 1) * (w.lb + 1) * (w.lb + 1) >= 1024
                    ? 128
                    : ((w.la + 1) * (w.la + 1) * (w.lb + 1) * (w.lb + 1) >= 256 ? 64 : 32);
    P.r1 = r1_total;
    P.scr = scr_total;
    r1_total += w.npp * (int64_t)n_r(w.la + w.lb + 1);
    scr_total += (int64_t)w.npairs * off;
  }
  int64_t npairs_all = 0;
  for (const ClassWork& w : work) npairs_all = std::max<int64_t>(npairs_all, (int64_t)w.pair_base + w.npairs);
  double* r1buf = nullptr;
  double* scr = nullptr;
  double* partial = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&r1buf, sizeof(double) * (size_t)std::max<int64_t>(r1_total, 1), stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&scr, sizeof(double) * (size_t)std::max<int64_t>(scr_total, 1), stream);
  if (e == cudaSuccess && contract)
    e = cudaMallocAsync((void**)&partial, sizeof(double) * 6 * (size_t)std::max<int64_t>(npairs_all, 1), stream);
  if (e != cudaSuccess) {
    if (r1buf) cudaFreeAsync(r1buf, stream);
    if (scr) cudaFreeAsync(scr, stream);
    cudaGetLastError();
    *err = std::string("derivative buffers: ") + cudaGetErrorString(e);
    return SHGO_ERR_OOM;
  }
  e = ensure_max_dynamic_smem((const void*)k_deriv_block);
  cudaStream_t* pool = nullptr;
  int npool = 0;
  if (e == cudaSuccess) e = pool_streams(&pool, &npool);
  // classes by decreasing work, dealt round-robin over the pool streams
  std::vector<int> order(work.size());
  for (size_t c = 0; c < work.size(); ++c) order[c] = (int)c;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    auto cost = [&](int c) {
      const double nW = (double)(work[c].la + 1) * (work[c].la + 1) * (work[c].lb + 1) * (work[c].lb + 1);
      return (double)work[c].npp * ((double)ncenters * n_r(work[c].la + work[c].lb + 1) + 8.0 * nW * plan[c].d.nkind);
    };
    return cost(x) > cost(y);
  });
  const int ns = (int)std::min<size_t>(order.size(), (size_t)std::max(npool, 1));
  cudaEvent_t fork = nullptr;
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(fork, stream);
  for (int i = 0; i < ns && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(pool[i], fork, 0);
  for (size_t k = 0; k < order.size() && e == cudaSuccess; ++k) {
    const int ci = order[k];
    const ClassWork& w = work[ci];
    if (w.npairs == 0) continue;
    cudaStream_t s = pool[k % ns];
    Plan& P = plan[ci];
    const int lam1 = w.la + w.lb + 1;
    if (w.npp > 0) {
      CouplingArgs ca;
      ca.npp = w.npp;
      ca.pp_base = w.pp_base;
      ca.rbase = P.r1;
      ca.pp_pair = db.pp_pair;
      ca.pair_a = db.pair_a;
      ca.shell_xyz = db.shell_xyz;
      ca.mv.ncenters = ncenters;
      ca.mv.nbf = nbf;
      ca.centers = centers;
      ca.charges = charges;
      ca.boys_tab = dt.boys;
      ca.rmap = dt.rmap + th.rmap_off[lam1];
      ca.rnorm = dt.rnorm + th.rmap_off[lam1];
      ca.site_rot = db.site_rot;
      ca.pair_site = db.pair_site;
      ca.ppd = db.ppd;
      ca.rbuf = r1buf;
      ca.one_warp_ok = db.coupling_one_warp;
      e = launch_coupling_fp64(lam1, lam1 <= 12 ? 32 : 16, ca, grid_cap_sm(w.npp, 8), s);
      if (e != cudaSuccess) break;
    }
    DerivArgs& d = P.d;
    const int lam = w.la + w.lb;
    d.rbase = P.r1;
    d.scratch = scr + P.scr;
    d.pair_a = db.pair_a;
    d.pair_b = db.pair_b;
    d.pair_ppoff = db.pair_ppoff;
    d.pair_site = db.pair_site;
    d.rot_per = rot_block(db.rot_lmax);
    d.rotd = db.rotd;
    d.shell_poff = db.shell_poff;
    d.shell_nprim = db.shell_nprim;
    d.prim_exp = db.prim_exp;
    d.pp_ij = db.pp_ij;
    d.etab = dt.etab;
    d.eoff = dt.eoff;
    const int cids[3] = {class_id(w.la, w.lb), w.la > 0 ? class_of(w.la - 1, w.lb) : -1,
                         w.lb > 0 ? class_of(w.la, w.lb - 1) : -1};
    for (int p = 0; p < 3; ++p) {
      if (cids[p] < 0) continue;
      d.rowinfo[p] = dt.g_rowinfo + th.g_rowbase[cids[p]];
      d.grp[p] = dt.g_grp + 2 * th.g_grpbase[cids[p]];
      d.gterms[p] = dt.g_terms + th.g_termbase[cids[p]];
    }
    d.map0 = dt.d_map0 + th.d_map0_off[lam];
    d.mapm = dt.d_mapm + th.d_mapm_off[lam];
    d.raise = dt.d_raise + (size_t)th.d_xoff[lam] * 3 * kDerivSlots;
    d.fconst = dt.d_field + (size_t)th.d_xoff[lam] * 3 * kDerivSlots;
    d.low_a = w.la > 0 ? dt.d_low + th.d_low_off[w.la] : nullptr;
    d.low_b = w.lb > 0 ? dt.d_low + th.d_low_off[w.lb] : nullptr;
    d.ppd = db.ppd;
    d.r1buf = r1buf;
    const dim3 grid((unsigned)grid_cap_sm(w.npairs, 16), (unsigned)d.nkind);
    k_deriv_block<<<grid, P.threads, P.smem, s>>>(d);
    e = cudaGetLastError();
    if (e != cudaSuccess) break;
    if (contract) {
      ContractArgs g;
      g.la = w.la;
      g.lb = w.lb;
      g.npairs = w.npairs;
      g.pair_base = w.pair_base;
      g.nbf = nbf;
      for (int k = 0; k < kSlots; ++k) g.soff[k] = d.soff[k];
      g.per_pair = d.per_pair;
      g.scratch = d.scratch;
      g.pair_a = db.pair_a;
      g.pair_b = db.pair_b;
      g.pair_site = db.pair_site;
      g.site_rot = db.site_rot;
      g.shell_foff = db.shell_foff;
      g.P = contract->P;
      g.partial = partial;
      const int nab = (2 * w.la + 1) * (2 * w.lb + 1);
      int G = 1;
      while (G < 32 && G < nab) G *= 2;
      const int grid = grid_cap_sm(((int64_t)w.npairs * G + 127) / 128, 16);
      switch (G) {
        case 1: k_deriv_contract<1><<<grid, 128, 0, s>>>(g); break;
        case 2: k_deriv_contract<2><<<grid, 128, 0, s>>>(g); break;
        case 4: k_deriv_contract<4><<<grid, 128, 0, s>>>(g); break;
        case 8: k_deriv_contract<8><<<grid, 128, 0, s>>>(g); break;
        case 16: k_deriv_contract<16><<<grid, 128, 0, s>>>(g); break;
        default: k_deriv_contract<32><<<grid, 128, 0, s>>>(g); break;
      }
      e = cudaGetLastError();
      continue;
    }
    CombineArgs& c = P.c;
    c.la = w.la;
    c.lb = w.lb;
    c.npairs = w.npairs;
    c.pair_base = w.pair_base;
    c.field = field;
    c.nbf = nbf;
    for (int k = 0; k < kSlots; ++k) c.soff[k] = d.soff[k];
    c.per_pair = d.per_pair;
    c.scratch = d.scratch;
    c.pair_a = db.pair_a;
    c.pair_b = db.pair_b;
    c.pair_site = db.pair_site;
    c.site_rot = db.site_rot;
    c.shell_foff = db.shell_foff;
    c.out = out;
    k_deriv_combine<<<grid_cap_sm(((int64_t)w.npairs * (2 * w.la + 1) * (2 * w.lb + 1) + 255) / 256, 8), 256, 0, s>>>(c);
    e = cudaGetLastError();
  }
  for (int i = 0; i < ns && fork; ++i) {
    cudaEvent_t join;
    if (cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess) break;
    cudaEventRecord(join, pool[i]);
    cudaStreamWaitEvent(stream, join, 0);
    cudaEventDestroy(join);
  }
  if (fork) cudaEventDestroy(fork);
  if (e == cudaSuccess && contract) {
    k_shell_gradient<<<grid_cap_sm(((int64_t)contract->n_shells + 3) / 4, 16), 128, 0, stream>>>(
        contract->n_shells, contract->shell_off, contract->shell_list, partial, contract->grad);
    e = cudaGetLastError();
  }
  if (partial) cudaFreeAsync(partial, stream);
  cudaFreeAsync(scr, stream);
  cudaFreeAsync(r1buf, stream);
  if (e != cudaSuccess) {
    *err = std::string("derivative launch: ") + cudaGetErrorString(e);
    return SHGO_ERR_CUDA;
  }
  return SHGO_OK;
}

}  // namespace shgo
