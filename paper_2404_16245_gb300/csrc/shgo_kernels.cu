// CUDA kernels (sm_103a, FP64) of the SHGO nuclear-attraction path.
//
//  k_coupling_block  (S1 + S2): one warp per primitive pair (alpha_i on a, beta_j on b).
//      Gaussian product (Eq. 5): p, P.  Then, for every nucleus C (one lane per nucleus,
//      chunks of 32 or 16): d = C - P, T = p |d|^2, Boys F_0..F_Lambda(T), the radial factors
//      beta_{L,k}(T) = sum_j k!/j! T^j F_{L+j}(T) scaled by Z_C, and the real solid harmonics
//      S_LM(d); the lanes stage them in shared memory and then contract over the nuclei of the
//      chunk, each lane owning entries of
//          R[L,M,k] = sum_C Z_C S_LM(C - P) beta_{L,k}(T_C),
//      which is stored as R' = 2 pi p^{-(k+1)} R (the one-centre integral of Eq. 12 in coupled
//      form, before the Gaunt coupling).
//  k_pair_block      (S3 + S4 + S5): one warp per shell pair.  Couples R' of each primitive
//      pair with the real Gaunt coefficients into W[l1 m1][l2 m2], scales by c_i c_j K_AB
//      (beta/p)^{la-l1} (alpha/p)^{lb-l2} and sums over primitive pairs (Eq. 11); then the
//      translation ("vector uncoupling", Eq. 7) V = T_A W T_B^T with
//      T_A[ma][l1 m1] = sum_nu E^{la}(ma; l1 m1; nu) S_{la-l1,nu}(b - a) and T_B likewise with
//      a - b; writes the block and its transpose into V.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <string>

#include "shgo_internal.h"
#include "shgo_math.h"

namespace shgo {

__constant__ HarmCoef c_harm;
__constant__ BoysConst c_boys;
__constant__ int c_lof[(kLmax + 1) * (kLmax + 1)];  // l of a packed harmonic index (l <= 8)

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;


// |B - A|^2 and K_AB = exp(-alpha beta/(alpha + beta) |B - A|^2) of Eq. 5, with every operation
// rounded explicitly so that the coupling and pair kernels agree bit for bit on which primitive
// pairs have K_AB == 0 (the coupling kernel skips those, the pair kernel never reads them).
__device__ __forceinline__ double pair_ab2(const double* __restrict__ xyz, int a, int b) {
  const double dx = __dsub_rn(xyz[3 * b], xyz[3 * a]);
  const double dy = __dsub_rn(xyz[3 * b + 1], xyz[3 * a + 1]);
  const double dz = __dsub_rn(xyz[3 * b + 2], xyz[3 * a + 2]);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}
__device__ __forceinline__ double prim_kab(double ea, double eb, double ab2) {
  return exp(-__dmul_rn(__ddiv_rn(__dmul_rn(ea, eb), __dadd_rn(ea, eb)), ab2));
}

// Bound on every element of one primitive pair's block, per unit of total nuclear charge:
// |S_lm(r)| <= |r|^l (Racah normalisation) and |r_A| <= r_P + |PA|, and the potential of a non-negative
// radial density at any point is at most its value at the centre, int f(r)/r d^3r; so
//   |<a_i|1/|r-C||b_j>| <= |c_i c_j| K_AB 4 pi int_0^inf (r + |PA|)^la (r + |PB|)^lb e^{-p r^2} r dr.
// The overlap integrand is bounded the same way with r^2 dr; the larger of the two is returned.
// Moments: int_0^inf r^n e^{-p r^2} dr = M_n with M_0 = sqrt(pi/p)/2, M_1 = 1/(2p),
// M_{n+2} = (n+1)/(2p) M_n.
__device__ double prim_pair_bound(int la, int lb, double pa, double pb, double p, double pref) {
  double M[2 * kLmax + 4];
  M[0] = 0.5 * sqrt(3.14159265358979323846 / p);
  M[1] = 0.5 / p;
  for (int n = 0; n + 2 < 2 * kLmax + 4; ++n) M[n + 2] = (n + 1) * M[n] * (0.5 / p);
  double i1 = 0.0, i2 = 0.0, ca = 1.0;  // ca = C(la, i) pa^(la-i)
  double pa_pow[kLmax + 1], pb_pow[kLmax + 1];
  pa_pow[0] = pb_pow[0] = 1.0;
  for (int k = 1; k <= kLmax; ++k) {
    pa_pow[k] = pa_pow[k - 1] * pa;
    pb_pow[k] = pb_pow[k - 1] * pb;
  }
  for (int i = 0; i <= la; ++i) {
    ca = (i == 0) ? 1.0 : ca * (la - i + 1) / i;
    double cb = 1.0;
    for (int j = 0; j <= lb; ++j) {
      cb = (j == 0) ? 1.0 : cb * (lb - j + 1) / j;
      const double w = ca * cb * pa_pow[la - i] * pb_pow[lb - j];
      i1 += w * M[i + j + 1];
      i2 += w * M[i + j + 2];
    }
  }
  return fabs(pref) * 4.0 * 3.14159265358979323846 * fmax(i1, i2);
}

// Step S1, once per basis: the Gaussian-product data of every primitive pair.  A primitive pair whose
// bound (prim_pair_bound) is below kPrimSkip gets pref = 0, which every kernel treats as "skip": it
// changes any V element by at most kPrimSkip x sum |Z_C| (and any S element by at most kPrimSkip).
__global__ void k_pair_build(int64_t npp, const int* __restrict__ pp_pair, const int* __restrict__ pp_ij,
                             const int* __restrict__ pair_a, const int* __restrict__ pair_b,
                             const double* __restrict__ shell_xyz, const int* __restrict__ shell_l,
                             const int* __restrict__ shell_poff, const double* __restrict__ prim_exp,
                             const double* __restrict__ prim_coef, int use_bound, PPData* __restrict__ ppd) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npp; q += (int64_t)gridDim.x * blockDim.x) {
    const int pr = pp_pair[q], ij = pp_ij[q];
    const int a = pair_a[pr], b = pair_b[pr];
    const int ia = shell_poff[a] + (ij >> 8), ib = shell_poff[b] + (ij & 255);
    const double ea = prim_exp[ia], eb = prim_exp[ib];
    const double ab2 = pair_ab2(shell_xyz, a, b);
    PPData d;
    d.p = ea + eb;
    d.rp = 1.0 / d.p;
    d.sp = sqrt(d.p);
    d.kab = prim_kab(ea, eb, ab2);
    d.pref = prim_coef[ia] * prim_coef[ib] * d.kab;
    d.ra = eb * d.rp;
    d.rb = ea * d.rp;
    const double ab = sqrt(ab2);
    d.shift = d.ra * ab;
    if (use_bound && d.pref != 0.0 &&
        prim_pair_bound(shell_l[a], shell_l[b], d.shift, d.rb * ab, d.p, d.pref) < kPrimSkip)
      d.pref = 0.0;
    ppd[q] = d;
  }
}

// Per shell pair: whether any of its primitive pairs is kept (the block-sparse layout's criterion, the same
// test the pair kernel applies before writing a block).
__global__ void k_pair_live(int64_t npairs, const int64_t* __restrict__ pair_ppoff, int64_t npp_total,
                            const PPData* __restrict__ ppd, uint8_t* __restrict__ live) {
  for (int64_t pr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pr < npairs;
       pr += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q1 = pr + 1 < npairs ? pair_ppoff[pr + 1] : npp_total;
    uint8_t any = 0;
    for (int64_t q = pair_ppoff[pr]; q < q1 && !any; ++q) any = ppd[q].pref != 0.0;
    live[pr] = any;
  }
}

// Per class (classes given by their first pair, pair_cls[c] .. pair_cls[c + 1]): live primitive pairs
// (pref != 0), shell pairs with at least one, and the sum over live primitive pairs of their
// molecule's nucleus count (batches; 0 otherwise).
__global__ void k_live_counts(int npairs, int ncls, const int* __restrict__ pair_cls,
                              const int64_t* __restrict__ pair_ppoff, int64_t npp_total,
                              const PPData* __restrict__ ppd, const int* __restrict__ pair_mol,
                              const int64_t* __restrict__ mol_nc, unsigned long long* __restrict__ live_pp,
                              unsigned long long* __restrict__ live_pairs, double* __restrict__ live_cent) {
  for (int pr = blockIdx.x * blockDim.x + threadIdx.x; pr < npairs; pr += gridDim.x * blockDim.x) {
    int c = 0;
    while (c + 1 < ncls && pair_cls[c + 1] <= pr) ++c;
    const int64_t q1 = pr + 1 < npairs ? pair_ppoff[pr + 1] : npp_total;
    unsigned long long n = 0;
    for (int64_t q = pair_ppoff[pr]; q < q1; ++q) n += ppd[q].pref != 0.0;
    if (n) {
      atomicAdd(live_pp + c, n);
      atomicAdd(live_pairs + c, 1ull);
      if (pair_mol) atomicAdd(live_cent + c, (double)n * (double)mol_nc[pair_mol[pr]]);
    }
  }
}

// Shared-memory bytes of one block of k_pair_block.
__host__ __device__ inline size_t pair_smem(int la, int lb) {
  const int nWa = (la + 1) * (la + 1);
  const int na = 2 * la + 1, nb = 2 * lb + 1;
  return sizeof(double) * ((size_t)nWa * w_stride(lb) + na * na + nb * nb + (la + 1) * na + (lb + 1) * nb + nWa * nb +
                           2 * na * nb + (la + 1) * (lb + 1) + n_r(la + lb) + 32);
}

// Threads per block of k_pair_block for a class: enough to cover the W entries of large classes.
__host__ __device__ inline int pair_threads(int la, int lb) {
  const int nW = (la + 1) * (la + 1) * (lb + 1) * (lb + 1);
  return nW >= 1024 ? 128 : (nW >= 256 ? 64 : 32);
}


// Real rotation matrices D^l(R), l <= lm, R = Q^T (row-major in Rq), for the block's threads:
// D^0 = 1, D^1 from R, then D^{l+1} from D^l through the harmonic part of u_c S_{l,m'}(u) (the
// Gaunt product rule with one factor of degree 1).  Ends without a barrier after the last level.
__device__ void build_rotations(int lm, const double* Rq, double* Dm, const int* __restrict__ rot_ptr,
                                const GTerm* __restrict__ rot_terms) {
  const int tid = threadIdx.x, nth = blockDim.x;
  if (tid == 0) Dm[0] = 1.0;
  if (lm >= 1 && tid < 9) {
    const int m = tid / 3 - 1, c = tid % 3;  // row m, Cartesian column c (x, y, z)
    const int crow = m == -1 ? 1 : (m == 0 ? 2 : 0);
    const int mp = c == 0 ? 1 : (c == 1 ? -1 : 0);
    Dm[1 + (m + 1) * 3 + (mp + 1)] = Rq[crow * 3 + c];
  }
  for (int l = 1; l < lm; ++l) {
    __syncthreads();
    const double* Dl = Dm + rot_doff(l);
    double* Dn = Dm + rot_doff(l + 1);
    const int n1 = 2 * l + 3;
    for (int e = tid; e < n1 * n1; e += nth) {
      const int m = e / n1 - (l + 1), M = e % n1 - (l + 1);
      const int q = rot_index(l, M);
      double s = 0.0;
      if (m >= -l && m <= l) {
        for (int t = rot_ptr[q]; t < rot_ptr[q + 1]; ++t) {
          const GTerm g = rot_terms[t];
          s = fma(g.coef * Rq[6 + g.ridx], Dl[(m + l) * (2 * l + 1) + g.pad + l], s);
        }
        s *= c_harm.a[harm_index(l, m)];
      } else {
        const double* top = Dl + (2 * l) * (2 * l + 1);  // row m = l
        const double* bot = Dl;                          // row m = -l
        for (int t = rot_ptr[q]; t < rot_ptr[q + 1]; ++t) {
          const GTerm g = rot_terms[t];
          const double rx = Rq[g.ridx], ry = Rq[3 + g.ridx];
          const double v = (m > 0) ? (rx * top[g.pad + l] - ry * bot[g.pad + l])
                                   : (ry * top[g.pad + l] + rx * bot[g.pad + l]);
          s = fma(g.coef, v, s);
        }
        s *= c_harm.c[l];
      }
      Dn[e] = s;
    }
  }
}

// Once per basis: |B - A| and the rotation matrices D^0 .. D^lmax of the pair frame of every ordered
// pair of centres (one block each; they depend on the two positions only).
__global__ void __launch_bounds__(64) k_pair_rotations(int n_sites, int lmax, const int* __restrict__ site_rep,
                                                       const int* __restrict__ pair_a, const int* __restrict__ pair_b,
                                                       const double* __restrict__ site_rot,
                                                       const double* __restrict__ shell_xyz,
                                                       const int* __restrict__ rot_ptr,
                                                       const GTerm* __restrict__ rot_terms, double* __restrict__ rotd) {
  extern __shared__ double smem[];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int64_t per = rot_block(lmax);
  const int nD = rot_doff(lmax + 1);
  double* Dm = smem;
  double* Rq = Dm + nD;
  for (int i = blockIdx.x; i < n_sites; i += gridDim.x) {
    const int pr = site_rep[i];
    __syncthreads();
    if (tid < 9) Rq[tid] = site_rot[9 * i + (tid % 3) * 3 + tid / 3];
    __syncthreads();
    build_rotations(lmax, Rq, Dm, rot_ptr, rot_terms);
    __syncthreads();
    double* o = rotd + (int64_t)i * per;
    if (tid == 0) o[0] = sqrt(pair_ab2(shell_xyz, pair_a[pr], pair_b[pr]));
    for (int e = tid; e < nD; e += nth) o[1 + e] = Dm[e];
  }
}

__global__ void __launch_bounds__(128) k_pair_block(int la, int lb, int npairs, int pair_base, int64_t pp_base,
                                                    int64_t rbase, const int* __restrict__ pair_a,
                                                    const int* __restrict__ pair_b,
                                                    const int64_t* __restrict__ pair_ppoff,
                                                    const int* __restrict__ pair_site, int64_t rot_per,
                                                    const double* __restrict__ rotd,
                                                    const int* __restrict__ shell_poff,
                                                    const int* __restrict__ shell_nprim,
                                                    const int64_t* __restrict__ shell_foff,
                                                    const double* __restrict__ prim_exp,
                                                    const double* __restrict__ prim_coef,
                                                    const double* __restrict__ etab, const int* __restrict__ eoff,
                                                    const int* __restrict__ g_rowinfo,
                                                    const int* __restrict__ g_grp,
                                                    const GTerm* __restrict__ g_terms,
                                                    const PPData* __restrict__ ppd,
                                                    const double* __restrict__ rbuf, MolView mv,
                                                    double* __restrict__ out, WorkQueue wq) {
  extern __shared__ double smem[];
  __shared__ long long s_next[2];
  __shared__ unsigned long long s_t0;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lam = la + lb;
  const int nR = n_r(lam);
  const int nWa = (la + 1) * (la + 1), nWb = (lb + 1) * (lb + 1), nW = nWa * nWb;
  const int ws = w_stride(lb), nWs = nWa * ws, nrp = (nW + 31) & ~31;
  const int na = 2 * la + 1, nb = 2 * lb + 1;
  const int lm = la > lb ? la : lb;
  const int nDb = la != lb ? nb * nb : 0;
  double* W = smem;                        // [l1 m1][l2 m2], row stride ws
  double* Dm = W + nWs;                    // D^{la}(Q^T), then D^{lb}(Q^T) when lb != la
  double* tA = Dm + na * na + nb * nb;     // [l1][ma]
  double* tB = tA + (la + 1) * na;         // [l2][mb]
  double* Zb = tB + (lb + 1) * nb;         // [l1 m1][mb]
  double* Vp = Zb + nWa * nb;              // [ma][mb] in the pair frame, later the final block
  double* Yb = Vp + na * nb;               // [ma][mb]
  double* fab = Yb + na * nb;              // [l1][l2]
  double* Rs = fab + (la + 1) * (lb + 1);  // coupling block of one primitive pair
  double* scal = Rs + nR;                  // per primitive pair: prefactor, beta/p, alpha/p
  double* dpow = scal + 4;                 // |b - a|^k, k <= max(la, lb)
  wq_for_each(wq, npairs, s_next, &s_t0, [&](long long wn) {
    const int w = (int)wn;
    const int pr = pair_base + w;
    const int a = pair_a[pr], b = pair_b[pr];
    const double* rd = rotd + (int64_t)pair_site[pr] * rot_per;
    __syncthreads();
    if (tid == 0) {
      const double dist = rd[0];
      double v = 1.0;
      for (int k = 0; k <= lm; ++k) {
        dpow[k] = v;
        v *= dist;
      }
    }
    for (int e = tid; e < na * na; e += nth) Dm[e] = rd[1 + rot_doff(la) + e];
    for (int e = tid; e < nDb; e += nth) Dm[na * na + e] = rd[1 + rot_doff(lb) + e];
    for (int e = tid; e < nWs; e += nth) W[e] = 0.0;
    __syncthreads();
    // translation along z (Eq. 7 with Eq. 8 coefficients, real basis): only nu = 0 survives,
    // t_A(l1, ma) = E^{la}(ma; l1 ma; 0) |b-a|^{la-l1}, t_B(l2, mb) = E^{lb}(mb; l2 mb; 0) (-|b-a|)^{lb-l2}
    for (int e = tid; e < (la + 1) * na; e += nth) {
      const int l1 = e / na, ma = e % na - la, lr = la - l1;
      double v = 0.0;
      if (l1 >= (ma < 0 ? -ma : ma)) {
        v = etab[eoff[la] + translation_offset_dev(la, ma, l1, ma) + lr] * dpow[lr];
      }
      tA[e] = v;
    }
    for (int e = tid; e < (lb + 1) * nb; e += nth) {
      const int l2 = e / nb, mb = e % nb - lb, lr = lb - l2;
      double v = 0.0;
      if (l2 >= (mb < 0 ? -mb : mb)) {
        v = etab[eoff[lb] + translation_offset_dev(lb, mb, l2, mb) + lr] * ((lr & 1) ? -dpow[lr] : dpow[lr]);
      }
      tB[e] = v;
    }
    // coupling (Gaunt) and primitive contraction, in the pair frame
    const int npa = shell_nprim[a], npb = shell_nprim[b];
    const int64_t q0 = pair_ppoff[pr];
    bool live = false;  // uniform over the block
    for (int ij = 0; ij < npa * npb; ++ij) {
      __syncthreads();  // the previous primitive pair is done with Rs, fab and scal
      if (tid == 0) {
        const PPData pd = ppd[q0 + ij];
        scal[0] = pd.pref;
        scal[1] = pd.ra;
        scal[2] = pd.rb;
        scal[3] = pd.kab;
      }
      __syncthreads();
      if (scal[0] == 0.0) continue;  // uniform over the block; the coupling kernel skipped this pair too
      live = true;
      const double pref = scal[0];
      const double* R = rbuf + rbase + (q0 + ij - pp_base) * (int64_t)nR;
      for (int e = tid; e < nR; e += nth) Rs[e] = R[e];
      if (tid < (la + 1) * (lb + 1)) {
        const int l1 = tid / (lb + 1), l2 = tid % (lb + 1);
        double v = pref;
        const double ra = scal[1], rb = scal[2];
        for (int k = 0; k < la - l1; ++k) v *= ra;
        for (int k = 0; k < lb - l2; ++k) v *= rb;
        fab[tid] = v;
      }
      __syncthreads();
      // rows r of one warp form one group: equal trip counts, one coalesced load per term
      for (int r = tid; r < nrp; r += nth) {
        const int info = g_rowinfo[r];
        const int gi = r >> 5, K = g_grp[2 * gi + 1];
        const GTerm* tp = g_terms + g_grp[2 * gi] + (r & 31);
        double acc0 = 0.0, acc1 = 0.0;
        int j = 0;
        for (; j + 1 < K; j += 2) {
          const GTerm g0 = tp[32 * j], g1 = tp[32 * j + 32];
          acc0 = fma(g0.coef, Rs[g0.ridx], acc0);
          acc1 = fma(g1.coef, Rs[g1.ridx], acc1);
        }
        if (j < K) {
          const GTerm g0 = tp[32 * j];
          acc0 = fma(g0.coef, Rs[g0.ridx], acc0);
        }
        if (info >= 0) {
          const int e = info & 0xffff, l1 = (info >> 16) & 15, l2 = (info >> 20) & 15;
          W[e] = fma(fab[l1 * (lb + 1) + l2], acc0 + acc1, W[e]);
        }
      }
    }
    __syncthreads();
    if (!live) {
      // every primitive pair skipped: the block is zero (and omitted from a block-sparse output)
      if (mv.blk_off) return;
      const int64_t fa0 = shell_foff[a], fb0 = shell_foff[b];
      int64_t obase, ld;
      mol_output(mv, pr, obase, ld);
      double* o = out + obase;
      for (int e = tid; e < na * nb; e += nth) {
        const int ma = e / nb, mb = e % nb;
        o[(fa0 + ma) * ld + fb0 + mb] = 0.0;
        if (a != b) o[(fb0 + mb) * ld + fa0 + ma] = 0.0;
      }
      return;
    }
    // V' = t_A W t_B (diagonal in m), first over l2.  Threads are ordered by |m| (m = 0, 1, -1,
    // 2, -2, ...) so that the lanes of a warp run loops of (nearly) equal length.
    for (int e = tid; e < nWa * nb; e += nth) {
      const int q = e / nWa, i1 = e - q * nWa;
      const int amb = (q + 1) >> 1, mb = (q & 1) ? amb : -amb;
      double s = 0.0;
      for (int l2 = amb; l2 <= lb; ++l2) s = fma(tB[l2 * nb + mb + lb], W[i1 * ws + l2 * l2 + l2 + mb], s);
      Zb[i1 * nb + mb + lb] = s;
    }
    __syncthreads();
    for (int e = tid; e < na * nb; e += nth) {
      const int q = e / nb, mb = e - q * nb;
      const int ama = (q + 1) >> 1, ma = (q & 1) ? ama : -ama;
      double s = 0.0;
      for (int l1 = ama; l1 <= la; ++l1) s = fma(tA[l1 * na + ma + la], Zb[(l1 * l1 + l1 + ma) * nb + mb], s);
      Vp[(ma + la) * nb + mb] = s;
    }
    __syncthreads();
    // back to the molecular frame: V = D^{la} V' (D^{lb})^T
    const double* Da = Dm;
    const double* Db = la != lb ? Dm + na * na : Dm;
    for (int e = tid; e < na * nb; e += nth) {
      const int ma = e / nb, mb = e % nb;
      double s = 0.0;
      for (int k = 0; k < nb; ++k) s = fma(Vp[ma * nb + k], Db[mb * nb + k], s);
      Yb[e] = s;
    }
    __syncthreads();
    for (int e = tid; e < na * nb; e += nth) {
      const int ma = e / nb, mb = e % nb;
      double s = 0.0;
      for (int k = 0; k < na; ++k) s = fma(Da[ma * na + k], Yb[k * nb + mb], s);
      Vp[e] = s;
    }
    __syncthreads();
    if (mv.blk_off) {
      // block-sparse output: the block alone, row-major
      const int64_t off = mv.blk_off[pr];
      if (off < 0) return;
      double* o = out + off;
      for (int e = tid; e < na * nb; e += nth) {
        const int ma = e / nb, mb = e % nb;
        o[e] = (a == b && ma > mb) ? Vp[mb * nb + ma] : Vp[e];
      }
      return;
    }
    const int64_t fa0 = shell_foff[a], fb0 = shell_foff[b];
    int64_t obase, ld;
    mol_output(mv, pr, obase, ld);
    double* o = out + obase;
    for (int e = tid; e < na * nb; e += nth) {
      const int ma = e / nb, mb = e % nb;
      // diagonal shell block: the upper triangle serves both halves (exact symmetry)
      const double v = (a == b && ma > mb) ? Vp[mb * nb + ma] : Vp[e];
      o[(fa0 + ma) * ld + fb0 + mb] = v;
      if (a != b) o[(fb0 + mb) * ld + fa0 + ma] = v;
    }
    });
}

// Adjoint of the pair kernel for the electrostatic potential: for one shell pair and a symmetric
// density D, the weights G'[e] of every primitive pair such that
//   sum_{mu in a, nu in b} D_{mu nu} V_{mu nu} (+ the transposed block when a != b) = sum_pp sum_e G'_pp[e] racc_pp[e],
// racc being the unscaled nucleus sums of the coupling kernel.  Steps reversed: the density block is
// rotated into the pair frame (D' = D^la^T D_blk D^lb), weighted by the translation factors
// (Wbar[l1 m1][l2 m2] = t_A(l1, m1) t_B(l2, m2) D'[m1][m2]), pulled back through the Gaunt coupling
// (transposed program, primitive factors) and scaled by 2 pi k! p^{-(k+1)} N_LM.
__host__ __device__ inline size_t esp_adjoint_smem(int la, int lb) {
  const int nWa = (la + 1) * (la + 1), na = 2 * la + 1, nb = 2 * lb + 1, lm = la > lb ? la : lb;
  return sizeof(double) * ((size_t)nWa * w_stride(lb) + na * na + nb * nb + (la + 1) * na + (lb + 1) * nb +
                           3 * na * nb + (la + 1) * (lb + 1) + (la + lb) / 2 + 1 + lm + 1 + 8 + 32);
}

__global__ void __launch_bounds__(128) k_esp_adjoint(int la, int lb, int npairs, int pair_base, int64_t pp_base,
                                                     const int* __restrict__ pair_a, const int* __restrict__ pair_b,
                                                     const int64_t* __restrict__ pair_ppoff,
                                                     const int* __restrict__ pair_site, int64_t rot_per,
                                                     const double* __restrict__ rotd,
                                                     const int* __restrict__ shell_nprim,
                                                     const int64_t* __restrict__ shell_foff,
                                                     const double* __restrict__ etab, const int* __restrict__ eoff,
                                                     const int* __restrict__ gt_ptr, const GTerm* __restrict__ gt_terms,
                                                     const int* __restrict__ rmap, const double* __restrict__ rnorm,
                                                     const PPData* __restrict__ ppd, const double* __restrict__ D,
                                                     int64_t ld, double* __restrict__ gam) {
  extern __shared__ double smem[];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lam = la + lb, nR = n_r(lam);
  const int nWa = (la + 1) * (la + 1), ws = w_stride(lb), nWs = nWa * ws;
  const int na = 2 * la + 1, nb = 2 * lb + 1;
  const int lm = la > lb ? la : lb;
  const int nDb = la != lb ? nb * nb : 0;
  double* Wb = smem;                       // [l1 m1][l2 m2], row stride ws
  double* Dm = Wb + nWs;                   // D^la, then D^lb when lb != la
  double* tA = Dm + na * na + nb * nb;
  double* tB = tA + (la + 1) * na;
  double* Db = tB + (lb + 1) * nb;         // density block [ma][mb]
  double* Y = Db + na * nb;
  double* Dp = Y + na * nb;                // pair-frame density
  double* fab = Dp + na * nb;
  double* scl = fab + (la + 1) * (lb + 1);
  double* dpow = scl + lam / 2 + 1;
  double* scal = dpow + lm + 1;
  for (int w = blockIdx.x; w < npairs; w += gridDim.x) {
    const int pr = pair_base + w;
    const int a = pair_a[pr], b = pair_b[pr];
    const double* rd = rotd + (int64_t)pair_site[pr] * rot_per;
    const int64_t fa0 = shell_foff[a], fb0 = shell_foff[b];
    __syncthreads();
    if (tid == 0) {
      double v = 1.0;
      for (int k = 0; k <= lm; ++k) {
        dpow[k] = v;
        v *= rd[0];
      }
    }
    for (int e = tid; e < na * na; e += nth) Dm[e] = rd[1 + rot_doff(la) + e];
    for (int e = tid; e < nDb; e += nth) Dm[na * na + e] = rd[1 + rot_doff(lb) + e];
    for (int e = tid; e < na * nb; e += nth) {
      const int ma = e / nb, mb = e % nb;
      double v = D[(fa0 + ma) * ld + fb0 + mb];
      if (a != b) v += D[(fb0 + mb) * ld + fa0 + ma];
      Db[e] = v;
    }
    __syncthreads();
    for (int e = tid; e < (la + 1) * na; e += nth) {
      const int l1 = e / na, ma = e % na - la, lr = la - l1;
      tA[e] = l1 >= (ma < 0 ? -ma : ma) ? etab[eoff[la] + translation_offset_dev(la, ma, l1, ma) + lr] * dpow[lr] : 0.0;
    }
    for (int e = tid; e < (lb + 1) * nb; e += nth) {
      const int l2 = e / nb, mb = e % nb - lb, lr = lb - l2;
      tB[e] = l2 >= (mb < 0 ? -mb : mb)
                  ? etab[eoff[lb] + translation_offset_dev(lb, mb, l2, mb) + lr] * ((lr & 1) ? -dpow[lr] : dpow[lr])
                  : 0.0;
    }
    const double* Da = Dm;
    const double* Dbr = la != lb ? Dm + na * na : Dm;
    // Y = D_blk D^lb, then D' = D^la^T Y
    for (int e = tid; e < na * nb; e += nth) {
      const int ma = e / nb, k = e % nb;
      double sacc = 0.0;
      for (int mb = 0; mb < nb; ++mb) sacc = fma(Db[ma * nb + mb], Dbr[mb * nb + k], sacc);
      Y[e] = sacc;
    }
    __syncthreads();
    for (int e = tid; e < na * nb; e += nth) {
      const int k = e / nb, k2 = e % nb;
      double sacc = 0.0;
      for (int ma = 0; ma < na; ++ma) sacc = fma(Da[ma * na + k], Y[ma * nb + k2], sacc);
      Dp[e] = sacc;
    }
    __syncthreads();
    for (int e = tid; e < nWs; e += nth) {
      const int i1 = e / ws, i2 = e % ws;
      double v = 0.0;
      if (i2 < (lb + 1) * (lb + 1)) {
        int l1 = 0, l2 = 0;
        while ((l1 + 1) * (l1 + 1) <= i1) ++l1;
        while ((l2 + 1) * (l2 + 1) <= i2) ++l2;
        const int m1 = i1 - l1 * l1 - l1, m2 = i2 - l2 * l2 - l2;
        v = tA[l1 * na + m1 + la] * tB[l2 * nb + m2 + lb] * Dp[(m1 + la) * nb + m2 + lb];
      }
      Wb[e] = v;
    }
    const int npp = shell_nprim[a] * shell_nprim[b];
    const int64_t q0 = pair_ppoff[pr];
    for (int ij = 0; ij < npp; ++ij) {
      __syncthreads();
      if (tid == 0) {
        const PPData pd = ppd[q0 + ij];
        scal[0] = pd.pref;
        scal[1] = pd.ra;
        scal[2] = pd.rb;
        scal[3] = pd.rp;
      }
      __syncthreads();
      double* g = gam + (q0 + ij - pp_base) * (int64_t)nR;
      if (scal[0] == 0.0) continue;  // skipped by the potential kernel as well
      if (tid < (la + 1) * (lb + 1)) {
        const int l1 = tid / (lb + 1), l2 = tid % (lb + 1);
        double v = scal[0];
        for (int k = 0; k < la - l1; ++k) v *= scal[1];
        for (int k = 0; k < lb - l2; ++k) v *= scal[2];
        fab[tid] = v;
      }
      if (tid <= lam / 2) {
        double sv = 6.283185307179586476925286766559 * scal[3];
        for (int k = 1; k <= tid; ++k) sv *= double(k) * scal[3];
        scl[tid] = sv;
      }
      __syncthreads();
      for (int e = tid; e < nR; e += nth) {
        double acc = 0.0;
        for (int t = gt_ptr[e]; t < gt_ptr[e + 1]; ++t) {
          const GTerm gt = gt_terms[t];
          acc = fma(gt.coef * fab[gt.pad], Wb[gt.ridx], acc);
        }
        const int code = __ldg(rmap + e);
        g[e] = acc * (scl[(code >> 24) & 0xff] * __ldg(rnorm + e));
      }
    }
  }
}

// Overlap block of one shell pair (Eqs. 9-10): both orbitals translated to P (Eq. 7) in the pair
// frame, where the one-centre integrals are diagonal by orthogonality,
//   int S_{l1 m1}(r_P) S_{l2 m2}(r_P) e^{-p r_P^2} = delta delta 4 pi (pi/2)^{1/2} (2 l1 - 1)!! / (2p)^{l1+3/2},
// so S'[ma][mb] = delta_{ma mb} sum_{l1 >= |ma|} t_A(l1, ma) t_B(l1, ma) w(l1) with
// w(l1) = sum_ij c~_i c~_j K_ij (beta/p)^{la-l1} (alpha/p)^{lb-l1} 4 pi (pi/2)^{1/2} (2 l1 - 1)!!/(2p)^{l1+3/2};
// the block is rotated back with D^{la} S' (D^{lb})^T.
//
// One launch covers every class: the shell pairs of all classes form one list of work items, class c holding
// items [first[c], first[c + 1]) (its shell pairs pair_base[c] onwards).  One warp per shell pair, four per
// block, each with its own slice of shared memory and no block-wide barrier: the work per pair is a few
// hundred operations behind a short chain of loads, so what counts is how many pairs are in flight.
constexpr int kOverlapMaxClasses = 64;
struct OverlapClasses {
  int n;
  int first[kOverlapMaxClasses + 1];
  int pair_base[kOverlapMaxClasses];
  unsigned char la[kOverlapMaxClasses], lb[kOverlapMaxClasses];
};
constexpr int kOverlapWarps = 4;

// Shared doubles of one warp for angular momenta up to lm: D^{la} and D^{lb}, t_A and t_B, w(l1), |b - a|^k,
// d(m) and X = D^{la} diag(d).
__host__ __device__ inline int overlap_warp_doubles(int lm) {
  const int n = 2 * lm + 1;
  return 3 * n * n + 2 * (lm + 1) * n + 2 * (lm + 1) + n + 1;
}

__global__ void __launch_bounds__(32 * kOverlapWarps) k_overlap(OverlapClasses cls, int lm_max,
                                                                const int* __restrict__ pair_a,
                                                                const int* __restrict__ pair_b,
                                                                const int64_t* __restrict__ pair_ppoff,
                                                                const int* __restrict__ pair_site, int64_t rot_per,
                                                                const double* __restrict__ rotd,
                                                                const int* __restrict__ shell_nprim,
                                                                const int64_t* __restrict__ shell_foff,
                                                                const double* __restrict__ etab,
                                                                const int* __restrict__ eoff,
                                                                const PPData* __restrict__ ppd, MolView mv,
                                                                double* __restrict__ out) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* wsm = smem + wib * overlap_warp_doubles(lm_max);
  const int total = cls.first[cls.n];
  for (int item = blockIdx.x * kOverlapWarps + wib; item < total; item += gridDim.x * kOverlapWarps) {
    int c = 0, hi = cls.n - 1;  // class of the item (uniform over the warp)
    while (c < hi) {
      const int mid = (c + hi + 1) >> 1;
      if (cls.first[mid] <= item)
        c = mid;
      else
        hi = mid - 1;
    }
    const int la = cls.la[c], lb = cls.lb[c];
    const int pr = cls.pair_base[c] + (item - cls.first[c]);
    const int na = 2 * la + 1, nb = 2 * lb + 1;
    const int lm = la > lb ? la : lb, ln = la < lb ? la : lb;
    const int nDb = la != lb ? nb * nb : 0;
    double* Dm = wsm;  // D^{la}(Q^T), then D^{lb}(Q^T) when lb != la
    double* tA = Dm + na * na + nb * nb;
    double* tB = tA + (la + 1) * na;
    double* wl = tB + (lb + 1) * nb;  // w(l1)
    double* dpow = wl + lm + 1;       // |b - a|^k
    double* dm = dpow + lm + 1;       // d(m), m = -ln..ln
    double* X = dm + 2 * lm + 1;      // [ma][m] = D^{la}[ma][m] d(m)
    const int nm = 2 * ln + 1;
    const int a = pair_a[pr], b = pair_b[pr];
    const double* rd = rotd + (int64_t)pair_site[pr] * rot_per;
    __syncwarp();  // the warp's previous pair is done with its tables
    if (lane == 0) {
      const double dist = rd[0];
      double v = 1.0;
      for (int k = 0; k <= lm; ++k) {
        dpow[k] = v;
        v *= dist;
      }
    }
    for (int e = lane; e < na * na; e += 32) Dm[e] = rd[1 + rot_doff(la) + e];
    for (int e = lane; e < nDb; e += 32) Dm[na * na + e] = rd[1 + rot_doff(lb) + e];
    // radial sums over primitive pairs, one l1 per lane
    if (lane <= ln) {
      const int l1 = lane;
      double dfact = 1.0;
      for (int k = 2 * l1 - 1; k > 1; k -= 2) dfact *= k;
      // 4 pi (pi/2)^{1/2} / 2^{l1 + 3/2} (2 l1 - 1)!!
      double cf = 4.0 * 3.14159265358979323846 * 1.2533141373155002512 * dfact * 0.35355339059327376220;
      for (int k = 0; k < l1; ++k) cf *= 0.5;
      const int64_t q0 = pair_ppoff[pr];
      const int npp = shell_nprim[a] * shell_nprim[b];
      double acc = 0.0;
      for (int ij = 0; ij < npp; ++ij) {
        const PPData pd = ppd[q0 + ij];
        if (pd.pref == 0.0) continue;
        double v = pd.pref * pd.rp / pd.sp;  // p^{-3/2}
        for (int k = 0; k < l1; ++k) v *= pd.rp;
        for (int k = 0; k < la - l1; ++k) v *= pd.ra;
        for (int k = 0; k < lb - l1; ++k) v *= pd.rb;
        acc += v;
      }
      wl[l1] = cf * acc;
    }
    __syncwarp();
    for (int e = lane; e < (la + 1) * na; e += 32) {
      const int l1 = e / na, ma = e % na - la, lr = la - l1;
      tA[e] = l1 >= (ma < 0 ? -ma : ma) ? etab[eoff[la] + translation_offset_dev(la, ma, l1, ma) + lr] * dpow[lr] : 0.0;
    }
    for (int e = lane; e < (lb + 1) * nb; e += 32) {
      const int l2 = e / nb, mb = e % nb - lb, lr = lb - l2;
      tB[e] = l2 >= (mb < 0 ? -mb : mb)
                  ? etab[eoff[lb] + translation_offset_dev(lb, mb, l2, mb) + lr] * ((lr & 1) ? -dpow[lr] : dpow[lr])
                  : 0.0;
    }
    __syncwarp();
    // S' = diag(d), d(m) = sum_{l1 >= |m|} t_A(l1, m) t_B(l1, m) w(l1) for |m| <= min(la, lb), once per pair
    if (lane < nm) {
      const int m = lane - ln, am = m < 0 ? -m : m;
      double d = 0.0;
      for (int l1 = am; l1 <= ln; ++l1) d = fma(tA[l1 * na + m + la] * tB[l1 * nb + m + lb], wl[l1], d);
      dm[lane] = d;
    }
    __syncwarp();
    const double* Da = Dm;
    const double* Db = la != lb ? Dm + na * na : Dm;
    for (int e = lane; e < na * nm; e += 32) {
      const int r = e / nm, j = e - r * nm;
      X[e] = Da[r * na + j - ln + la] * dm[j];
    }
    __syncwarp();
    // S = X (D^{lb})^T; a diagonal block (a == b) takes the entry below its diagonal from the products of the
    // entry above it, so it is exactly symmetric
    const int64_t fa0 = shell_foff[a], fb0 = shell_foff[b];
    int64_t obase, ld;
    mol_output(mv, pr, obase, ld);
    double* o = out + obase;
    for (int e = lane; e < na * nb; e += 32) {
      const int ma = e / nb, mb = e % nb;
      const bool lower = a == b && ma > mb;
      const int r = lower ? mb : ma, q = lower ? ma : mb;
      double s = 0.0;
      for (int j = 0; j < nm; ++j) s = fma(X[r * nm + j], Db[q * nb + j - ln + lb], s);
      o[(fa0 + ma) * ld + fb0 + mb] = s;
      if (a != b) o[(fb0 + mb) * ld + fa0 + ma] = s;
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// Device tables
// ---------------------------------------------------------------------------------------------
namespace {
std::mutex g_tab_mu;
DeviceTables g_tabs[64];
bool g_tab_ok[64] = {};

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& src) {
  cudaError_t e = cudaMalloc((void**)dst, sizeof(T) * (src.empty() ? 1 : src.size()));
  if (e != cudaSuccess) return e;
  if (!src.empty()) e = cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
  return e;
}
}  // namespace

shgo_status device_tables(int device, const DeviceTables** out, std::string* err) {
  if (device < 0 || device >= 64) {
    *err = "device ordinal out of range";
    return SHGO_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_tab_mu);
  if (g_tab_ok[device]) {
    *out = &g_tabs[device];
    return SHGO_OK;
  }
  const Tables& t = tables_host();
  DeviceTables d;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = upload(&d.boys, t.boys);
  if (e == cudaSuccess) e = upload(&d.etab, t.etab);
  if (e == cudaSuccess) e = upload(&d.eoff, t.eoff);
  if (e == cudaSuccess) e = upload(&d.g_rowinfo, t.g_rowinfo);
  if (e == cudaSuccess) e = upload(&d.g_grp, t.g_grp);
  if (e == cudaSuccess) e = upload(&d.gt_ptr, t.gt_ptr);
  if (e == cudaSuccess) e = upload(&d.gt_terms, t.gt_terms);
  if (e == cudaSuccess) e = upload(&d.g_terms, t.g_terms);
  if (e == cudaSuccess) e = upload(&d.rmap, t.rmap);
  if (e == cudaSuccess) e = upload(&d.rnorm, t.rnorm);
  if (e == cudaSuccess) e = upload(&d.rot_ptr, t.rot_ptr);
  if (e == cudaSuccess) e = upload(&d.rot_terms, t.rot_terms);
  if (e == cudaSuccess) e = upload(&d.c2_ptr, t.c2_ptr);
  if (e == cudaSuccess) e = upload(&d.c2_terms, t.c2_terms);
  if (e == cudaSuccess) e = upload(&d.c2_a, t.c2_a);
  if (e == cudaSuccess) e = upload(&d.eri_eps, t.eri_eps);
  if (e == cudaSuccess) e = upload(&d.c2_cbase, t.c2_base);
  if (e == cudaSuccess) e = upload(&d.boys_ff, boys_table_pairs(t.boys));
  if (e == cudaSuccess) e = upload(&d.exp_ff, exp_table_pairs());
  if (e == cudaSuccess) e = upload(&d.rnorm_ff, pairs_of(t.rnorm));
  if (e == cudaSuccess) e = upload(&d.f32_items, coupling_f32_items(t.rmap_off));
  if (e == cudaSuccess) e = upload(&d.d_map0, t.d_map0);
  if (e == cudaSuccess) e = upload(&d.d_mapm, t.d_mapm);
  if (e == cudaSuccess) e = upload(&d.d_raise, t.d_raise);
  if (e == cudaSuccess) e = upload(&d.d_field, t.d_field);
  if (e == cudaSuccess) e = upload(&d.d_low, t.d_low);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_harm, &harm_coef_host(), sizeof(HarmCoef));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_boys, &boys_const_host(), sizeof(BoysConst));
  if (e == cudaSuccess) e = coupling_fp64_setup();
  if (e == cudaSuccess) e = coupling_f32_setup();
  if (e == cudaSuccess) {
    int lof[(kLmax + 1) * (kLmax + 1)];
    for (int l = 0; l <= kLmax; ++l)
      for (int m = -l; m <= l; ++m) lof[harm_index(l, m)] = l;
    e = cudaMemcpyToSymbol(c_lof, lof, sizeof(lof));
  }
  if (e != cudaSuccess) {
    *err = std::string("uploading tables: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SHGO_ERR_OOM : SHGO_ERR_CUDA;
  }
  g_tabs[device] = d;
  g_tab_ok[device] = true;
  *out = &g_tabs[device];
  return SHGO_OK;
}

// The __constant__ recursion coefficients and Boys constants on the current device, without any
// allocation (used by the allocation-free entry point, which keeps its tables elsewhere).
shgo_status upload_constants(std::string* err) {
  cudaError_t e = cudaMemcpyToSymbol(c_harm, &harm_coef_host(), sizeof(HarmCoef));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_boys, &boys_const_host(), sizeof(BoysConst));
  if (e == cudaSuccess) e = coupling_fp64_setup();
  if (e == cudaSuccess) {
    int lof[(kLmax + 1) * (kLmax + 1)];
    for (int l = 0; l <= kLmax; ++l)
      for (int m = -l; m <= l; ++m) lof[harm_index(l, m)] = l;
    e = cudaMemcpyToSymbol(c_lof, lof, sizeof(lof));
  }
  if (e != cudaSuccess) {
    *err = std::string("uploading constants: ") + cudaGetErrorString(e);
    return SHGO_ERR_CUDA;
  }
  return SHGO_OK;
}

// ---------------------------------------------------------------------------------------------
// Launch
// ---------------------------------------------------------------------------------------------
static int grid_cap(int64_t n, int per_sm) {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 152;
  }
  const int64_t cap = (int64_t)nsm * per_sm;
  return (int)(n < cap ? n : cap);
}

namespace {
constexpr int kPoolStreams = 16;
std::mutex g_pool_mu;
cudaStream_t g_pool[64][kPoolStreams];
bool g_pool_ok[64] = {};
bool g_attr_ok[64] = {};

// Per-device pool of non-blocking streams on which the classes of one call run concurrently.
cudaError_t stream_pool(cudaStream_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool_ok[dev]) {
    for (int i = 0; i < kPoolStreams; ++i) {
      e = cudaStreamCreateWithFlags(&g_pool[dev][i], cudaStreamNonBlocking);
      if (e != cudaSuccess) return e;
    }
    g_pool_ok[dev] = true;
  }
  *out = g_pool[dev];
  return cudaSuccess;
}

}  // namespace

cudaError_t pool_streams(cudaStream_t** out, int* n) {
  *n = kPoolStreams;
  return stream_pool(out);
}

int grid_cap_sm(int64_t n, int per_sm) { return grid_cap(n, per_sm); }

namespace {
// Dynamic shared-memory limits, once per device.
void set_kernel_attributes() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (g_attr_ok[dev]) return;
  set_max_dynamic_smem((const void*)k_pair_block);
  g_attr_ok[dev] = true;
}

struct Launcher {
  const DeviceBasis& db;
  const DeviceTables& dt;
  const Tables& th;
  MolView mv;
  const double* centers;
  const double* charges;
  double* out;
  const std::vector<ClassTune>* tune;  // per entry of `work`, or nullptr for the default shapes

  int nch_of(size_t c, int lam) const {
    if (tune && (*tune)[c].nch) return (*tune)[c].nch;
    return lam <= 12 ? 32 : 16;
  }
  int threads_of(size_t c, int la, int lb) const {
    if (tune && (*tune)[c].threads) return (*tune)[c].threads;
    return pair_threads(la, lb);
  }

  // Work queue of class c's coupling (which = 0) or pair (which = 1) launch.  A launch over the whole
  // class of a batch takes its work from the queue in the batch's cost order; the uniform work of one
  // molecule, and the pieces of a class whose coupling buffer is split into regions, stride instead.
  // All keep the time limit.
  // Without a limit and without a queue the launch is the plain strided one (no atomics, no clock).
  WorkQueue queue(const ClassWork& w, size_t c, int which) const {
    WorkQueue q;
    const int* items = which == 0 ? db.cp_items : db.pr_items;
    const bool timed = db.limit_ns != ~0ull, queued = db.region == 0 && items;
    if (!db.ctrl || (!timed && !queued)) return q;
    unsigned char* slot = db.ctrl + kCtrlHead + kCtrlSlot * (2 * c + (size_t)which);
    if (timed) {
      q.t0 = reinterpret_cast<unsigned long long*>(slot + 8);
      q.err = reinterpret_cast<int*>(db.ctrl);
      q.limit_ns = db.limit_ns;
    }
    if (queued) {
      q.qctr = reinterpret_cast<unsigned long long*>(slot);
      q.items = items + (which == 0 ? w.pp_base : (int64_t)w.pair_base);
    }
    return q;
  }
  // Clears class c's two queue slots on `s` (before launching the class again within one call).
  cudaError_t reset(size_t c, cudaStream_t s) const {
    if (!db.ctrl || (db.limit_ns == ~0ull && !db.cp_items && !db.pr_items)) return cudaSuccess;
    return cudaMemsetAsync(db.ctrl + kCtrlHead + kCtrlSlot * 2 * c, 0, 2 * kCtrlSlot, s);
  }

  void coupling(const ClassWork& w, size_t c, int64_t rbase, cudaStream_t s) const {
    if (w.npp == 0) return;
    const int lam = w.la + w.lb;
    const int nch = nch_of(c, lam);
    const int* rmap = dt.rmap + th.rmap_off[lam];
    CouplingArgs a;
    a.q = queue(w, c, 0);
    a.npp = w.npp;
    a.pp_base = w.pp_base;
    a.rbase = rbase;
    a.pp_pair = db.pp_pair;
    a.pair_a = db.pair_a;
    a.shell_xyz = db.shell_xyz;
    a.mv = mv;
    a.centers = centers;
    a.charges = charges;
    a.boys_tab = dt.boys;
    a.rmap = rmap;
    a.rnorm = dt.rnorm + th.rmap_off[lam];
    a.site_rot = db.site_rot;
    a.pair_site = db.pair_site;
    a.ppd = db.ppd;
    a.rbuf = db.rbuf;
    a.one_warp_ok = db.coupling_one_warp;
    if (db.precision != SHGO_PREC_FP64) {
      a.boys_ff = dt.boys_ff;
      a.exp_ff = dt.exp_ff;
      a.items = dt.f32_items + th.rmap_off[lam];
      a.rnorm_ff = dt.rnorm_ff + th.rmap_off[lam];
      launch_coupling_f32(lam, db.precision == SHGO_PREC_FP32_BULK, a, grid_cap(w.npp, 8), s);
      return;
    }
    launch_coupling_fp64(lam, nch, a, grid_cap(w.npp, 8), s);
  }
  void pair(const ClassWork& w, size_t c, int64_t rbase, cudaStream_t s) const {
    if (w.npairs == 0) return;
    const int cid = class_id(w.la, w.lb);
    const size_t sm = pair_smem(w.la, w.lb);
    k_pair_block<<<grid_cap(w.npairs, 16), threads_of(c, w.la, w.lb), sm, s>>>(
        w.la, w.lb, w.npairs, w.pair_base, w.pp_base, rbase, db.pair_a, db.pair_b, db.pair_ppoff, db.pair_site,
        rot_block(db.rot_lmax), db.rotd,
        db.shell_poff, db.shell_nprim, db.shell_foff, db.prim_exp, db.prim_coef, dt.etab, dt.eoff,
        dt.g_rowinfo + th.g_rowbase[cid], dt.g_grp + 2 * th.g_grpbase[cid], dt.g_terms + th.g_termbase[cid],
        db.ppd, db.rbuf, mv, out, queue(w, c, 1));
  }
};

// Clears the queue slots of a basis's control block (counters, start times) on `stream`; the error word
// stays set until the host reads it.
cudaError_t clear_ctrl(const DeviceBasis& db, size_t nclasses, cudaStream_t stream) {
  if (!db.ctrl || (db.limit_ns == ~0ull && !db.cp_items && !db.pr_items)) return cudaSuccess;
  return cudaMemsetAsync(db.ctrl + kCtrlHead, 0, ctrl_bytes(nclasses) - kCtrlHead, stream);
}

// Pieces of a class whose coupling blocks fit `region` doubles, cut between shell pairs.
std::vector<ClassWork> class_chunks(const ClassWork& w, const int64_t* ppoff, int64_t region) {
  std::vector<ClassWork> out;
  const int64_t nR = n_r(w.la + w.lb);
  int q = w.pair_base;
  const int qend = w.pair_base + w.npairs;
  while (q < qend) {
    ClassWork ch{w.la, w.lb, 0, q, 0, ppoff[q]};
    int64_t used = 0;
    while (q < qend && (ch.npairs == 0 || used + (ppoff[q + 1] - ppoff[q]) * nR <= region)) {
      used += (ppoff[q + 1] - ppoff[q]) * nR;
      ++ch.npairs;
      ++q;
    }
    ch.npp = ppoff[q] - ch.pp_base;
    out.push_back(ch);
  }
  return out;
}

// Fork the work of `order` over the pool streams after the work already queued on `stream`, and
// make `stream` wait for all of it.  phase: 0 = coupling only, 1 = pair blocks only, 2 = both.
// With a bounded coupling buffer (db.region > 0) stream i uses region i and runs each of its
// classes chunk by chunk (both kernels per chunk; phase must be 2).
cudaError_t run_concurrent(const Launcher& L, const std::vector<ClassWork>& work, const std::vector<int64_t>& rbases,
                           const std::vector<int>& order, int phase, cudaStream_t stream) {
  cudaStream_t* pool = nullptr;
  cudaError_t e = stream_pool(&pool);
  if (e != cudaSuccess) return e;
  const int ns = (int)std::min<size_t>(order.size(), (size_t)kPoolStreams);
  if (ns == 0) return cudaSuccess;
  cudaEvent_t fork;
  e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e != cudaSuccess) return e;
  cudaEventRecord(fork, stream);
  for (int i = 0; i < ns; ++i) cudaStreamWaitEvent(pool[i], fork, 0);
  for (size_t k = 0; k < order.size(); ++k) {
    const int c = order[k];
    cudaStream_t s = pool[k % ns];
    if (L.db.region > 0) {
      const int64_t rb = (int64_t)(k % ns) * L.db.region;
      for (const ClassWork& ch : class_chunks(work[c], L.db.h_ppoff, L.db.region)) {
        L.coupling(ch, c, rb, s);
        L.pair(ch, c, rb, s);
      }
      continue;
    }
    if (phase != 1) L.coupling(work[c], c, rbases[c], s);
    if (phase != 0) L.pair(work[c], c, rbases[c], s);
  }
  for (int i = 0; i < ns; ++i) {
    cudaEvent_t join;
    e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    if (e != cudaSuccess) break;
    cudaEventRecord(join, pool[i]);
    cudaStreamWaitEvent(stream, join, 0);
    cudaEventDestroy(join);
  }
  cudaEventDestroy(fork);
  return e;
}

std::vector<int64_t> class_rbases(const std::vector<ClassWork>& work) {
  std::vector<int64_t> rbases(work.size());
  int64_t rbase = 0;
  for (size_t c = 0; c < work.size(); ++c) {
    rbases[c] = rbase;
    rbase += work[c].npp * n_r(work[c].la + work[c].lb);
  }
  return rbases;
}

// Classes by decreasing estimated cost (dealt round-robin over the pool streams).
std::vector<int> class_order(const std::vector<ClassWork>& work, double nuclei_per_pair) {
  std::vector<int> order(work.size());
  std::vector<double> cost(work.size());
  for (size_t c = 0; c < work.size(); ++c) {
    order[c] = (int)c;
    const int lam = work[c].la + work[c].lb;
    const double nW = (double)(work[c].la + 1) * (work[c].la + 1) * (work[c].lb + 1) * (work[c].lb + 1);
    cost[c] = (double)work[c].npp * (nuclei_per_pair * n_r(lam) + 8.0 * nW) + (double)work[c].npairs * 30.0 * nW;
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  return order;
}

shgo_status launch_error(std::string* err) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    *err = std::string("kernel launch: ") + cudaGetErrorString(e);
    return SHGO_ERR_CUDA;
  }
  return SHGO_OK;
}
}  // namespace

shgo_status launch_nuclear_attraction(const DeviceBasis& db, const DeviceTables& dt,
                                      const std::vector<ClassWork>& work, int64_t nbf, int64_t ncenters,
                                      const double* centers, const double* charges, double* out,
                                      cudaStream_t stream, std::string* err, cudaEvent_t* events, bool concurrent,
                                      const int64_t* blk_off, int64_t out_doubles) {
  if (events) cudaEventRecord(events[0], stream);
  if (nbf == 0 || ncenters == 0) {
    if (events) cudaEventRecord(events[1], stream);
  }
  if (nbf == 0) {
    if (events) cudaEventRecord(events[2], stream);
    return SHGO_OK;
  }
  if (ncenters == 0) {
    const size_t n = blk_off ? (size_t)out_doubles : (size_t)nbf * (size_t)nbf;
    cudaError_t e = n ? cudaMemsetAsync(out, 0, sizeof(double) * n, stream) : cudaSuccess;
    if (events) cudaEventRecord(events[2], stream);
    if (e != cudaSuccess) {
      *err = cudaGetErrorString(e);
      return SHGO_ERR_CUDA;
    }
    return SHGO_OK;
  }
  set_kernel_attributes();
  const Tables& th = tables_host();
  const std::vector<int64_t> rbases = class_rbases(work);
  MolView mv;
  mv.ncenters = ncenters;
  mv.nbf = nbf;
  mv.blk_off = blk_off;
  const Launcher L{db, dt, th, mv, centers, charges, out, nullptr};
  cudaError_t e = clear_ctrl(db, work.size(), stream);
  if (events && db.region > 0) {
    *err = "phase timing needs the whole coupling buffer; this basis uses bounded regions";
    return SHGO_ERR_INVALID_ARG;
  }
  if (e != cudaSuccess) {
  } else if (!concurrent) {
    for (size_t c = 0; c < work.size(); ++c) L.coupling(work[c], c, rbases[c], stream);
    if (events) cudaEventRecord(events[1], stream);
    for (size_t c = 0; c < work.size(); ++c) L.pair(work[c], c, rbases[c], stream);
  } else {
    const std::vector<int> order = class_order(work, (double)ncenters);
    if (events) {
      e = run_concurrent(L, work, rbases, order, 0, stream);
      cudaEventRecord(events[1], stream);
      if (e == cudaSuccess) e = run_concurrent(L, work, rbases, order, 1, stream);
    } else {
      e = run_concurrent(L, work, rbases, order, 2, stream);
    }
  }
  if (events) cudaEventRecord(events[2], stream);
  if (e != cudaSuccess) {
    *err = std::string("kernel launch: ") + cudaGetErrorString(e);
    return SHGO_ERR_CUDA;
  }
  return launch_error(err);
}

shgo_status launch_class_timed(const DeviceBasis& db, const DeviceTables& dt, const std::vector<ClassWork>& work,
                               const MolView& mv, const double* centers, const double* charges, double* out,
                               cudaStream_t stream, double* ms, std::string* err) {
  if (work.empty()) return SHGO_OK;
  set_kernel_attributes();
  const Tables& th = tables_host();
  const std::vector<int64_t> rbases = class_rbases(work);
  const Launcher L{db, dt, th, mv, centers, charges, out, nullptr};
  std::vector<cudaEvent_t> ev(3 * work.size(), nullptr);
  cudaError_t e = clear_ctrl(db, work.size(), stream);
  for (auto& x : ev)
    if (e == cudaSuccess) e = cudaEventCreate(&x);
  for (size_t c = 0; c < work.size() && e == cudaSuccess; ++c) {
    cudaEventRecord(ev[3 * c], stream);
    L.coupling(work[c], c, rbases[c], stream);
    cudaEventRecord(ev[3 * c + 1], stream);
    L.pair(work[c], c, rbases[c], stream);
    cudaEventRecord(ev[3 * c + 2], stream);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(ev.back());
  for (size_t c = 0; c < work.size() && e == cudaSuccess; ++c) {
    float a = 0, b = 0;
    e = cudaEventElapsedTime(&a, ev[3 * c], ev[3 * c + 1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[3 * c + 1], ev[3 * c + 2]);
    ms[2 * c] = a;
    ms[2 * c + 1] = b;
  }
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  if (e != cudaSuccess) {
    *err = std::string("class timing: ") + cudaGetErrorString(e);
    return SHGO_ERR_CUDA;
  }
  return SHGO_OK;
}

shgo_status launch_batched(const DeviceBasis& db, const DeviceTables& dt, const std::vector<ClassWork>& work,
                           const MolView& mv, double nuclei_per_pair, const double* centers, const double* charges,
                           double* out, const std::vector<ClassTune>* tune, cudaStream_t stream, std::string* err) {
  if (work.empty()) return SHGO_OK;
  set_kernel_attributes();
  const Tables& th = tables_host();
  const std::vector<int64_t> rbases = class_rbases(work);
  const Launcher L{db, dt, th, mv, centers, charges, out, tune};
  cudaError_t e = clear_ctrl(db, work.size(), stream);
  if (e == cudaSuccess) e = run_concurrent(L, work, rbases, class_order(work, nuclei_per_pair), 2, stream);
  if (e != cudaSuccess) {
    *err = std::string("kernel launch: ") + cudaGetErrorString(e);
    return SHGO_ERR_CUDA;
  }
  return launch_error(err);
}

shgo_status autotune_batched(const DeviceBasis& db, const DeviceTables& dt, const std::vector<ClassWork>& work,
                             const MolView& mv, const double* centers, const double* charges, double* out,
                             std::vector<ClassTune>* tune, cudaStream_t stream, std::string* err) {
  // Each candidate shape of a class runs the class's real work once (the output is rewritten by
  // every candidate, so the call's result stays exact); the fastest by CUDA events is kept.
  set_kernel_attributes();
  const Tables& th = tables_host();
  const std::vector<int64_t> rbases = class_rbases(work);
  tune->assign(work.size(), ClassTune{});
  clear_ctrl(db, work.size(), stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto time_it = [&](auto&& fn) {
    cudaEventRecord(e0, stream);
    fn();
    cudaEventRecord(e1, stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  };
  for (size_t c = 0; c < work.size(); ++c) {
    const ClassWork& w = work[c];
    const std::vector<ClassWork> chunks =
        db.region > 0 ? class_chunks(w, db.h_ppoff, db.region) : std::vector<ClassWork>{w};
    const int64_t rb = db.region > 0 ? 0 : rbases[c];
    const ClassWork& first = chunks[0];
    std::vector<ClassTune> trial(work.size());
    const Launcher L{db, dt, th, mv, centers, charges, out, &trial};
    float best = 1e30f;
    int best_nch = 32;
    for (int nch : {16, 32}) {
      trial[c].nch = nch;
      L.reset(c, stream);
      L.coupling(first, c, rb, stream);  // warm
      L.reset(c, stream);
      const float ms = time_it([&] { L.coupling(first, c, rb, stream); });
      if (ms < best) {
        best = ms;
        best_nch = nch;
      }
    }
    trial[c].nch = best_nch;
    L.reset(c, stream);
    L.coupling(first, c, rb, stream);  // the kept shape leaves its coupling block in place
    (*tune)[c].nch = best_nch;
    best = 1e30f;
    int best_thr = pair_threads(w.la, w.lb);
    for (int thr : {32, 64, 128}) {
      trial[c].threads = thr;
      L.reset(c, stream);
      L.pair(first, c, rb, stream);  // warm
      L.reset(c, stream);
      const float ms = time_it([&] { L.pair(first, c, rb, stream); });
      if (ms < best) {
        best = ms;
        best_thr = thr;
      }
    }
    (*tune)[c].threads = best_thr;
    trial[c].threads = best_thr;
    for (size_t k = 0; k < chunks.size(); ++k) {  // the whole class with the kept shapes
      L.reset(c, stream);
      if (k > 0) L.coupling(chunks[k], c, rb, stream);
      L.pair(chunks[k], c, rb, stream);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return launch_error(err);
}

shgo_status launch_pair_rotations(const DeviceBasis& db, const DeviceTables& dt, cudaStream_t stream, std::string* err) {
  if (db.n_sites == 0) return SHGO_OK;
  const size_t sm = sizeof(double) * ((size_t)rot_doff(db.rot_lmax + 1) + 16);
  k_pair_rotations<<<grid_cap(db.n_sites, 16), 64, sm, stream>>>(db.n_sites, db.rot_lmax, db.site_rep, db.pair_a,
                                                                   db.pair_b, db.site_rot, db.shell_xyz, dt.rot_ptr,
                                                                   dt.rot_terms, db.rotd);
  return launch_error(err);
}

shgo_status launch_pair_build(const DeviceBasis& db, int64_t npp, cudaStream_t stream, std::string* err) {
  if (npp == 0) return SHGO_OK;
  const int64_t blocks = std::min<int64_t>((npp + 255) / 256, 152 * 32);
  k_pair_build<<<(int)blocks, 256, 0, stream>>>(npp, db.pp_pair, db.pp_ij, db.pair_a, db.pair_b, db.shell_xyz,
                                                 db.shell_l, db.shell_poff, db.prim_exp, db.prim_coef, db.prim_bound,
                                                 db.ppd);
  return launch_error(err);
}

shgo_status launch_pair_live(const DeviceBasis& db, int64_t npairs, int64_t npp, uint8_t* live, cudaStream_t stream,
                             std::string* err) {
  if (npairs == 0) return SHGO_OK;
  const int64_t blocks = std::min<int64_t>((npairs + 255) / 256, 152 * 32);
  k_pair_live<<<(int)blocks, 256, 0, stream>>>(npairs, db.pair_ppoff, npp, db.ppd, live);
  return launch_error(err);
}

shgo_status live_counts(const DeviceBasis& db, const std::vector<ClassWork>& work, int64_t npairs, int64_t npp,
                        const int* pair_mol, const int64_t* mol_nc, std::vector<int64_t>& live_pp,
                        std::vector<int64_t>& live_pairs, std::vector<double>& live_cent, std::string* err) {
  const int nc = (int)work.size();
  live_pp.assign(nc, 0);
  live_pairs.assign(nc, 0);
  live_cent.assign(nc, 0.0);
  if (nc == 0 || npairs == 0) return SHGO_OK;
  std::vector<int> cls(nc);
  for (int c = 0; c < nc; ++c) cls[c] = work[c].pair_base;
  // one scratch block: class starts, then the three counters
  const size_t b_cls = sizeof(int) * nc, b_cnt = sizeof(unsigned long long) * nc, b_cent = sizeof(double) * nc;
  unsigned char* scratch = nullptr;
  cudaError_t e = cudaMalloc((void**)&scratch, b_cls + 2 * b_cnt + b_cent + 64);
  if (e == cudaSuccess) e = cudaMemset(scratch, 0, b_cls + 2 * b_cnt + b_cent + 64);
  int* d_cls = reinterpret_cast<int*>(scratch);
  unsigned long long* d_pp = reinterpret_cast<unsigned long long*>(scratch + ((b_cls + 15) & ~(size_t)15));
  unsigned long long* d_pairs = d_pp + nc;
  double* d_cent = reinterpret_cast<double*>(d_pairs + nc);
  if (e == cudaSuccess) e = cudaMemcpy(d_cls, cls.data(), b_cls, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const int64_t blocks = std::min<int64_t>((npairs + 255) / 256, 152 * 16);
    k_live_counts<<<(int)blocks, 256>>>((int)npairs, nc, d_cls, db.pair_ppoff, npp, db.ppd, pair_mol, mol_nc, d_pp,
                                        d_pairs, d_cent);
    e = cudaGetLastError();
  }
  std::vector<unsigned long long> hp(nc), hq(nc);
  if (e == cudaSuccess) e = cudaMemcpy(hp.data(), d_pp, b_cnt, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(hq.data(), d_pairs, b_cnt, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(live_cent.data(), d_cent, b_cent, cudaMemcpyDeviceToHost);
  cudaFree(scratch);
  if (e != cudaSuccess) {
    *err = std::string("counting live primitive pairs: ") + cudaGetErrorString(e);
    return SHGO_ERR_CUDA;
  }
  for (int c = 0; c < nc; ++c) {
    live_pp[c] = (int64_t)hp[c];
    live_pairs[c] = (int64_t)hq[c];
  }
  return SHGO_OK;
}

shgo_status launch_esp(const DeviceBasis& db, const DeviceTables& dt, const std::vector<ClassWork>& work,
                       int64_t nbf, const double* D, int64_t npoints, const double* points, double* phi, double* gbuf,
                       bool gradient, cudaStream_t stream, std::string* err) {
  ensure_max_dynamic_smem((const void*)k_esp_adjoint);
  const Tables& th = tables_host();
  cudaError_t e =
      cudaMemsetAsync(phi, 0, sizeof(double) * (size_t)std::max<int64_t>(npoints, 1) * (gradient ? 3 : 1), stream);
  int64_t gb = 0;
  for (const ClassWork& w : work) {
    if (w.npairs == 0 || e != cudaSuccess) continue;
    const int lam = w.la + w.lb, cid = class_id(w.la, w.lb);
    double* g = gbuf + gb;
    k_esp_adjoint<<<grid_cap(w.npairs, 16), pair_threads(w.la, w.lb), esp_adjoint_smem(w.la, w.lb), stream>>>(
        w.la, w.lb, w.npairs, w.pair_base, w.pp_base, db.pair_a, db.pair_b, db.pair_ppoff, db.pair_site,
        rot_block(db.rot_lmax), db.rotd, db.shell_nprim, db.shell_foff, dt.etab, dt.eoff,
        dt.gt_ptr + th.gt_base[cid], dt.gt_terms + th.gt_termbase[cid], dt.rmap + th.rmap_off[lam],
        dt.rnorm + th.rmap_off[lam], db.ppd, D, nbf, g);
    e = cudaGetLastError();
    if (e != cudaSuccess || npoints == 0) {
      gb += w.npp * n_r(lam);
      continue;
    }
    EspArgs A;
    A.npp = w.npp;
    A.pp_base = w.pp_base;
    A.pp_pair = db.pp_pair;
    A.pair_a = db.pair_a;
    A.shell_xyz = db.shell_xyz;
    A.site_rot = db.site_rot;
    A.pair_site = db.pair_site;
    A.ppd = db.ppd;
    A.boys_tab = dt.boys;
    A.rmap = dt.rmap + th.rmap_off[lam];
    A.gam = g;
    A.npoints = npoints;
    A.points = points;
    A.phi = phi;
    const int pts = gradient ? 16 : 32;
    A.nchunks = (int)((npoints + pts - 1) / pts);
    A.nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(w.npp, (int64_t)152 * 8 / A.nchunks));
    e = gradient ? launch_esp_grad_fp64(lam, A, stream) : launch_esp_fp64(lam, A, stream);
    gb += w.npp * n_r(lam);
  }
  if (e != cudaSuccess) {
    *err = std::string("electrostatic potential: ") + cudaGetErrorString(e);
    return SHGO_ERR_CUDA;
  }
  return SHGO_OK;
}

// Two-centre Coulomb integrals (a|b) of one class, one block per shell pair.  With Eq. 3 each primitive is
// N (2 alpha)^{-l} S_l(grad_A) exp(-alpha |r - A|^2), so for R = A - B (grad_B = -grad_R on functions of R)
//   (a|b) = c_a c_b (2 alpha)^{-la} (2 beta)^{-lb} (-1)^lb S_la(grad_R) S_lb(grad_R) g(|R|^2),
//   g(u) = 2 pi^{5/2} / (alpha beta sqrt(alpha + beta)) F_0(rho u),  rho = alpha beta / (alpha + beta),
// the Coulomb integral of two s Gaussians.  The product rule of solid harmonics (the Gaunt coupling of the
// pair kernel) gives S_la S_lb = sum_{L,M} G |v|^{2k} S_LM with k = (la + lb - L)/2, Hobson's theorem
// S_LM(grad) f(u) = 2^L S_LM(R) f^{(L)}(u), and the Laplacian of S_LM(R) f(u) is S_LM(R) (4u f'' + (4L + 6) f'),
// so every term is 2^L S_LM(R) sum_j a_{k,j}(L) u^j g^{(L+k+j)}(u), with
// g^{(n)}(u) = 2 pi^{5/2} / (alpha beta sqrt(alpha + beta)) (-rho)^n F_n(rho u).
// Threads: one primitive pair each for the Boys values, one L each for the radial sums over primitive pairs,
// one block entry each for the coupling; the block and its transpose are written as in the overlap.
// Real solid harmonics S_lm(x, y, z), l <= lmax, by columns: thread t of nth takes the columns
// m = t - lmax, t + nth - lmax, ...; each walks the diagonal chain S_{l+1,+-(l+1)} = c_l (x S_ll -+ y S_{l,-l})
// (S_11 = x, S_1-1 = y) up to |m| and then S_{l+1,m} = a_lm z S_lm - b_lm r^2 S_{l-1,m} (the recursion of
// solid_harmonics, whose entries it reproduces operation for operation) into S[l^2 + l + m].
__device__ void solid_harmonics_columns(int lmax, double x, double y, double z, double* S, int tid, int nth) {
  const double r2 = x * x + y * y + z * z;
  for (int col = tid; col < 2 * lmax + 1; col += nth) {
    const int m = col - lmax, am = m < 0 ? -m : m;
    double sp = 1.0, sm = 0.0;  // S_{l,l}, S_{l,-l}
    if (am >= 1) {
      sp = x;
      sm = y;
      for (int l = 1; l < am; ++l) {
        const double c = c_harm.c[l];
        const double np = c * (x * sp - y * sm), nm = c * (y * sp + x * sm);
        sp = np;
        sm = nm;
      }
    }
    double prv = 0.0, cur = m < 0 ? sm : sp;
    S[am * am + am + m] = cur;
    for (int l = am; l < lmax; ++l) {
      const int k = l * l + l + m;
      double v = c_harm.a[k] * (z * cur);
      if (m > -l && m < l) v -= c_harm.b[k] * (r2 * prv);
      S[(l + 1) * (l + 1) + l + 1 + m] = v;
      prv = cur;
      cur = v;
    }
  }
}

__global__ void __launch_bounds__(64) k_coulomb2c(int la, int lb, int npairs, int pair_base,
                                                  const int* __restrict__ pair_a, const int* __restrict__ pair_b,
                                                  const double* __restrict__ shell_xyz,
                                                  const int* __restrict__ shell_poff, const int* __restrict__ shell_nprim,
                                                  const int64_t* __restrict__ shell_foff,
                                                  const double* __restrict__ prim_exp,
                                                  const double* __restrict__ prim_coef,
                                                  const double* __restrict__ boys_tab, const int* __restrict__ c2_ptr,
                                                  const GTerm* __restrict__ c2_terms, const double* __restrict__ c2_a,
                                                  MolView mv, double* __restrict__ out) {
  extern __shared__ double smem[];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lam = la + lb, na = 2 * la + 1, nb = 2 * lb + 1, nf = lam + 1;
  double* S = smem;                      // [(lam + 1)^2] S_LM(R)
  double* X = S + nf * nf;               // [lam + 1] radial sums over primitive pairs, by L
  double* F = X + nf;                    // [64][lam + 1] Boys values of a batch of primitive pairs
  double* pf = F + 64 * nf;              // [64] prefactors
  double* mr = pf + 64;                  // [64] -rho
  double* ru = mr + 64;                  // [1] |R|^2
  for (int w = blockIdx.x; w < npairs; w += gridDim.x) {
    const int pr = pair_base + w;
    const int a = pair_a[pr], b = pair_b[pr];
    const double Rx = shell_xyz[3 * a] - shell_xyz[3 * b], Ry = shell_xyz[3 * a + 1] - shell_xyz[3 * b + 1],
                 Rz = shell_xyz[3 * a + 2] - shell_xyz[3 * b + 2];
    const double u = Rx * Rx + Ry * Ry + Rz * Rz;
    __syncthreads();  // the previous pair is done with S and X
    solid_harmonics_columns(lam, Rx, Ry, Rz, S, tid, nth);
    if (tid == 0) *ru = u;
    if (tid < nf) X[tid] = 0.0;
    const int npa = shell_nprim[a], npb = shell_nprim[b], npp = npa * npb;
    for (int q0 = 0; q0 < npp; q0 += 64) {
      __syncthreads();  // the previous batch is consumed
      const int q = q0 + tid;
      if (tid < 64 && q < npp) {
        const int i = q / npb, j = q - i * npb;
        const double al = prim_exp[shell_poff[a] + i], be = prim_exp[shell_poff[b] + j];
        const double rho = al * be / (al + be);
        double v = prim_coef[shell_poff[a] + i] * prim_coef[shell_poff[b] + j] * 6.2831853071795864769 *
                   5.5683279968317078453 / (al * be * sqrt(al + be));  // 2 pi^{5/2} = 2 pi x pi^{3/2}
        const double ia = 0.5 / al, ib = 0.5 / be;
        for (int k = 0; k < la; ++k) v *= ia;
        for (int k = 0; k < lb; ++k) v *= ib;
        pf[tid] = (lb & 1) ? -v : v;
        mr[tid] = -rho;
        boys_eval(lam, rho * u, F + tid * nf, 1, boys_tab, c_boys);
      }
      __syncthreads();
      const int nq = min(64, npp - q0);
      // radial sums: one L per thread (L = la - lb, la - lb + 2, ..., la + lb)
      const int L = la - lb + 2 * tid;
      if (L <= lam) {
        const int k = (lam - L) / 2;
        const double* ak = c2_a + ((size_t)L * (kC2K + 1) + k) * (kC2K + 1);
        double acc = X[L];
        for (int t = 0; t < nq; ++t) {
          const double* Ft = F + t * nf;
          double mrp = 1.0;  // (-rho)^{L+k}
          for (int n = 0; n < L + k; ++n) mrp *= mr[t];
          double s = 0.0, uj = 1.0;
          for (int j = 0; j <= k; ++j) {
            s = fma(ak[j] * uj, mrp * Ft[L + k + j], s);
            uj *= u;
            mrp *= mr[t];
          }
          acc = fma(pf[t], s, acc);
        }
        X[L] = acc;
      }
    }
    __syncthreads();
    if (tid <= lam) X[tid] = ldexp(X[tid], tid);  // 2^L X_L
    __syncthreads();
    // coupling: sum over (L, M) of G 2^L S_LM(R) X_L, one block entry per thread
    const int64_t fa0 = shell_foff[a], fb0 = shell_foff[b];
    int64_t obase, ld;
    mol_output(mv, pr, obase, ld);
    double* o = out + obase;
    const int* ptr = c2_ptr;
    for (int e = tid; e < na * nb; e += nth) {
      double v = 0.0;
      for (int t = ptr[e]; t < ptr[e + 1]; ++t) {
        const GTerm g = c2_terms[t];
        v = fma(g.coef * S[g.ridx], X[g.pad], v);
      }
      const int ma = e / nb, mb = e - ma * nb;
      o[(fa0 + ma) * ld + fb0 + mb] = v;
      if (a != b) o[(fb0 + mb) * ld + fa0 + ma] = v;
    }
  }
}

size_t coulomb2c_smem(int la, int lb) {
  const int nf = la + lb + 1;
  return sizeof(double) * ((size_t)nf * nf + nf + 64 * (size_t)nf + 64 + 64 + 1 + 8);
}

// Launches `launch(w, s)` for every non-empty class of `work`, the classes (which write disjoint blocks) spread
// over the pool streams, the costliest first (cost: an estimate of the class's work), after the work already
// queued on `stream`, which then waits for all of them.
template <typename Cost, typename Launch>
cudaError_t classes_concurrent(const std::vector<ClassWork>& work, cudaStream_t stream, Cost&& cost, Launch&& launch) {
  cudaStream_t* pool = nullptr;
  cudaError_t e = stream_pool(&pool);
  std::vector<int> order;
  for (size_t c = 0; c < work.size(); ++c)
    if (work[c].npairs > 0) order.push_back((int)c);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(work[x]) > cost(work[y]); });
  const int ns = (int)std::min<size_t>(order.size(), (size_t)kPoolStreams);
  cudaEvent_t fork = nullptr;
  if (e == cudaSuccess && ns > 0) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e == cudaSuccess && fork) e = cudaEventRecord(fork, stream);
  for (int i = 0; i < ns && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(pool[i], fork, 0);
  for (size_t k = 0; k < order.size() && e == cudaSuccess; ++k) {
    launch(work[order[k]], pool[k % ns]);
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
  return e;
}

shgo_status launch_coulomb2c(const DeviceBasis& db, const DeviceTables& dt, const Tables& th,
                             const std::vector<ClassWork>& work, const MolView& mv, double* out, cudaStream_t stream,
                             std::string* err) {
  const cudaError_t e = classes_concurrent(
      work, stream,
      [](const ClassWork& w) {
        return (double)w.npp * (w.la + w.lb + 1) + (double)w.npairs * (2 * w.la + 1) * (2 * w.lb + 1);
      },
      [&](const ClassWork& w, cudaStream_t s) {
        k_coulomb2c<<<grid_cap(w.npairs, 16), 64, coulomb2c_smem(w.la, w.lb), s>>>(
            w.la, w.lb, w.npairs, w.pair_base, db.pair_a, db.pair_b, db.shell_xyz, db.shell_poff, db.shell_nprim,
            db.shell_foff, db.prim_exp, db.prim_coef, dt.boys, dt.c2_ptr + th.c2_base[class_id(w.la, w.lb)],
            dt.c2_terms, dt.c2_a, mv, out);
      });
  if (e != cudaSuccess) {
    *err = std::string("two-centre launch: ") + cudaGetErrorString(e);
    return SHGO_ERR_CUDA;
  }
  return launch_error(err);
}

// ---------------------------------------------------------------------------------------------
// Four-centre electron-repulsion integrals (ab|cd) (Eqs. 13-15), in the SHGO form re-derived from
// Eqs. 3 and 7-8 (the printed Eq. 15 carries the same-centre coupling defect of Eq. 12):
//  1. Each pair is translated to its product centre (Eq. 7, real addition theorem) and its two
//     harmonics at P coupled by the Gaunt coefficients:
//       phi_a phi_b = c c' K_AB sum_{L,M,k} Y[L,M,k] r_P^{2k} S_LM(r_P) e^{-p r_P^2}.
//  2. r^{2k} S_LM e^{-pr^2} = sum_n eps_{k,n}(L) p^{-(k+n)} Laplacian^n [S_LM e^{-pr^2}], and by Eq. 3
//     S_LM(r_P) e^{-p r_P^2} = (2p)^{-L} S_LM(grad_P) e^{-p r_P^2}, so the pair is
//       sum_{L,M,n} D[L,M,n] Laplacian_P^n S_LM(grad_P) e^{-p r_P^2}
//     (k_eri_dist writes D per primitive pair and block entry (ma, mb)).
//  3. For two such terms at P and Q, with R = P - Q and u = |R|^2, every operator acts on the s-s integral
//     g(u) = 2 pi^{5/2} / (p q sqrt(p + q)) F_0(rho u), rho = pq/(p + q), as grad_P = grad_R, grad_Q = -grad_R:
//       (-1)^{L2} Laplacian^{n1+n2} S_L1M1(grad) S_L2M2(grad) g
//         = (-1)^{L2} sum_{L,M} G(L1M1, L2M2; LM) 2^L S_LM(R) sum_j a_{K,j}(L) u^j g^{(L+K+j)}(u),
//     K = (L1 + L2 - L)/2 + n1 + n2 (product rule, Hobson's theorem and Laplacian_L of the two-centre
//     kernel), g^{(N)}(u) = 2 pi^{5/2} / (p q sqrt(p + q)) (-rho)^N F_N(rho u).
//  4. (ab|cd) = sum over primitive quartets of D_ab I D_cd^T (k_eri_part, summed by k_eri_reduce).
// The entries (L, M, n) of a pair use the (L, M, k) layout of the coupling buffer for Lambda = la + lb.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int lmk_first(int lam, int L) {
  int off = 0;
  for (int Lp = 0; Lp < L; ++Lp) off += (2 * Lp + 1) * (kmax_of(lam, Lp) + 1);
  return off;
}

__device__ __forceinline__ int l_of_index(int h) {
  int L = (int)sqrtf((float)h);
  while (L * L > h) --L;
  while ((L + 1) * (L + 1) <= h) ++L;
  return L;
}

// One primitive pair per block iteration: D[(ma mb) nr + e], e over the (L, M, n) entries of
// Lambda = la + lb, for the class's primitive pairs pp_base .. pp_base + npp (dist: the class block).
__global__ void __launch_bounds__(128) k_eri_dist(int la, int lb, int64_t npp, int64_t pp_base,
                                                  const int* __restrict__ pp_pair, const int* __restrict__ pp_ij,
                                                  const int* __restrict__ pair_a, const int* __restrict__ pair_b,
                                                  const double* __restrict__ shell_xyz,
                                                  const int* __restrict__ shell_poff,
                                                  const double* __restrict__ prim_exp,
                                                  const double* __restrict__ prim_coef, const double* __restrict__ etab,
                                                  const int* __restrict__ eoff, const int* __restrict__ gt_ptr,
                                                  const GTerm* __restrict__ gt_terms, const double* __restrict__ eps,
                                                  double* __restrict__ dist) {
  extern __shared__ double smem[];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lam = la + lb, na = 2 * la + 1, nb = 2 * lb + 1, nr = n_r(lam), nh = n_harm(lam);
  const int nha = n_harm(la), nhb = n_harm(lb), ws = w_stride(lb);
  double* S = smem;             // [nha] S_lm(B - A)
  double* EA = S + nha;         // [na][nha] translation of a to P
  double* EB = EA + na * nha;   // [nb][nhb] translation of b to P
  for (int64_t w = blockIdx.x; w < npp; w += gridDim.x) {
    const int64_t pp = pp_base + w;
    const int pr = pp_pair[pp], ij = pp_ij[pp];
    const int a = pair_a[pr], b = pair_b[pr];
    const int ia = shell_poff[a] + (ij >> 8), ib = shell_poff[b] + (ij & 255);
    const double al = prim_exp[ia], be = prim_exp[ib], p = al + be, ip = 1.0 / p;
    const double dx = shell_xyz[3 * b] - shell_xyz[3 * a], dy = shell_xyz[3 * b + 1] - shell_xyz[3 * a + 1],
                 dz = shell_xyz[3 * b + 2] - shell_xyz[3 * a + 2];
    __syncthreads();  // the previous primitive pair is done with S, EA, EB
    solid_harmonics_columns(la, dx, dy, dz, S, tid, nth);
    __syncthreads();
    // S_la,ma(r - A) = sum_{l1 m1} EA[ma][l1 m1] S_l1m1(r - P): P - A = (beta/p)(B - A)
    for (int e = tid; e < na * nha; e += nth) {
      const int ma = e / nha - la, i1 = e - (ma + la) * nha, l1 = c_lof[i1], m1 = i1 - l1 * l1 - l1, lr = la - l1;
      const double* t = etab + eoff[la] + translation_offset_dev(la, ma, l1, m1);
      double v = 0.0, f = 1.0;
      for (int nu = -lr; nu <= lr; ++nu) v = fma(t[nu + lr], S[lr * lr + lr + nu], v);
      for (int k = 0; k < lr; ++k) f *= be * ip;
      EA[e] = v * f;
    }
    // P - B = (alpha/p)(A - B) and S_l(A - B) = (-1)^l S_l(B - A)
    for (int e = tid; e < nb * nhb; e += nth) {
      const int mb = e / nhb - lb, i2 = e - (mb + lb) * nhb, l2 = c_lof[i2], m2 = i2 - l2 * l2 - l2, lr = lb - l2;
      const double* t = etab + eoff[lb] + translation_offset_dev(lb, mb, l2, m2);
      double v = 0.0, f = 1.0;
      for (int nu = -lr; nu <= lr; ++nu) v = fma(t[nu + lr], S[lr * lr + lr + nu], v);
      for (int k = 0; k < lr; ++k) f *= -al * ip;
      EB[e] = v * f;
    }
    __syncthreads();
    const double ab2 = dx * dx + dy * dy + dz * dz;
    const double pref = prim_coef[ia] * prim_coef[ib] * exp(-al * be * ip * ab2);
    double* out = dist + w * (int64_t)(na * nb) * nr;
    // one (ma mb, L, M) per thread: Y[L,M,k] for every k by the Gaunt coupling, then the Laplacian form
    for (int g = tid; g < na * nb * nh; g += nth) {
      const int mamb = g / nh, h = g - mamb * nh, L = c_lof[h], M = h - L * L - L, km = kmax_of(lam, L);
      const int ma = mamb / nb, mb = mamb - ma * nb;
      const int e0 = lmk_first(lam, L) + (M + L) * (km + 1);
      double Y[kC2K + 1];
#pragma unroll
      for (int k = 0; k <= kC2K; ++k) {
        double y = 0.0;
        if (k <= km)
          for (int t = gt_ptr[e0 + k]; t < gt_ptr[e0 + k + 1]; ++t) {
            const GTerm gtm = gt_terms[t];
            const int i1 = gtm.ridx / ws, i2 = gtm.ridx - i1 * ws;
            y = fma(gtm.coef * EA[ma * nha + i1], EB[mb * nhb + i2], y);
          }
        Y[k] = y;
      }
      double scale = pref;
      for (int k = 0; k < L; ++k) scale *= 0.5 * ip;
#pragma unroll
      for (int n = 0; n <= kC2K; ++n) {
        if (n > km) break;
        const double* en = eps + (size_t)L * (kC2K + 1) * (kC2K + 1) + n;
        double v = 0.0, pw = 1.0;
        for (int k = 0; k < 2 * n; ++k) pw *= ip;  // p^{-(k+n)} at k = n
#pragma unroll
        for (int k = 0; k <= kC2K; ++k) {
          if (k < n || k > km) continue;
          v = fma(en[k * (kC2K + 1)] * pw, Y[k], v);
          pw *= ip;
        }
        out[mamb * nr + e0 + n] = scale * v;
      }
    }
  }
}

size_t eri_dist_smem(int la, int lb) {
  return sizeof(double) * ((size_t)n_harm(la) + (2 * la + 1) * n_harm(la) + (2 * lb + 1) * n_harm(lb) + 8);
}

// Work item of k_eri_part: one bra primitive pair pp1 (of the bra class, in [pp_lo, pp_hi)), one slice of
// its bra entries (nslice slices of equal height) and one ket shell pair q2 (of the ket class, in
// [q2_lo, q2_hi)); for the same class only q2 <= q1 is needed.  The item computes the slice's rows of
// X = sum over the ket primitive pairs of I D_cd^T (I: the interaction matrix of step 3, built in tiles of
// kEriPartTile columns over (ket primitive pair, ket entry)) and writes its share of the block,
// D_ab[:, slice] X[slice, :], to part[(((pp1 - pp_lo) nslice + slice) n2w + q2 - q2_lo) nab ncd].
// Ket primitive pairs are taken `chunk` at a time: one thread per primitive pair for P - Q, its Boys values
// and the tables g^{(N)}(u), u^j; one thread per (primitive pair, column m) for the solid harmonics
// S_LM(P - Q); then the radial factors Z of all of them; then the tiles, contracted into X with 2 x 2
// register tiles (rows r, r + nxr and columns c, c + nxc).
constexpr int kEriPartTile = 32;
constexpr int kEriTileStride = kEriPartTile + 1;  // odd row stride: rows read together fall in distinct banks
constexpr size_t kEriSmemTarget = 56 * 1024;  // shared memory of a k_eri_part block (four per SM)

__global__ void __launch_bounds__(256) k_eri_part(
    int la, int lb, int lc, int ld, int64_t pp_lo, int64_t pp_hi, int base1, int q2_lo, int q2_hi, int same,
    int chunk, int nslice, const int* __restrict__ pp_pair, const int* __restrict__ pp_ij, const int* __restrict__ pair_a,
    const int* __restrict__ pair_b, const int64_t* __restrict__ pair_ppoff, int64_t pp_base1, int64_t pp_base2,
    int base2, const double* __restrict__ shell_xyz, const int* __restrict__ shell_poff,
    const int* __restrict__ shell_nprim, const double* __restrict__ prim_exp, const double* __restrict__ dist1,
    const double* __restrict__ dist2, const double* __restrict__ boys_tab, const int* __restrict__ rmap1,
    const int* __restrict__ rmap2, const int* __restrict__ rmapt, const int* __restrict__ c2_ptr,
    const int* __restrict__ c2_cbase, const GTerm* __restrict__ c2_terms, const double* __restrict__ c2_a,
    double* __restrict__ part) {
  extern __shared__ double smem[];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lam1 = la + lb, lam2 = lc + ld, lt = lam1 + lam2;
  const int nr1f = n_r(lam1), nr2 = n_r(lam2), nrt = n_r(lt), nht = n_harm(lt);
  const int nab = (2 * la + 1) * (2 * lb + 1), ncd = (2 * lc + 1) * (2 * ld + 1);
  const int n2w = q2_hi - q2_lo, rows = (nr1f + nslice - 1) / nslice;
  double* X = smem;                            // [rows][ncd]
  double* It = X + (size_t)rows * ncd;         // [rows][kEriTileStride]
  double* Dt = It + rows * kEriTileStride;     // [ncd][kEriTileStride] ket distributions of the tile
  double* S = Dt + ncd * kEriTileStride;       // [chunk][nht]
  double* F = S + (size_t)chunk * nht;         // [chunk][lt + 1]
  double* Z = F + (size_t)chunk * (lt + 1);    // [chunk][nrt]
  double* G = Z + (size_t)chunk * nrt;         // [chunk][lt + 1]: g^{(N)}(u) = cpq (-rho)^N F_N(rho u)
  double* U = G + (size_t)chunk * (lt + 1);    // [chunk][lt / 2 + 1]: u^j
  double* Rv = U + (size_t)chunk * (lt / 2 + 1);  // [chunk][3]: P - Q
  int* kap1 = (int*)(Rv + 3 * (size_t)chunk);    // bra entries: h | n << 12 | L << 20
  int* kap2 = kap1 + nr1f;                     // ket entries
  int* zoff = kap2 + nr2;                      // [lt + 1]
  for (int e = tid; e < nr1f; e += nth) {
    const int r = rmap1[e], h = r & 0xfff;
    kap1[e] = h | ((r >> 24) << 12) | (l_of_index(h) << 20);
  }
  for (int e = tid; e < nr2; e += nth) {
    const int r = rmap2[e], h = r & 0xfff;
    kap2[e] = h | ((r >> 24) << 12) | (l_of_index(h) << 20);
  }
  if (tid <= lt) zoff[tid] = lmk_first(lt, tid);
  const int64_t nitems = (pp_hi - pp_lo) * nslice * n2w;
  for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int64_t row = it / n2w, pp1 = pp_lo + row / nslice;
    const int slice = (int)(row - (row / nslice) * nslice), q2 = q2_lo + (int)(it - row * n2w);
    const int r_lo = slice * rows, nr1 = min(rows, nr1f - r_lo);  // bra entries r_lo .. r_lo + nr1
    // 2 x 2 register tiles of X: rows (r, r + nxr), columns (c, c + nxc), consecutive threads on consecutive c
    const int nxr = (nr1 + 1) >> 1, nxc = (ncd + 1) >> 1;
    const int pr1 = pp_pair[pp1];
    if (same && q2 > pr1 - base1) continue;  // uniform over the block
    const int ij = pp_ij[pp1], a = pair_a[pr1], b = pair_b[pr1];
    const double al = prim_exp[shell_poff[a] + (ij >> 8)], be = prim_exp[shell_poff[b] + (ij & 255)], p = al + be;
    const double ip = 1.0 / p;
    double P[3];
    for (int x = 0; x < 3; ++x) P[x] = (al * shell_xyz[3 * a + x] + be * shell_xyz[3 * b + x]) * ip;
    const int pr2 = base2 + q2, c = pair_a[pr2], d = pair_b[pr2], npd = shell_nprim[d];
    const int npp2 = shell_nprim[c] * npd;
    const double* d2p = dist2 + (pair_ppoff[pr2] - pp_base2) * (int64_t)ncd * nr2;
    __syncthreads();  // the previous item is done with X and the tables
    for (int x = tid; x < nr1 * ncd; x += nth) X[x] = 0.0;
    for (int k0 = 0; k0 < npp2; k0 += chunk) {
      const int nck = min(chunk, npp2 - k0);
      __syncthreads();  // S, F, Z, G of the previous chunk are consumed
      // one thread per ket primitive pair: P - Q, the Boys values, g^{(N)}(u) and u^j
      for (int w = tid; w < nck; w += nth) {
        const int i2 = k0 + w, ic = shell_poff[c] + i2 / npd, id = shell_poff[d] + i2 % npd;
        const double ga = prim_exp[ic], de = prim_exp[id], q = ga + de, iq = 1.0 / q;
        double R[3];
        for (int x = 0; x < 3; ++x) R[x] = P[x] - (ga * shell_xyz[3 * c + x] + de * shell_xyz[3 * d + x]) * iq;
        const double u = R[0] * R[0] + R[1] * R[1] + R[2] * R[2], rpq = 1.0 / (p + q), rho = p * q * rpq;
        for (int x = 0; x < 3; ++x) Rv[3 * w + x] = R[x];
        double* Fw = F + (size_t)w * (lt + 1);
        boys_eval(lt, rho * u, Fw, 1, boys_tab, c_boys);
        // g^{(N)}(u) = 2 pi^{5/2} / (p q sqrt(p + q)) (-rho)^N F_N(rho u), and u^j
        double gN = 2.0 * 5.5683279968317078453 * 3.1415926535897932385 * ip * iq * sqrt(rpq);
        double* Gw = G + (size_t)w * (lt + 1);
        for (int n = 0; n <= lt; ++n) {
          Gw[n] = gN * Fw[n];
          gN *= -rho;
        }
        double* Uw = U + (size_t)w * (lt / 2 + 1);
        double uj = 1.0;
        for (int j = 0; j <= lt / 2; ++j) {
          Uw[j] = uj;
          uj *= u;
        }
      }
      __syncthreads();
      // one thread per (ket primitive pair, harmonic column m) for S_LM(P - Q)
      for (int x = tid; x < nck * (2 * lt + 1); x += nth) {
        const int w = x / (2 * lt + 1), col = x - w * (2 * lt + 1);
        solid_harmonics_columns(lt, Rv[3 * w], Rv[3 * w + 1], Rv[3 * w + 2], S + (size_t)w * nht, col, 2 * lt + 1);
      }
      __syncthreads();
      for (int x = tid; x < nck * nrt; x += nth) {
        const int w = x / nrt, e = x - w * nrt;
        const int r = rmapt[e], h = r & 0xfff, K = r >> 24, L = l_of_index(h);
        const double* Gw = G + (size_t)w * (lt + 1) + L + K;
        const double* Uw = U + (size_t)w * (lt / 2 + 1);
        const double* aK = c2_a + ((size_t)L * (kC2K + 1) + K) * (kC2K + 1);
        double rad = 0.0;
        for (int j = 0; j <= K; ++j) rad = fma(aK[j] * Uw[j], Gw[j], rad);
        // 2^L S_LM(R) rad, the power of two exact
        Z[x] = (S[(size_t)w * nht + h] * rad) * __longlong_as_double((long long)(1023 + L) << 52);
      }
      __syncthreads();
      const int ncol = nck * nr2;  // columns (ket primitive pair, ket entry) of this chunk
      for (int t0 = 0; t0 < ncol; t0 += kEriPartTile) {
        const int tw = min(kEriPartTile, ncol - t0);
        for (int x = tid; x < nr1 * tw; x += nth) {
          const int e1 = x / tw, jj = x - e1 * tw, col = t0 + jj, w = col / nr2, e2 = col - w * nr2;
          const int k1 = kap1[r_lo + e1], k2 = kap2[e2];
          const int h1 = k1 & 0xfff, n1e = (k1 >> 12) & 0xff, L1 = k1 >> 20;
          const int h2 = k2 & 0xfff, n2e = (k2 >> 12) & 0xff, L2 = k2 >> 20;
          const int M1 = h1 - L1 * L1 - L1, M2 = h2 - L2 * L2 - L2;
          const int* lst = L1 >= L2 ? c2_ptr + c2_cbase[L1 * (L1 + 1) / 2 + L2] + (M1 + L1) * (2 * L2 + 1) + M2 + L2
                                    : c2_ptr + c2_cbase[L2 * (L2 + 1) / 2 + L1] + (M2 + L2) * (2 * L1 + 1) + M1 + L1;
          const double* Zw = Z + (size_t)w * nrt;
          double v = 0.0;
          for (int t = lst[0]; t < lst[1]; ++t) {
            const GTerm g = c2_terms[t];
            const int L = g.pad, K = (L1 + L2 - L) / 2 + n1e + n2e;
            v = fma(g.coef, Zw[zoff[L] + (g.ridx - L * L) * (kmax_of(lt, L) + 1) + K], v);
          }
          It[e1 * kEriTileStride + jj] = (L2 & 1) ? -v : v;
        }
        for (int x = tid; x < ncd * tw; x += nth) {
          const int cd = x / tw, jj = x - cd * tw, col = t0 + jj, w = col / nr2, e2 = col - w * nr2;
          Dt[cd * kEriTileStride + jj] = d2p[((int64_t)(k0 + w) * ncd + cd) * nr2 + e2];
        }
        __syncthreads();
        for (int x = tid; x < nxr * nxc; x += nth) {
          const int r0 = x / nxc, c0 = x - r0 * nxc, r1 = r0 + nxr, c1 = c0 + nxc;
          const bool r1ok = r1 < nr1, c1ok = c1 < ncd;
          const double* i0 = It + r0 * kEriTileStride;
          const double* i1 = It + (r1ok ? r1 : r0) * kEriTileStride;
          const double* j0 = Dt + c0 * kEriTileStride;
          const double* j1 = Dt + (c1ok ? c1 : c0) * kEriTileStride;
          double s00 = 0.0, s01 = 0.0, s10 = 0.0, s11 = 0.0;
          for (int jj = 0; jj < tw; ++jj) {
            const double x0 = i0[jj], x1 = i1[jj], y0 = j0[jj], y1 = j1[jj];
            s00 = fma(x0, y0, s00);
            s01 = fma(x0, y1, s01);
            s10 = fma(x1, y0, s10);
            s11 = fma(x1, y1, s11);
          }
          X[r0 * ncd + c0] += s00;
          if (c1ok) X[r0 * ncd + c1] += s01;
          if (r1ok) {
            X[r1 * ncd + c0] += s10;
            if (c1ok) X[r1 * ncd + c1] += s11;
          }
        }
        __syncthreads();
      }
    }
    // this bra primitive pair's and slice's share of the block: D_ab[:, slice] X
    const double* d1 = dist1 + (pp1 - pp_base1) * (int64_t)nab * nr1f + r_lo;
    double* o = part + (row * n2w + (q2 - q2_lo)) * (int64_t)nab * ncd;
    for (int x = tid; x < nab * ncd; x += nth) {
      const int ab = x / ncd, cd = x - ab * ncd;
      const double* dr = d1 + (int64_t)ab * nr1f;
      double s0 = 0.0;
      for (int e1 = 0; e1 < nr1; ++e1) s0 = fma(dr[e1], X[e1 * ncd + cd], s0);
      o[x] = s0;
    }
  }
}

size_t eri_part_smem(int la, int lb, int lc, int ld, int chunk, int nslice) {
  const int lam1 = la + lb, lam2 = lc + ld, lt = lam1 + lam2, nr1 = n_r(lam1), nr2 = n_r(lam2);
  const int rows = (nr1 + nslice - 1) / nslice;
  const size_t ncd = (size_t)(2 * lc + 1) * (2 * ld + 1);
  const size_t dbl = (size_t)rows * ncd + (size_t)rows * kEriTileStride + ncd * kEriTileStride +
                     (size_t)chunk * (n_harm(lt) + 2 * (lt + 1) + n_r(lt) + lt / 2 + 1 + 3);
  return sizeof(double) * dbl + sizeof(int) * (nr1 + nr2 + lt + 1);
}

// Sum of the shares (bra primitive pairs x slices) of each unique quartet (q1 in [q1_lo, q1_hi), q2 in [q2_lo, q2_hi),
// q2 <= q1 for the same class) in a fixed order, written to the eight permutations of every element.  Where
// a = b, c = d or the two pairs coincide the block holds several members of one permutation orbit; only the
// canonical member is written, so the output has the permutational symmetry exactly.  With a density
// (dens != nullptr) every distinct member (pq|rs) of the orbit adds (pq|rs) D_rs to Jm[p][q] and
// (pq|rs) D_qs to Km[p][r] (either may be nullptr); out may then be nullptr.
__global__ void __launch_bounds__(128) k_eri_reduce(int la, int lb, int lc, int ld, int q1_lo, int q1_hi,
                                                    int base1, int q2_lo, int q2_hi, int base2, int same,
                                                    int nslice, int64_t pp_lo, const int* __restrict__ pair_a,
                                                    const int* __restrict__ pair_b,
                                                    const int64_t* __restrict__ pair_ppoff,
                                                    const int* __restrict__ shell_nprim,
                                                    const int64_t* __restrict__ shell_foff,
                                                    const double* __restrict__ part, int64_t nbf,
                                                    double* __restrict__ out, const double* __restrict__ dens,
                                                    double* __restrict__ Jm, double* __restrict__ Km) {
  const int nb = 2 * lb + 1, nd = 2 * ld + 1, nab = (2 * la + 1) * nb, ncd = (2 * lc + 1) * nd;
  const int n2w = q2_hi - q2_lo;
  const int64_t nitems = (int64_t)(q1_hi - q1_lo) * n2w;
  for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int q1 = q1_lo + (int)(it / n2w), q2 = q2_lo + (int)(it - (it / n2w) * n2w);
    if (same && q2 > q1) continue;
    const int pr1 = base1 + q1, pr2 = base2 + q2;
    const int a = pair_a[pr1], b = pair_b[pr1], c = pair_a[pr2], d = pair_b[pr2];
    const int npp1 = shell_nprim[a] * shell_nprim[b] * nslice;  // shares: bra primitive pairs x slices
    const double* src = part + ((pair_ppoff[pr1] - pp_lo) * nslice * n2w + (q2 - q2_lo)) * (int64_t)nab * ncd;
    const int64_t stride = (int64_t)n2w * nab * ncd;
    const int64_t fa = shell_foff[a], fb = shell_foff[b], fc = shell_foff[c], fd = shell_foff[d];
    for (int x = threadIdx.x; x < nab * ncd; x += blockDim.x) {
      const int ab = x / ncd, cd = x - ab * ncd, ma = ab / nb, mb = ab - ma * nb, mc = cd / nd, md = cd - mc * nd;
      if ((a == b && ma < mb) || (c == d && mc < md) || (pr1 == pr2 && ab < cd)) continue;
      double v = 0.0;
      for (int i = 0; i < npp1; ++i) v += src[i * stride + x];
      const int64_t I = fa + ma, J = fb + mb, K = fc + mc, M = fd + md;
      if (out) {
        out[((I * nbf + J) * nbf + K) * nbf + M] = v;
        out[((J * nbf + I) * nbf + K) * nbf + M] = v;
        out[((I * nbf + J) * nbf + M) * nbf + K] = v;
        out[((J * nbf + I) * nbf + M) * nbf + K] = v;
        out[((K * nbf + M) * nbf + I) * nbf + J] = v;
        out[((M * nbf + K) * nbf + I) * nbf + J] = v;
        out[((K * nbf + M) * nbf + J) * nbf + I] = v;
        out[((M * nbf + K) * nbf + J) * nbf + I] = v;
      }
      if (dens) {
        const int64_t t[8][4] = {{I, J, K, M}, {J, I, K, M}, {I, J, M, K}, {J, I, M, K},
                                 {K, M, I, J}, {M, K, I, J}, {K, M, J, I}, {M, K, J, I}};
        for (int u = 0; u < 8; ++u) {
          bool dup = false;
          for (int w = 0; w < u; ++w)
            dup = dup || (t[w][0] == t[u][0] && t[w][1] == t[u][1] && t[w][2] == t[u][2] && t[w][3] == t[u][3]);
          if (dup) continue;
          if (Jm) atomicAdd(Jm + t[u][0] * nbf + t[u][1], v * dens[t[u][2] * nbf + t[u][3]]);
          if (Km) atomicAdd(Km + t[u][0] * nbf + t[u][2], v * dens[t[u][1] * nbf + t[u][3]]);
        }
      }
    }
  }
}

namespace {
// A rectangle of quartets (bra pairs [q1_lo, q1_hi) x ket pairs [q2_lo, q2_hi) of one class pair) whose
// shares fit one stream's scratch region.
struct EriRect {
  int q1_lo, q1_hi, q2_lo, q2_hi;
  int64_t pp_lo, pp_hi;
};

std::vector<EriRect> eri_rects(const ClassWork& w1, const ClassWork& w2, bool same, const int64_t* h_ppoff,
                               int64_t region, int nslice) {
  const int64_t blk = (int64_t)nslice * (2 * w1.la + 1) * (2 * w1.lb + 1) * (2 * w2.la + 1) * (2 * w2.lb + 1);
  const int64_t* pp = h_ppoff + w1.pair_base;  // bra pair q has primitive pairs pp[q] .. pp[q + 1]
  std::vector<EriRect> out;
  int q1 = 0;
  while (q1 < w1.npairs) {
    int q1e = q1 + 1;  // extend the run of bra pairs while the rectangle still fits
    while (q1e < w1.npairs && (pp[q1e + 1] - pp[q1]) * (same ? q1e + 1 : w2.npairs) * blk <= region) ++q1e;
    const int n2 = same ? q1e : w2.npairs;
    if ((pp[q1e] - pp[q1]) * n2 * blk <= region) {
      out.push_back(EriRect{q1, q1e, 0, n2, pp[q1], pp[q1e]});
    } else {  // a single bra pair against too many ket pairs: split the ket range
      const int step = (int)std::max<int64_t>(1, region / ((pp[q1 + 1] - pp[q1]) * blk));
      for (int q2 = 0; q2 < n2; q2 += step)
        out.push_back(EriRect{q1, q1 + 1, q2, std::min(n2, q2 + step), pp[q1], pp[q1 + 1]});
    }
    q1 = q1e;
  }
  return out;
}
}  // namespace

shgo_status launch_eri(const DeviceBasis& db, const DeviceTables& dt, const Tables& th,
                       const std::vector<ClassWork>& work, int64_t nbf, double* out, const double* dens,
                       double* Jm, double* Km, cudaStream_t stream, std::string* err) {
  const size_t nw = work.size();
  std::vector<int64_t> doff(nw + 1, 0);
  for (size_t c = 0; c < nw; ++c) {
    const ClassWork& w = work[c];
    doff[c + 1] = doff[c] + w.npp * (int64_t)(2 * w.la + 1) * (2 * w.lb + 1) * n_r(w.la + w.lb);
  }
  if (doff[nw] == 0) return SHGO_OK;
  ensure_max_dynamic_smem((const void*)k_eri_part);
  // class pairs, largest first, and each one's chunk of ket primitive pairs
  struct CP {
    size_t c1, c2;
    double cost;
    int chunk, nslice;
  };
  std::vector<CP> cps;
  int64_t need_max = 0, one_max = 1;
  for (size_t c1 = 0; c1 < nw; ++c1)
    for (size_t c2 = 0; c2 <= c1; ++c2) {
      const ClassWork &w1 = work[c1], &w2 = work[c2];
      if (w1.npairs == 0 || w2.npairs == 0) continue;
      const double nq = c1 == c2 ? 0.5 * w1.npp * (w1.npairs + 1) : (double)w1.npp * w2.npairs;
      const double ppq = nq * ((double)w2.npp / w2.npairs);
      const double cost = ppq * n_r(w1.la + w1.lb) * n_r(w2.la + w2.lb) * (2 * w2.la + 1) * (2 * w2.lb + 1);
      int maxnp = 1;
      for (int q = 0; q < w2.npairs; ++q)
        maxnp = (int)std::max<int64_t>(maxnp, db.h_ppoff[w2.pair_base + q + 1] - db.h_ppoff[w2.pair_base + q]);
      // shared memory within kEriSmemTarget (four blocks of 256 threads per SM): fewer ket primitive pairs per
      // chunk first, then the bra entries cut into slices
      int chunk = std::min(16, maxnp), nslice = 1;
      while (chunk > 1 && eri_part_smem(w1.la, w1.lb, w2.la, w2.lb, chunk, 1) > kEriSmemTarget) --chunk;
      while (nslice < n_r(w1.la + w1.lb) && eri_part_smem(w1.la, w1.lb, w2.la, w2.lb, chunk, nslice) > kEriSmemTarget)
        ++nslice;
      cps.push_back(CP{c1, c2, cost, chunk, nslice});
      const int64_t full = (c1 == c2 ? w1.npp * (int64_t)w1.npairs : w1.npp * (int64_t)w2.npairs) * nslice *
                           (2 * w1.la + 1) * (2 * w1.lb + 1) * (2 * w2.la + 1) * (2 * w2.lb + 1);
      need_max = std::max(need_max, full);
      int64_t np1 = 1;  // one bra pair against one ket pair must fit a region
      for (int q = 0; q < w1.npairs; ++q)
        np1 = std::max<int64_t>(np1, db.h_ppoff[w1.pair_base + q + 1] - db.h_ppoff[w1.pair_base + q]);
      one_max = std::max(one_max, np1 * nslice * (2 * w1.la + 1) * (2 * w1.lb + 1) * (2 * w2.la + 1) * (2 * w2.lb + 1));
    }
  std::stable_sort(cps.begin(), cps.end(), [](const CP& x, const CP& y) { return x.cost > y.cost; });
  cudaStream_t* pool = nullptr;
  cudaError_t e = stream_pool(&pool);
  if (e != cudaSuccess) {
    *err = std::string("stream pool: ") + cudaGetErrorString(e);
    return SHGO_ERR_CUDA;
  }
  const int ns = (int)std::min<size_t>(cps.size(), (size_t)kPoolStreams);
  // scratch region per stream: what the largest class pair needs, at most 8M doubles (64 MiB) unless
  // SHGO_ERI_SCRATCH_DOUBLES sets another cap; never less than one bra pair against one ket pair
  int64_t cap = (int64_t)1 << 23;
  if (const char* env = std::getenv("SHGO_ERI_SCRATCH_DOUBLES")) {
    const long long v = std::atoll(env);
    if (v > 0) cap = v;
  }
  const int64_t region = std::max<int64_t>(std::min<int64_t>(need_max, cap), one_max);
  double* dist = nullptr;
  e = cudaMallocAsync((void**)&dist, sizeof(double) * (size_t)(doff[nw] + (int64_t)ns * region), stream);
  if (e != cudaSuccess) {
    *err = std::string("distribution and scratch buffers: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SHGO_ERR_OOM : SHGO_ERR_CUDA;
  }
  double* scratch = dist + doff[nw];
  for (size_t c = 0; c < nw; ++c) {
    const ClassWork& w = work[c];
    if (w.npp == 0) continue;
    const int cid = class_id(w.la, w.lb);
    k_eri_dist<<<grid_cap(w.npp, 8), 128, eri_dist_smem(w.la, w.lb), stream>>>(
        w.la, w.lb, w.npp, w.pp_base, db.pp_pair, db.pp_ij, db.pair_a, db.pair_b, db.shell_xyz, db.shell_poff,
        db.prim_exp, db.prim_coef, dt.etab, dt.eoff, dt.gt_ptr + th.gt_base[cid], dt.gt_terms + th.gt_termbase[cid],
        dt.eri_eps, dist + doff[c]);
  }
  cudaEvent_t fork;
  e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaFreeAsync(dist, stream);
    *err = std::string("fork event: ") + cudaGetErrorString(e);
    return SHGO_ERR_CUDA;
  }
  bool joined = true;
  {
    cudaEventRecord(fork, stream);
    for (int i = 0; i < ns; ++i) cudaStreamWaitEvent(pool[i], fork, 0);
    for (size_t k = 0; k < cps.size(); ++k) {
      const ClassWork &w1 = work[cps[k].c1], &w2 = work[cps[k].c2];
      const bool same = cps[k].c1 == cps[k].c2;
      cudaStream_t s = pool[k % ns];
      double* reg = scratch + (int64_t)(k % ns) * region;
      const int lam1 = w1.la + w1.lb, lam2 = w2.la + w2.lb;
      const int nsl = cps[k].nslice;
      // threads per block: fewer for the small class pairs, so that more items are resident per SM
      const int xw = ((n_r(lam1) + nsl - 1) / nsl) * (2 * w2.la + 1) * (2 * w2.lb + 1);
      const int threads = xw >= 1024 ? 256 : (xw >= 256 ? 128 : 64);
      for (const EriRect& r : eri_rects(w1, w2, same, db.h_ppoff, region, nsl)) {
        const int64_t items = (r.pp_hi - r.pp_lo) * nsl * (int64_t)(r.q2_hi - r.q2_lo);
        // one block per item, so that blocks of the class pairs running on other streams share the SMs
        k_eri_part<<<(unsigned)std::min<int64_t>(items, 0x7fffffff), threads,
                     eri_part_smem(w1.la, w1.lb, w2.la, w2.lb, cps[k].chunk, nsl), s>>>(
            w1.la, w1.lb, w2.la, w2.lb, r.pp_lo, r.pp_hi, w1.pair_base, r.q2_lo, r.q2_hi, same ? 1 : 0,
            cps[k].chunk, nsl, db.pp_pair, db.pp_ij, db.pair_a, db.pair_b, db.pair_ppoff, w1.pp_base, w2.pp_base,
            w2.pair_base, db.shell_xyz, db.shell_poff, db.shell_nprim, db.prim_exp, dist + doff[cps[k].c1],
            dist + doff[cps[k].c2], dt.boys, dt.rmap + th.rmap_off[lam1], dt.rmap + th.rmap_off[lam2],
            dt.rmap + th.rmap_off[lam1 + lam2], dt.c2_ptr, dt.c2_cbase, dt.c2_terms, dt.c2_a, reg);
        const int64_t quartets = (int64_t)(r.q1_hi - r.q1_lo) * (r.q2_hi - r.q2_lo);
        k_eri_reduce<<<grid_cap(quartets, 16), 128, 0, s>>>(
            w1.la, w1.lb, w2.la, w2.lb, r.q1_lo, r.q1_hi, w1.pair_base, r.q2_lo, r.q2_hi, w2.pair_base,
            same ? 1 : 0, nsl, r.pp_lo, db.pair_a, db.pair_b, db.pair_ppoff, db.shell_nprim, db.shell_foff, reg, nbf, out,
            dens, Jm, Km);
      }
    }
    for (int i = 0; i < ns && joined; ++i) {
      cudaEvent_t join;
      if (cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess) {
        joined = false;
        break;
      }
      cudaEventRecord(join, pool[i]);
      cudaStreamWaitEvent(stream, join, 0);
      cudaEventDestroy(join);
    }
    cudaEventDestroy(fork);
  }
  shgo_status st = launch_error(err);
  if (!joined) {
    // `stream` does not wait for every pool stream: finish their work before the buffers are returned
    for (int i = 0; i < ns; ++i) cudaStreamSynchronize(pool[i]);
    if (st == SHGO_OK) {
      st = SHGO_ERR_CUDA;
      *err = "join event could not be created";
    }
  }
  cudaFreeAsync(dist, stream);
  return st;
}

shgo_status launch_overlap(const DeviceBasis& db, const DeviceTables& dt, const std::vector<ClassWork>& work,
                           const MolView& mv, double* out, cudaStream_t stream, std::string* err) {
  OverlapClasses cls{};
  int total = 0, lm_max = 0;
  for (const ClassWork& w : work) {
    if (w.npairs == 0) continue;
    if (cls.n == kOverlapMaxClasses) {
      *err = "overlap: more classes than one launch holds";
      return SHGO_ERR_INVALID_ARG;
    }
    cls.first[cls.n] = total;
    cls.pair_base[cls.n] = w.pair_base;
    cls.la[cls.n] = (unsigned char)w.la;
    cls.lb[cls.n] = (unsigned char)w.lb;
    ++cls.n;
    total += w.npairs;
    lm_max = std::max(lm_max, std::max(w.la, w.lb));
  }
  cls.first[cls.n] = total;
  if (total == 0) return SHGO_OK;
  const size_t sm = sizeof(double) * (size_t)kOverlapWarps * overlap_warp_doubles(lm_max);
  k_overlap<<<grid_cap((total + kOverlapWarps - 1) / kOverlapWarps, 12), 32 * kOverlapWarps, sm, stream>>>(
      cls, lm_max, db.pair_a, db.pair_b, db.pair_ppoff, db.pair_site, rot_block(db.rot_lmax), db.rotd,
      db.shell_nprim, db.shell_foff, dt.etab, dt.eoff, db.ppd, mv, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    *err = std::string("overlap launch: ") + cudaGetErrorString(e);
    return SHGO_ERR_CUDA;
  }
  return launch_error(err);
}

cudaError_t ensure_max_dynamic_smem(const void* func, int bytes) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, int>> done;  // (kernel, device) pairs already set
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  for (const auto& d : done)
    if (d.first == func && d.second == dev) return cudaSuccess;
  e = bytes > 0 ? cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
                : set_max_dynamic_smem(func);
  if (e == cudaSuccess) done.emplace_back(func, dev);
  return e;
}

int64_t launches_per_call(const std::vector<ClassWork>& work, int64_t nbf) {
  int64_t n = 0;
  for (const auto& w : work) n += (w.npp > 0 ? 1 : 0) + (w.npairs > 0 ? 1 : 0);
  return nbf == 0 ? 0 : n;
}

}  // namespace shgo
