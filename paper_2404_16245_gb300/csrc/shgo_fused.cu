// Fused shell-pair kernel: steps S2-S5 of the nuclear-attraction matrix for one shell pair in one block,
// the shell pairs taken from a device work queue.
//
// For a shell pair (a, b) of class (la, lb), Lambda = la + lb, the block loops over the primitive pairs
// (alpha_i, beta_j) of the pair (Eq. 5 product data built once per basis), and for each one
//   S2  sums over the nuclei C of the pair's molecule, in the pair frame (b - a along z), d = C - P:
//       R'[L,M,k] = 2 pi k! p^{-(k+1)} N_LM sum_C Z_C U_LM(d/|d|) |d|^L beta_{L,k}(T)/k!
//       (the coupled one-centre integral of Eq. 12, corrected as in the library's reading of it), with
//       chunks of 32 nuclei: lane i of all four warps owns nucleus i; warp 0 evaluates the Boys values
//       and radial sums, the warps split the unit-vector harmonic columns so their FP64 work balances;
//   S3  couples R' with the real Gaunt coefficients into W[l1 m1][l2 m2] (Supp. Eq. 4) and adds it,
//       scaled by c_i c_j K_AB (beta/p)^{la-l1} (alpha/p)^{lb-l2}, to the pair's W (the primitive
//       contraction of Eq. 11).
// Then, once per shell pair,
//   S4  translates W back to the two centres along the pair axis (Eq. 7 with the coefficients of
//       Eq. 8; in the pair frame only nu = 0 survives, so the translation is diagonal in m) and rotates
//       the block to the molecular frame with the real Wigner matrices of the pair's centre pair;
//   S5  writes the block and its transpose into V.
// R' and W never leave shared memory.  Every entry is computed with the operations of the two-kernel path
// (k_coupling_fp64 then k_pair_block) in the same order; the two agree to rounding (the compiler may fuse
// different products into multiply-adds in the two kernels).
//
// Work queue: one launch per Lambda (all classes la + lb = Lambda of a basis or of a whole batch); the
// launch's shell pairs are listed by decreasing estimated cost and each block takes the next one with
// one atomic increment.  No block ever waits on another.  A launch has a time limit: before taking a
// shell pair a block compares the time since the launch's first block started with the limit, and once
// it has passed it takes no more work and sets the launch's error word to SHGO_ERR_TIMEOUT, which the
// host reads back (shgo_basis_sync).
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "shgo_internal.h"
#include "shgo_math.h"
#include "shgo_point_tables.cuh"

namespace shgo {

namespace {

constexpr int kThreads = 128;  // four warps
constexpr int kWarps = kThreads / 32;
constexpr int kNch = 32;       // nuclei per chunk: one per lane
constexpr int kCS = kNch + 2;  // row stride of the nucleus tables

// First R' index, Gaunt row, group and term of each class in the device tables (class_id order).
__constant__ int k_cls_rowbase[kNumClasses];
__constant__ int k_cls_grpbase[kNumClasses];
__constant__ int k_cls_termbase[kNumClasses];

// Contiguous ranges of harmonic columns m for the four warps, [s[w], s[w + 1]): warp 0 also evaluates the
// Boys values and radial sums.  The split minimises the largest per-warp FP64 operation count: a column
// costs about 2 (Lambda - |m| + 1) operations and a warp's share of the diagonal chain 4 per level up to
// its largest |m|.
struct Split4 {
  int s[kWarps + 1];
};

__host__ __device__ constexpr int column_cost(int lam, int lo, int hi) {
  int c = 0, amax = -1;
  for (int m = lo; m < hi; ++m) {
    const int am = m < 0 ? -m : m;
    c += 2 * (lam - am + 1);
    amax = am > amax ? am : amax;
  }
  return c + (amax > 0 ? 4 * amax : 0);
}

__host__ __device__ constexpr Split4 column_split4(int lam) {
  const int radial = 5 * 7 + 1 + 3 * lam + 2 * lam + 1 + lam + 2 * (cn_beta(lam) - lam - 1);
  Split4 best{{-lam, -lam, -lam, -lam, lam + 1}};
  int best_load = 1 << 30;
  for (int s1 = -lam; s1 <= lam + 1; ++s1)
    for (int s2 = s1; s2 <= lam + 1; ++s2)
      for (int s3 = s2; s3 <= lam + 1; ++s3) {
        const int w0 = radial + column_cost(lam, -lam, s1), w1 = column_cost(lam, s1, s2),
                  w2 = column_cost(lam, s2, s3), w3 = column_cost(lam, s3, lam + 1);
        int mx = w0 > w1 ? w0 : w1;
        mx = mx > w2 ? mx : w2;
        mx = mx > w3 ? mx : w3;
        if (mx < best_load) {
          best_load = mx;
          best = Split4{{-lam, s1, s2, s3, lam + 1}};
        }
      }
  return best;
}

template <int LAM, int M0, int M1>
__device__ __forceinline__ void columns_if(double ex, double ey, double ez, double* col) {
  if constexpr (M0 <= M1) harmonic_columns<LAM, kCS, M0, M1>(ex, ey, ez, col);
}

// Tables of nucleus `lane` of the chunk (d = C - P in the pair frame, charge z) by the four warps.
template <int LAM>
__device__ __forceinline__ void point_tables4(int wid, int lane, double p, double dx, double dy, double dz, double z,
                                              const double* __restrict__ boys_tab, double* Stab, double* Btab) {
  constexpr Split4 S = column_split4(LAM);
  double s2, dn, ex, ey, ez;
  unit_offset(dx, dy, dz, s2, dn, ex, ey, ez);
  if (wid == 0) {
    radial_column<LAM, kCS>(p, s2, dn, z, boys_tab, Btab + lane);
    columns_if<LAM, S.s[0], S.s[1] - 1>(ex, ey, ez, Stab + lane);
  } else if (wid == 1) {
    columns_if<LAM, S.s[1], S.s[2] - 1>(ex, ey, ez, Stab + lane);
  } else if (wid == 2) {
    columns_if<LAM, S.s[2], S.s[3] - 1>(ex, ey, ez, Stab + lane);
  } else {
    columns_if<LAM, S.s[3], S.s[4] - 1>(ex, ey, ez, Stab + lane);
  }
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <int LAM>
__global__ void __launch_bounds__(kThreads) k_shell_pair_fp64(FusedArgs A) {
  constexpr int nS = cn_harm(LAM), nR = cn_r(LAM);
  extern __shared__ __align__(16) double smem[];
  double* U = smem;                       // nucleus tables S[h][c], B[b][c]; later W (one primitive pair) and
  double* Stab = U;                       // the epilogue's matrices
  double* Btab = U + nS * kCS;
  double* Wsep = U + A.u_doubles;         // W of contracted pairs (w_doubles; 0 when W lives in U)
  double* racc = Wsep + A.w_doubles;      // [nR] nucleus sums, then R'
  double* scl = racc + nR;                // [16] 2 pi k! p^{-(k+1)}
  double* fab = scl + 16;                 // [96] c_i c_j K_AB (beta/p)^{la-l1} (alpha/p)^{lb-l2}
  double* dpow = fab + 96;                // [16] |b - a|^k
  __shared__ int s_item;
  __shared__ unsigned long long s_t0;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) {
    const unsigned long long now = global_ns();
    const unsigned long long old = atomicCAS(A.t0, 0ull, now);
    s_t0 = old == 0ull ? now : old;
  }
  for (;;) {
    __syncthreads();  // every thread has read the previous item and finished with it
    if (tid == 0) {
      int item = -1;
      if (global_ns() - s_t0 >= A.limit_ns) {
        atomicExch(A.err, (int)SHGO_ERR_TIMEOUT);
      } else {
        const unsigned int q = atomicAdd(A.qctr, 1u);
        if (q < (unsigned int)A.nitems) item = A.items[q];
      }
      s_item = item;
    }
    __syncthreads();
    const int pr = s_item;
    if (pr < 0) break;
    const int a = A.pair_a[pr], b = A.pair_b[pr];
    const int la = A.shell_l[a], lb = LAM - la;
    const int cid = la * (la + 1) / 2 + lb;
    const int nWa = (la + 1) * (la + 1), nWb = (lb + 1) * (lb + 1), nW = nWa * nWb;
    const int ws = w_stride(lb), nWs = nWa * ws, nrp = (nW + 31) & ~31;
    const int na = 2 * la + 1, nb = 2 * lb + 1, nf = (la + 1) * (lb + 1);
    const int* __restrict__ rowinfo = A.g_rowinfo + k_cls_rowbase[cid];
    const int* __restrict__ grp = A.g_grp + 2 * k_cls_grpbase[cid];
    const GTerm* __restrict__ terms = A.g_terms + k_cls_termbase[cid];
    double* W = A.w_doubles > 0 ? Wsep : U;
    const double Ax = A.shell_xyz[3 * a], Ay = A.shell_xyz[3 * a + 1], Az = A.shell_xyz[3 * a + 2];
    const int site = A.pair_site[pr];
    double Q[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Q[k] = A.site_rot[9 * site + k];
    int64_t cbeg, ncen;
    mol_centers(A.mv, pr, cbeg, ncen);
    const int npp = A.shell_nprim[a] * A.shell_nprim[b];
    const int64_t q0 = A.pair_ppoff[pr];
    bool first = true;  // uniform over the block: no primitive pair added to W yet
    for (int ij = 0; ij < npp; ++ij) {
      const PPData pd = A.ppd[q0 + ij];
      // primitive pairs with a zero prefactor (K_AB of Eq. 5 underflowed, or the pair is below the
      // per-basis bound) are skipped; the test is uniform over the block
      if (pd.pref == 0.0) continue;
      __syncthreads();  // the previous primitive pair's coupling is done with racc and fab
      for (int e = tid; e < nR; e += kThreads) racc[e] = 0.0;
      if (tid <= LAM / 2) {
        double s = kTwoPiC * pd.rp;
        for (int k = 1; k <= tid; ++k) s *= double(k) * pd.rp;
        scl[tid] = s;
      }
      if (tid < nf) {
        const int l1 = tid / (lb + 1), l2 = tid % (lb + 1);
        double v = pd.pref;
        for (int k = 0; k < la - l1; ++k) v *= pd.ra;
        for (int k = 0; k < lb - l2; ++k) v *= pd.rb;
        fab[tid] = v;
      }
      // S2: nucleus chunks; C - P = (C - A) - (beta/p)(B - A) in the pair frame
      for (int64_t c0 = 0; c0 < ncen; c0 += kNch) {
        __syncthreads();  // the tables of the previous chunk are consumed
        {
          double dx = 0.0, dy = 0.0, dz = 0.0, z = 0.0;
          if (c0 + lane < ncen) {
            const int64_t c = mol_center_index(A.mv, cbeg + c0 + lane);
            pair_frame_offset(Q, Ax, Ay, Az, pd.shift, A.centers + 3 * c, dx, dy, dz);
            z = A.charges[c];
          }
          point_tables4<LAM>(wid, lane, pd.p, dx, dy, dz, z, A.boys_tab, Stab, Btab);
        }
        __syncthreads();
        // a partial last chunk sums only its occupied columns (rounded up to a pair; empty columns
        // carry Z = 0 and so add exact zeros)
        const int nv2 = ncen - c0 >= kNch ? kNch / 2 : (int)((ncen - c0 + 1) >> 1);
        for (int e = tid; e < nR; e += kThreads) {
          const int code = __ldg(A.rmap + e);
          const double2* S = reinterpret_cast<const double2*>(Stab + (code & 0xfff) * kCS);
          const double2* B = reinterpret_cast<const double2*>(Btab + ((code >> 12) & 0xfff) * kCS);
          double a0 = racc[e], a1 = 0.0;
          if (nv2 == kNch / 2) {
#pragma unroll
            for (int c = 0; c < kNch / 2; ++c) {
              const double2 s = S[c], bb = B[c];
              a0 = fma(s.x, bb.x, a0);
              a1 = fma(s.y, bb.y, a1);
            }
          } else {
#pragma unroll 4
            for (int c = 0; c < nv2; ++c) {
              const double2 s = S[c], bb = B[c];
              a0 = fma(s.x, bb.x, a0);
              a1 = fma(s.y, bb.y, a1);
            }
          }
          racc[e] = a0 + a1;
        }
      }
      // R' = scale x sums (each thread the entries it accumulated)
      for (int e = tid; e < nR; e += kThreads)
        racc[e] = racc[e] * (scl[(__ldg(A.rmap + e) >> 24) & 0xff] * __ldg(A.rnorm + e));
      __syncthreads();
      // S3: Gaunt coupling, rows of one warp form one group (equal trip counts, one coalesced load per term)
      for (int r = tid; r < nrp; r += kThreads) {
        const int info = rowinfo[r];
        const int gi = r >> 5, K = grp[2 * gi + 1];
        const GTerm* tp = terms + grp[2 * gi] + (r & 31);
        double acc0 = 0.0, acc1 = 0.0;
        int j = 0;
        for (; j + 1 < K; j += 2) {
          const GTerm g0 = tp[32 * j], g1 = tp[32 * j + 32];
          acc0 = fma(g0.coef, racc[g0.ridx], acc0);
          acc1 = fma(g1.coef, racc[g1.ridx], acc1);
        }
        if (j < K) {
          const GTerm g0 = tp[32 * j];
          acc0 = fma(g0.coef, racc[g0.ridx], acc0);
        }
        if (info >= 0) {
          const int e = info & 0xffff, l1 = (info >> 16) & 15, l2 = (info >> 20) & 15;
          W[e] = fma(fab[l1 * (lb + 1) + l2], acc0 + acc1, first ? 0.0 : W[e]);
        }
      }
      first = false;
    }
    __syncthreads();
    const int64_t fa0 = A.shell_foff[a], fb0 = A.shell_foff[b];
    int64_t obase, ld;
    mol_output(A.mv, pr, obase, ld);
    double* o = A.out + obase;
    if (first) {
      // every primitive pair skipped: the block is zero
      for (int e = tid; e < na * nb; e += kThreads) {
        const int ma = e / nb, mb = e % nb;
        o[(fa0 + ma) * ld + fb0 + mb] = 0.0;
        if (a != b) o[(fb0 + mb) * ld + fa0 + ma] = 0.0;
      }
      continue;
    }
    // S4: translation along the pair axis, t_A(l1, ma) = E^{la}(ma; l1 ma; 0) |b-a|^{la-l1} and
    // t_B(l2, mb) = E^{lb}(mb; l2 mb; 0) (-|b-a|)^{lb-l2}, then the rotation back, V = D^{la} V' (D^{lb})^T
    double* Dm = A.w_doubles > 0 ? U : U + nWs;  // D^{la}(Q^T), then D^{lb}(Q^T)
    double* tA = Dm + na * na + nb * nb;         // [l1][ma]
    double* tB = tA + (la + 1) * na;             // [l2][mb]
    double* Zb = tB + (lb + 1) * nb;             // [l1 m1][mb]
    double* Vp = Zb + nWa * nb;                  // [ma][mb] in the pair frame, later the final block
    double* Yb = Vp + na * nb;                   // [ma][mb]
    const double* rd = A.rotd + (int64_t)site * A.rot_per;
    const int lm = la > lb ? la : lb;
    if (tid == 0) {
      const double dist = rd[0];
      double v = 1.0;
      for (int k = 0; k <= lm; ++k) {
        dpow[k] = v;
        v *= dist;
      }
    }
    for (int e = tid; e < na * na; e += kThreads) Dm[e] = rd[1 + rot_doff(la) + e];
    if (la != lb)
      for (int e = tid; e < nb * nb; e += kThreads) Dm[na * na + e] = rd[1 + rot_doff(lb) + e];
    __syncthreads();
    for (int e = tid; e < (la + 1) * na; e += kThreads) {
      const int l1 = e / na, ma = e % na - la, lr = la - l1;
      double v = 0.0;
      if (l1 >= (ma < 0 ? -ma : ma)) v = A.etab[A.eoff[la] + translation_offset_dev(la, ma, l1, ma) + lr] * dpow[lr];
      tA[e] = v;
    }
    for (int e = tid; e < (lb + 1) * nb; e += kThreads) {
      const int l2 = e / nb, mb = e % nb - lb, lr = lb - l2;
      double v = 0.0;
      if (l2 >= (mb < 0 ? -mb : mb))
        v = A.etab[A.eoff[lb] + translation_offset_dev(lb, mb, l2, mb) + lr] * ((lr & 1) ? -dpow[lr] : dpow[lr]);
      tB[e] = v;
    }
    __syncthreads();
    // V' = t_A W t_B (diagonal in m), first over l2; threads ordered by |m| (m = 0, 1, -1, 2, -2, ...)
    // so the lanes of a warp run loops of nearly equal length
    for (int e = tid; e < nWa * nb; e += kThreads) {
      const int q = e / nWa, i1 = e - q * nWa;
      const int amb = (q + 1) >> 1, mb = (q & 1) ? amb : -amb;
      double s = 0.0;
      for (int l2 = amb; l2 <= lb; ++l2) s = fma(tB[l2 * nb + mb + lb], W[i1 * ws + l2 * l2 + l2 + mb], s);
      Zb[i1 * nb + mb + lb] = s;
    }
    __syncthreads();
    for (int e = tid; e < na * nb; e += kThreads) {
      const int q = e / nb, mb = e - q * nb;
      const int ama = (q + 1) >> 1, ma = (q & 1) ? ama : -ama;
      double s = 0.0;
      for (int l1 = ama; l1 <= la; ++l1) s = fma(tA[l1 * na + ma + la], Zb[(l1 * l1 + l1 + ma) * nb + mb], s);
      Vp[(ma + la) * nb + mb] = s;
    }
    __syncthreads();
    const double* Da = Dm;
    const double* Db = la != lb ? Dm + na * na : Dm;
    for (int e = tid; e < na * nb; e += kThreads) {
      const int ma = e / nb, mb = e % nb;
      double s = 0.0;
      for (int k = 0; k < nb; ++k) s = fma(Vp[ma * nb + k], Db[mb * nb + k], s);
      Yb[e] = s;
    }
    __syncthreads();
    for (int e = tid; e < na * nb; e += kThreads) {
      const int ma = e / nb, mb = e % nb;
      double s = 0.0;
      for (int k = 0; k < na; ++k) s = fma(Da[ma * na + k], Yb[k * nb + mb], s);
      Vp[e] = s;
    }
    __syncthreads();
    // S5: the block and its transpose; a diagonal shell block takes its upper triangle for both halves
    for (int e = tid; e < na * nb; e += kThreads) {
      const int ma = e / nb, mb = e % nb;
      const double v = (a == b && ma > mb) ? Vp[mb * nb + ma] : Vp[e];
      o[(fa0 + ma) * ld + fb0 + mb] = v;
      if (a != b) o[(fb0 + mb) * ld + fa0 + ma] = v;
    }
  }
}

using FusedKernel = void (*)(FusedArgs);

template <int... L>
constexpr FusedKernel fused_kernel_at(int lam, std::integer_sequence<int, L...>) {
  FusedKernel k = nullptr;
  ((lam == L ? (k = &k_shell_pair_fp64<L>, 0) : 0), ...);
  return k;
}

using Lams = std::make_integer_sequence<int, kLamMax + 1>;

// Blocks of one launch that fit an SM at once, per (device, Lambda, shared-memory bytes).
int resident_blocks(int device, int lam, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, size_t>, int> cache;
  const auto key = std::make_tuple(device, lam, smem);
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_kernel_at(lam, Lams{}), kThreads, smem) != cudaSuccess ||
      n < 1)
    n = 1;
  cache[key] = n;
  return n;
}

}  // namespace

size_t fused_smem(int lam, int64_t u_doubles, int64_t w_doubles) {
  return sizeof(double) * (size_t)(u_doubles + w_doubles + n_r(lam) + 16 + 96 + 16);
}

// Shared-memory regions of one launch over the classes (la, Lambda - la), la in [la_lo, la_hi]: the union
// region holds the nucleus tables or (when W lives there) W and the epilogue's matrices.
void fused_regions(int lam, int la_lo, int la_hi, bool w_alias, int64_t* u_doubles, int64_t* w_doubles) {
  int64_t u = (int64_t)(n_harm(lam) + n_beta(lam)) * kCS, w = 0;
  for (int la = la_lo; la <= la_hi; ++la) {
    const int lb = lam - la;
    const int64_t nWa = (la + 1) * (la + 1), na = 2 * la + 1, nb = 2 * lb + 1;
    const int64_t nWs = nWa * w_stride(lb);
    const int64_t epi = na * na + nb * nb + (la + 1) * na + (lb + 1) * nb + nWa * nb + 2 * na * nb;
    u = std::max(u, (w_alias ? nWs : 0) + epi);
    if (!w_alias) w = std::max(w, nWs);
  }
  *u_doubles = (u + 1) & ~(int64_t)1;  // keeps the regions after it 16-byte aligned
  *w_doubles = (w + 1) & ~(int64_t)1;
}

cudaError_t fused_setup() {
  const Tables& t = tables_host();
  if (t.g_rowbase.size() < (size_t)kNumClasses || t.g_grpbase.size() < (size_t)kNumClasses ||
      t.g_termbase.size() < (size_t)kNumClasses)
    return cudaErrorInvalidValue;
  int rb[kNumClasses], gb[kNumClasses], tb[kNumClasses];
  for (int c = 0; c < kNumClasses; ++c) {
    rb[c] = t.g_rowbase[c];
    gb[c] = t.g_grpbase[c];
    tb[c] = t.g_termbase[c];
  }
  cudaError_t e = cudaMemcpyToSymbol(k_harm, &harm_coef_host(), sizeof(HarmCoef));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(k_boys, &boys_const_host(), sizeof(BoysConst));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(k_cls_rowbase, rb, sizeof(rb));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(k_cls_grpbase, gb, sizeof(gb));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(k_cls_termbase, tb, sizeof(tb));
  // the largest dynamic shared memory a block may take: the device's opt-in limit less the kernel's own
  // static shared memory (the queue item and start time)
  int dev = 0, optin = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  for (int lam = 0; lam <= kLamMax && e == cudaSuccess; ++lam) {
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fused_kernel_at(lam, Lams{}));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fused_kernel_at(lam, Lams{}), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin - (int)fa.sharedSizeBytes);
  }
  return e;
}

cudaError_t launch_fused(int lam, const FusedArgs& args, size_t smem, cudaStream_t stream) {
  if (lam < 0 || lam > kLamMax) return cudaErrorInvalidValue;
  if (args.nitems <= 0) return cudaSuccess;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t resident = (int64_t)nsm * resident_blocks(dev, lam, smem);
  const int grid = (int)std::min<int64_t>(args.nitems, resident);
  fused_kernel_at(lam, Lams{})<<<grid, kThreads, smem, stream>>>(args);
  return cudaGetLastError();
}

}  // namespace shgo
