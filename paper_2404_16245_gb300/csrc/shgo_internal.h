// Internal declarations shared by the host API, the table builder and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/shgo.h"

namespace shgo {

constexpr int kLmax = SHGO_LMAX;          // largest shell l
constexpr int kLamMax = 2 * kLmax;         // largest la + lb
constexpr int kLamDer = kLamMax + 1;       // largest Lambda of a coupling block (la + lb + 1: derivatives)
constexpr int kHarmMax = kLamDer;          // largest l of S_lm(C - P)

// Boys grid: T_g = g * h for g = 0..kBoysNg-1, h = 1/16, up to T = kBoysTsw.  Row g holds
// exp(-T_g) followed by F_n(T_g), n = 0..kBoysNmax.  A value is the Taylor expansion about the
// nearest T_g with kBoysK + 1 terms (|T - T_g| <= 1/32).
constexpr int kBoysK = 7;
constexpr double kBoysInvH = 16.0;
constexpr double kBoysTsw = 40.0;
constexpr int kBoysNg = 641;
constexpr int kBoysNmax = kLamMax + 1 + kBoysK;  // 24: F_{Lambda+1} may be needed by the expansion
constexpr int kBoysStride = kBoysNmax + 2;       // exp slot + orders 0..kBoysNmax

// Sizes of the per-primitive-pair layouts for Lambda = la + lb.
__host__ __device__ constexpr inline int n_harm(int lam) { return (lam + 1) * (lam + 1); }
__host__ __device__ constexpr inline int kmax_of(int lam, int L) { return (lam - L) >> 1; }
__host__ __device__ constexpr inline int n_beta(int lam) {
  int n = 0;
  for (int L = 0; L <= lam; ++L) n += kmax_of(lam, L) + 1;
  return n;
}
__host__ __device__ constexpr inline int n_r(int lam) { return (lam + 1) * (lam + 2) * (lam + 3) / 6; }
__host__ __device__ inline int harm_index(int l, int m) { return l * l + l + m; }

// Coefficients of the real solid-harmonic recursion (Racah normalisation):
//   S_{l+1,l+1}  = c_l (x S_{l,l} - y S_{l,-l})          (l >= 1; S_11 = x)
//   S_{l+1,-l-1} = c_l (y S_{l,l} + x S_{l,-l})          (l >= 1; S_1-1 = y)
//   S_{l+1,m}    = a_lm z S_{l,m} - b_lm r^2 S_{l-1,m}    (|m| <= l)
// with c_l = sqrt((2l+1)/(2l+2)), a_lm = (2l+1)/sqrt((l+m+1)(l-m+1)),
// b_lm = sqrt((l+m)(l-m)/((l+m+1)(l-m+1))).
struct HarmCoef {
  double a[(kHarmMax + 1) * (kHarmMax + 1)];
  double b[(kHarmMax + 1) * (kHarmMax + 1)];
  double c[kHarmMax + 1];
  // Unnormalised harmonics U_lm = S_lm / N_lm of a unit vector, whose recursion needs one constant:
  //   U_{l+1,m} = z U_lm + ng_lm U_{l-1,m} (|m| < l),  U_{l+1,+-l} = z U_{l,+-l},
  //   U_{l+1,l+1} = x U_ll - y U_{l,-l},  U_{l+1,-l-1} = y U_ll + x U_{l,-l}.
  double ng[(kHarmMax + 1) * (kHarmMax + 1)];  // -gamma_lm
  double n[(kHarmMax + 1) * (kHarmMax + 1)];   // N_lm
};
const HarmCoef& harm_coef_host();

// One term of a Gaunt program: 16 bytes, loaded with one vector load.
struct __align__(16) GTerm {
  double coef;
  int ridx;
  int pad;
};

// Host tables, built once per process (long double arithmetic, stored as double).
struct Tables {
  std::vector<double> boys;  // [kBoysNg][kBoysStride]
  // Real translation tensors: for la, entry (ma, l1, m1, nu) at etab[eoff[la] + ...] with the
  // index ((ma + la) * (la+1)^2 + l1^2 + l1 + m1) * (2 la + 1) + (nu + la - l1) ... packed densely
  // per (ma, l1 m1) over nu = -(la-l1)..(la-l1): see translation_index().
  std::vector<double> etab;
  std::vector<int> eoff;  // [kLmax + 2]
  // Gaunt programs per class (la >= lb): one row per W entry (l1 m1, l2 m2), rows sorted by
  // decreasing term count and cut into groups of 32 (one warp; the last group padded with empty
  // rows).  Row r has g_rowinfo[r] = W index (row-major with w_stride(lb) columns) | l1 << 16 |
  // l2 << 20, or -1 for padding.  Group g holds K_g = g_grp[2g + 1] terms per row, interleaved:
  // term j of the row in lane i is g_terms[g_grp[2g] + 32 j + i] (coefficient, R' index for
  // Lambda = la + lb), zero-coefficient terms filling rows shorter than K_g.
  std::vector<int> g_rowinfo;   // class c rows at g_rowbase[c] .., a multiple of 32 per class
  std::vector<int> g_grp;       // class c groups at 2 g_grpbase[c] ..; term offsets local to the class
  std::vector<GTerm> g_terms;
  std::vector<int> g_rowbase;   // [n classes]
  std::vector<int> g_grpbase;   // [n classes]
  std::vector<int> g_termbase;  // [n classes]
  std::vector<int> g_nnz;       // [n classes] nonzero coupling coefficients (without padding)
  // The same coupling, transposed (for the adjoint used by the electrostatic potential): per class,
  // for each R' entry e of Lambda = la + lb, terms gt_terms[gt_ptr[gt_base[c] + e] .. + 1] of
  // (coefficient, W index (row-major, w_stride(lb) columns), l1 (lb + 1) + l2).
  std::vector<int> gt_ptr;      // class c: gt_base[c] .. + n_r(Lambda) + 1 (term offsets local to the class)
  std::vector<GTerm> gt_terms;
  std::vector<int> gt_base;     // [n classes]
  std::vector<int> gt_termbase; // [n classes]
  // R layout per Lambda: packed (harm index | beta index << 12 | k << 24) for entry e.
  std::vector<int> rmap;
  std::vector<int> rmap_off;  // [kLamDer + 2]
  std::vector<double> rnorm;  // N_LM of entry e (HarmCoef::n), aligned with rmap
  // Real rotation matrices D^{l+1} from D^l (S_lm(R y) = sum_m' D^l[m][m'] S_lm'(y)): the
  // harmonic part of u_c S_{l,m'}(u) for a Cartesian component c is sum_M G(1 m(c), l m'; l+1 M)
  // S_{l+1,M}.  For l = 0..kLmax-1 and M = -(l+1)..l+1 the list rot_terms[rot_ptr[q] .. rot_ptr[q+1]]
  // (q = l^2 + 2l + M + l + 1 ... see rot_index()) holds (G, Cartesian component c, m').
  std::vector<int> rot_ptr;
  std::vector<GTerm> rot_terms;
  // Two-centre Coulomb integrals: per class (la >= lb) and block entry e = (ma + la)(2lb + 1) + mb + lb,
  // the product-rule terms S_la,ma S_lb,mb = sum_{L,M} G |v|^{2k} S_LM as c2_terms[c2_ptr[c2_base[c] + e] ..
  // c2_ptr[c2_base[c] + e + 1]) = (G, L^2 + L + M, L); and the coefficients of
  // (Delta_L)^k f^{(L)} = sum_j a_{k,j}(L) u^j f^{(L+k+j)}, Delta_L f = 4u f'' + (4L + 6) f', at
  // c2_a[(L (kC2K + 1) + k)(kC2K + 1) + j].
  std::vector<int> c2_ptr;
  std::vector<GTerm> c2_terms;
  std::vector<int> c2_base;  // [n classes]
  std::vector<double> c2_a;
  // Derivative integrals (shgo_deriv.cu).  For each Lambda <= kLamMax the coupling block of Lambda + 1
  // serves the class: d_map0 maps each entry (L, M, k) of the Lambda layout, d_mapm each entry of the
  // Lambda - 1 layout, to the same (L, M, k) of the Lambda + 1 layout (offsets d_map0_off[Lambda],
  // d_mapm_off[Lambda]).  With rho = G(1 m(c), L M; L+1 M') and g = G(1 m(c), L M; L-1 M') (m(x) = 1,
  // m(y) = -1, m(z) = 0), for entry e of the Lambda layout and Cartesian component c, kDerivSlots terms
  // each (zero-coefficient padding, R' indices in the Lambda + 1 layout):
  //   d_raise:  r^{2k} x_c S_LM = sum rho r^{2k} S_{L+1,M'} + sum g r^{2k+2} S_{L-1,M'}
  //   d_field:  the p-free part of d/dx_c [r^{2k} S_LM e^{-p r^2}] e^{+p r^2}
  //             = sum 2k rho r^{2k-2} S_{L+1,M'} + sum (2k + 2L + 1) g r^{2k} S_{L-1,M'}  (the rest is
  //             -2p times the d_raise terms)
  // at ((d_xoff[Lambda] + e) * 3 + c) * kDerivSlots.  d_low: for l = 1..kLmax, the lowering
  // d/dx_c S_lm = (2l + 1) sum_M' G(1 m(c), l m; l-1 M') S_{l-1,M'} as a dense [c][m][M'] array at
  // d_low_off[l].
  std::vector<int> d_map0, d_map0_off, d_mapm, d_mapm_off, d_xoff;
  std::vector<GTerm> d_raise, d_field;
  std::vector<double> d_low;
  std::vector<int> d_low_off;
  // Four-centre electron repulsion: r^{2k} S_LM(r) e^{-p r^2} = sum_{n<=k} eps_{k,n}(L) p^{-(k+n)}
  // Laplacian^n [S_LM(r) e^{-p r^2}], with eps_{k,n}(L) at eri_eps[(L (kC2K + 1) + k)(kC2K + 1) + n].
  std::vector<double> eri_eps;
};
constexpr int kC2K = kLamMax / 2;  // largest k of the two-centre radial factors
constexpr int kDerivSlots = 4;     // terms per entry and component of Tables::d_raise / d_field
const Tables& tables_host();

// Index of the (l -> l+1, M) list of the rotation recursion: lists for l = 0.. are stored one after
// the other, 2l + 3 of them per l.
__host__ __device__ inline int rot_index(int l, int M) { return l * (l + 2) + M + l + 1; }

inline int class_id(int la, int lb) { return la * (la + 1) / 2 + lb; }  // la >= lb

// Row stride of the coupling block W[(l1 m1)][(l2 m2)] in shared memory: (lb + 1)^2 rounded up to an
// odd count, so that a warp reading one column (consecutive rows) touches distinct banks.
__host__ __device__ inline int w_stride(int lb) { return ((lb + 1) * (lb + 1)) | 1; }
constexpr int kNumClasses = (kLmax + 1) * (kLmax + 2) / 2;

// Offset inside the la block of etab for (ma, l1, m1); nu runs over 2(la - l1) + 1 values.
int translation_offset(int la, int ma, int l1, int m1);

// The same offset on the device (the translation kernels' inner index).
__device__ __forceinline__ int translation_offset_dev(int la, int ma, int l1, int m1) {
  int per_ma = 0, below = 0;
  for (int k = 0; k <= la; ++k) {
    const int t = (2 * k + 1) * (2 * (la - k) + 1);
    per_ma += t;
    if (k < l1) below += t;
  }
  return (ma + la) * per_ma + below + (m1 + l1) * (2 * (la - l1) + 1);
}

double gaunt_real(int l1, int m1, int l2, int m2, int L, int M);
double translation_real(int la, int ma, int l1, int m1, int nu);
void boys_host(int nmax, double T, double* F);

// Device copies of the tables (one set per device, created on first use).
struct DeviceTables {
  double* boys = nullptr;
  double* etab = nullptr;
  int* eoff = nullptr;
  int* g_rowinfo = nullptr;
  int* g_grp = nullptr;
  int* gt_ptr = nullptr;
  GTerm* gt_terms = nullptr;
  GTerm* g_terms = nullptr;
  int* rmap = nullptr;
  double* rnorm = nullptr;
  int* rot_ptr = nullptr;
  GTerm* rot_terms = nullptr;
  int* c2_ptr = nullptr;
  GTerm* c2_terms = nullptr;
  double* c2_a = nullptr;
  double* eri_eps = nullptr;  // Tables::eri_eps
  int* c2_cbase = nullptr;    // Tables::c2_base (first c2_ptr entry of each class)
  float2* boys_ff = nullptr;  // boys as (hi, lo) FP32 pairs
  float2* exp_ff = nullptr;   // exp(-g/16) as (hi, lo) FP32 pairs
  float2* rnorm_ff = nullptr; // rnorm as (hi, lo) FP32 pairs
  int* f32_items = nullptr;   // FP32-bulk work items, aligned with rmap (rmap_off)
  // derivative tables (Tables::d_*)
  int* d_map0 = nullptr;
  int* d_mapm = nullptr;
  GTerm* d_raise = nullptr;
  GTerm* d_field = nullptr;
  double* d_low = nullptr;
};
shgo_status device_tables(int device, const DeviceTables** out, std::string* err);

// Molecules of a batch, seen from the kernels: pair -> molecule, and per molecule its first
// nucleus, nucleus count, offset of its V block in the output and its basis size (the leading
// dimension of that block).  pair_mol == nullptr means one molecule with the scalar fields.
struct MolView {
  const int* pair_mol = nullptr;
  const int64_t* c0 = nullptr;
  const int64_t* nc = nullptr;
  const int64_t* out_off = nullptr;
  const int64_t* ld = nullptr;
  int64_t ncenters = 0;
  int64_t nbf = 0;
  // Screening: when set, the nuclei of pair pr are centers[clist[clist_off[pr] .. clist_off[pr + 1])]
  const int* clist = nullptr;
  const int64_t* clist_off = nullptr;
  // Block-sparse output: when set, pair pr's block goes row-major to out + blk_off[pr] (nothing for -1)
  const int64_t* blk_off = nullptr;
};

__device__ __forceinline__ void mol_centers(const MolView& mv, int pr, int64_t& c_begin, int64_t& n) {
  if (mv.clist) {
    c_begin = mv.clist_off[pr];
    n = mv.clist_off[pr + 1] - c_begin;
  } else if (mv.pair_mol) {
    const int m = mv.pair_mol[pr];
    c_begin = mv.c0[m];
    n = mv.nc[m];
  } else {
    c_begin = 0;
    n = mv.ncenters;
  }
}

// Index into centers/charges of the k-th nucleus slot returned by mol_centers.
__device__ __forceinline__ int64_t mol_center_index(const MolView& mv, int64_t k) { return mv.clist ? mv.clist[k] : k; }

__device__ __forceinline__ void mol_output(const MolView& mv, int pr, int64_t& base, int64_t& ld) {
  if (mv.pair_mol) {
    const int m = mv.pair_mol[pr];
    base = mv.out_off[m];
    ld = mv.ld[m];
  } else {
    base = 0;
    ld = mv.nbf;
  }
}

// Work queue of one launch of the coupling or pair kernel.  A block takes its next primitive pair (or
// shell pair) with one atomic increment of qctr; items, when set, lists the launch's work in decreasing
// estimated cost (local indices), otherwise the work is taken in index order.  With qctr == nullptr the
// blocks stride over the work instead (uniform work, where a queue would only add the atomic's latency).  Time limit: t0 receives the start time of the launch's first
// block; before taking work a block that finds limit_ns passed since then (or a limit of 0) takes no
// more and sets *err = SHGO_ERR_TIMEOUT.  t0 == nullptr disables the limit.  No block waits on another.
struct WorkQueue {
  unsigned long long* qctr = nullptr;
  unsigned long long* t0 = nullptr;
  int* err = nullptr;
  const int* items = nullptr;
  unsigned long long limit_ns = ~0ull;
};

__device__ __forceinline__ unsigned long long wq_clock() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0 of a block: records (or reads) the launch's start time into *t0_block.
__device__ __forceinline__ void wq_begin(const WorkQueue& q, unsigned long long* t0_block) {
  if (threadIdx.x == 0 && q.t0) {
    const unsigned long long now = wq_clock();
    const unsigned long long old = atomicCAS(q.t0, 0ull, now);
    *t0_block = old == 0ull ? now : old;
  }
}

// Thread 0 of a block: index of its next piece of work among n, or -1 when the queue is empty or the
// time limit has passed.  `it` counts the block's iterations (used by the strided order).
__device__ __forceinline__ long long wq_take(const WorkQueue& q, long long n, long long it, unsigned long long t0) {
  if (q.t0 && q.limit_ns != ~0ull) {
    const unsigned long long now = wq_clock();
    if (q.limit_ns == 0ull || (now > t0 && now - t0 >= q.limit_ns)) {
      atomicExch(q.err, (int)SHGO_ERR_TIMEOUT);
      return -1;
    }
  }
  const long long k = q.qctr ? (long long)atomicAdd(q.qctr, 1ull) : (long long)blockIdx.x + it * (long long)gridDim.x;
  if (k >= n) return -1;
  return q.items ? (long long)q.items[k] : k;
}

// Runs body(w) for this block's share of the n work items of a launch.  Without a queue or a time limit
// the blocks stride over the work (body must start with a block-wide barrier before it reuses shared
// memory, and may return early only uniformly over the block).  Otherwise thread 0 takes the next item
// from the queue while the block runs the current one, a barrier closing each iteration.  body appears
// once, so both orders run the same compiled arithmetic.
template <typename Body>
__device__ __forceinline__ void wq_for_each(const WorkQueue& q, long long n, long long* s_next,
                                            unsigned long long* s_t0, Body&& body) {
  const bool queued = q.qctr != nullptr || q.t0 != nullptr;  // uniform over the grid
  long long w;
  if (queued) {
    wq_begin(q, s_t0);
    if (threadIdx.x == 0) s_next[0] = wq_take(q, n, 0, *s_t0);
    __syncthreads();
    w = s_next[0];
  } else {
    w = (long long)blockIdx.x < n ? (long long)blockIdx.x : -1;
  }
  for (long long it = 0; w >= 0; ++it) {
    if (queued && threadIdx.x == 0) s_next[(it + 1) & 1] = wq_take(q, n, it + 1, *s_t0);
    body(w);
    if (queued) {
      __syncthreads();  // every thread has read slot it & 1 before thread 0 refills it
      w = s_next[(it + 1) & 1];
    } else {
      w += gridDim.x;
      if (w >= n) w = -1;
    }
  }
}

// Control block of a basis (device): the error word (zero until a launch times out; cleared when the host
// reads it), then per class a queue slot for its coupling launch and one for its pair launch (counter,
// start time), cleared at the start of every call.
constexpr size_t kCtrlHead = 16;
constexpr size_t kCtrlSlot = 16;
inline size_t ctrl_bytes(size_t nclasses) { return kCtrlHead + 2 * kCtrlSlot * nclasses; }

// Kernel launchers (shgo_kernels.cu).
struct ClassWork {
  int la, lb;
  int npairs;      // shell pairs in this class
  int pair_base;   // first pair of the class in the pair arrays
  int64_t npp;     // primitive pairs of the class
  int64_t pp_base; // first primitive pair of the class in the primitive-pair arrays
};

// Rotations of the pair frames, from the basis alone, built once per basis by k_pair_rotations for
// every ordered pair of centre positions (A, B) that some shell pair (a on A, b on B) uses:
// |B - A| followed by the real rotation matrices D^l(Q^T), l = 0..lmax, row-major (2l+1)^2 each,
// D^l at offset 1 + rot_doff(l).  Shell pairs on the same two centres share one block.
__host__ __device__ inline int rot_doff(int l) { return l * (2 * l - 1) * (2 * l + 1) / 3; }
__host__ __device__ inline int64_t rot_block(int lmax) { return 1 + (int64_t)rot_doff(lmax + 1); }

// Ordered centre pairs of the shell pairs (pa[q], pb[q]): pair_site[q] = index of the pair of
// positions (xyz[pa[q]], xyz[pb[q]]) (exact coordinates), site_rep[i] = one shell pair using pair i,
// site_rot[9 i ..] = its frame Q (pair_frame).
void build_site_pairs(const double* shell_xyz, const std::vector<int>& pa, const std::vector<int>& pb,
                      std::vector<int>& pair_site, std::vector<int>& site_rep, std::vector<double>& site_rot);

// Per primitive pair, from the basis alone (Gaussian product, Eq. 5), built once per basis by
// k_pair_build: p = alpha + beta, 1/p, sqrt(p), K_AB, prefactor c~_i c~_j K_AB, beta/p, alpha/p and
// |P - A| (the offset of P along the pair axis).  kab == 0 marks a pair both kernels skip.
struct PPData {
  double p, rp, sp, kab, pref, ra, rb, shift;
};

struct DeviceBasis {
  // shells
  double* shell_xyz = nullptr;  // [n_shells][3]
  int* shell_l = nullptr;
  int* shell_nprim = nullptr;
  int* shell_poff = nullptr;    // first primitive
  int64_t* shell_foff = nullptr;  // first function
  double* prim_exp = nullptr;
  double* prim_coef = nullptr;  // normalised contraction coefficient
  // pairs, class-sorted; pair_a has l >= pair_b's l
  int* pair_a = nullptr;
  int* pair_b = nullptr;
  int64_t* pair_ppoff = nullptr;  // first primitive pair of the pair
  double* site_rot = nullptr;     // per ordered centre pair, 3x3 row-major Q with Q (B - A)/|B - A| = z (identity if A = B)
  // primitive pairs, class-sorted: owning pair, i (prim of a), j (prim of b)
  int* pp_pair = nullptr;
  int* pp_ij = nullptr;          // i << 8 | j
  int64_t* pp_roff = nullptr;    // offset of the pair's coupling block in rbuf
  PPData* ppd = nullptr;         // per primitive pair (class order)
  int* pair_site = nullptr;      // per pair: its ordered centre pair (a block of rotd)
  double* rotd = nullptr;        // per ordered centre pair: |B - A|, D^0 .. D^rot_lmax (rot_block doubles)
  int* site_rep = nullptr;       // per ordered centre pair: one shell pair on it
  int n_sites = 0;               // ordered centre pairs
  int rot_lmax = 0;              // largest shell l of the basis
  double* rbuf = nullptr;        // coupling buffer R'[L,M,k] per primitive pair
  int64_t rbuf_len = 0;
  int precision = SHGO_PREC_FP64;  // a shgo_precision value
  int prim_bound = 1;              // 1: primitive pairs below the elementwise bound are skipped
  int coupling_one_warp = 0;       // 1: the FP64 coupling kernel runs one warp per block at small Lambda
  // Bounded coupling buffer: region > 0 means rbuf holds one region of `region` doubles per pool
  // stream and each class runs in chunks of whole shell pairs that fit its stream's region;
  // h_ppoff (host, npairs + 1) gives the primitive-pair offsets used to cut the chunks.
  int64_t region = 0;
  const int64_t* h_ppoff = nullptr;
  // work queues (nullptr ctrl: strided blocks, no time limit): control block, items per class in
  // decreasing cost (local indices at the class's primitive-pair / pair offset; nullptr = index order),
  // and the time limit of each launch
  unsigned char* ctrl = nullptr;
  const int* cp_items = nullptr;
  const int* pr_items = nullptr;
  unsigned long long limit_ns = ~0ull;
};

// Coupling-buffer cap (doubles) above which a basis switches to per-stream regions (2 GiB).
constexpr int64_t kRbufCapDoubles = (int64_t)1 << 28;
constexpr int kPoolStreamsPublic = 16;

// Frame of a shell pair: rows (e1, e2, n) of a rotation Q with Q n = z for n = (B - A)/|B - A|,
// e1 perpendicular to n along the axis least aligned with it, e2 = n x e1 (det Q = +1).
// Q is the identity when A = B.
inline void pair_frame(const double* A, const double* B, double* Q) {
  const double d[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
  const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  for (int k = 0; k < 9; ++k) Q[k] = (k % 4 == 0) ? 1.0 : 0.0;
  if (!(r2 > 0.0)) return;
  const double r = std::sqrt(r2);
  const double n[3] = {d[0] / r, d[1] / r, d[2] / r};
  int ax = 0;
  for (int k = 1; k < 3; ++k)
    if (std::fabs(n[k]) < std::fabs(n[ax])) ax = k;
  double u[3] = {0, 0, 0};
  u[ax] = 1.0;
  double e1[3] = {u[1] * n[2] - u[2] * n[1], u[2] * n[0] - u[0] * n[2], u[0] * n[1] - u[1] * n[0]};
  const double l1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  for (double& v : e1) v /= l1;
  const double e2[3] = {n[1] * e1[2] - n[2] * e1[1], n[2] * e1[0] - n[0] * e1[2], n[0] * e1[1] - n[1] * e1[0]};
  for (int k = 0; k < 3; ++k) {
    Q[k] = e1[k];
    Q[3 + k] = e2[k];
    Q[6 + k] = n[k];
  }
}

// Raises `func`'s dynamic shared-memory limit on the current device to the most a block may take: the
// device's opt-in per-block limit less the kernel's static shared memory.
inline cudaError_t set_max_dynamic_smem(const void* func) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, func);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  return e;
}

// Raises `func`'s dynamic shared-memory limit to `bytes` (0: the most a block may take) on the current
// device, once per (kernel, device) and under a lock: the attribute belongs to one device, so a process
// on several devices sets it on each.
cudaError_t ensure_max_dynamic_smem(const void* func, int bytes = 0);

// blk_off (device, per pair) selects the block-sparse output of out_doubles values (see MolView::blk_off).
shgo_status launch_nuclear_attraction(const DeviceBasis& db, const DeviceTables& dt,
                                      const std::vector<ClassWork>& work, int64_t nbf, int64_t ncenters,
                                      const double* centers, const double* charges, double* out,
                                      cudaStream_t stream, std::string* err, cudaEvent_t* events = nullptr,
                                      bool concurrent = true, const int64_t* blk_off = nullptr,
                                      int64_t out_doubles = 0);
// Per shell pair: 1 when at least one of its primitive pairs is kept (pref != 0), else 0 (device, async).
shgo_status launch_pair_live(const DeviceBasis& db, int64_t npairs, int64_t npp, uint8_t* live, cudaStream_t stream,
                             std::string* err);
int64_t launches_per_call(const std::vector<ClassWork>& work, int64_t nbf);

// The same launches one class after another on `stream`, with the device time of each class's
// coupling and pair kernels in ms[2 c], ms[2 c + 1] (blocks until done).
shgo_status launch_class_timed(const DeviceBasis& db, const DeviceTables& dt, const std::vector<ClassWork>& work,
                               const MolView& mv, const double* centers, const double* charges, double* out,
                               cudaStream_t stream, double* ms, std::string* err);

// Electrostatic potential phi[k] = sum_ab D_ab <a|1/|r - points_k||b> of a single basis (D device,
// nbf x nbf row-major, symmetric); gbuf holds n_r(Lambda) doubles per primitive pair of every class.
// gradient = true: phi receives grad_x phi at each point, [npoints][3].
shgo_status launch_esp(const DeviceBasis& db, const DeviceTables& dt, const std::vector<ClassWork>& work,
                       int64_t nbf, const double* D, int64_t npoints, const double* points, double* phi, double* gbuf,
                       bool gradient, cudaStream_t stream, std::string* err);

// Contraction of the centre derivatives with a density (shgo_nuclear_attraction_gradient): P (device,
// nbf x nbf), the shells' lists of (pair, side) entries pr * 2 + side in pair order (side 1: the pair's ket
// shell), CSR over shells, and grad (device, [n_shells][3]).
struct DerivContraction {
  const double* P = nullptr;
  int n_shells = 0;
  const int64_t* shell_off = nullptr;
  const int64_t* shell_list = nullptr;
  double* grad = nullptr;
};

// Derivative integrals of a single basis, computed in FP64 (shgo_deriv.cu).  field = false: out[X] (X = x, y, z,
// nbf x nbf each) receives dV_ab/d(centre of a)_X; field = true: sum_C Z_C dV_ab/dC_X (symmetric).  With
// contract (field = false), no matrix is written: contract->grad receives the density-contracted gradient.
shgo_status launch_nuclear_deriv(const DeviceBasis& db, const DeviceTables& dt, const std::vector<ClassWork>& work,
                                 int64_t nbf, int64_t ncenters, const double* centers, const double* charges,
                                 double* out, bool field, cudaStream_t stream, std::string* err,
                                 const DerivContraction* contract = nullptr);
// The per-device pool of non-blocking streams on which the classes of one call run concurrently.
cudaError_t pool_streams(cudaStream_t** out, int* n);
// Blocks for n units of work, at most per_sm per SM.
int grid_cap_sm(int64_t n, int per_sm);

// Overlap blocks of every shell pair into out (one molecule or a batch, per mv).
shgo_status launch_overlap(const DeviceBasis& db, const DeviceTables& dt, const std::vector<ClassWork>& work,
                           const MolView& mv, double* out, cudaStream_t stream, std::string* err);

// Arguments of the FP64 coupling kernel for one class (shgo_coupling.cu).
struct CouplingArgs {
  int64_t npp = 0, pp_base = 0, rbase = 0;
  WorkQueue q;
  const int* pp_pair = nullptr;
  const int* pair_a = nullptr;
  const double* shell_xyz = nullptr;
  MolView mv;
  const double* centers = nullptr;
  const double* charges = nullptr;
  const double* boys_tab = nullptr;
  const int* rmap = nullptr;     // R layout of this Lambda
  const double* rnorm = nullptr; // N_LM per R entry of this Lambda
  const double* site_rot = nullptr;
  const int* pair_site = nullptr;
  const PPData* ppd = nullptr;
  double* rbuf = nullptr;
  // FP32-bulk kernel only: the Boys grid and exp(-g/16), g < 2048, as (hi, lo) FP32 pairs
  const float2* boys_ff = nullptr;
  const float2* exp_ff = nullptr;
  const int* items = nullptr;         // work items of this Lambda (coupling_f32_items)
  const float2* rnorm_ff = nullptr;   // rnorm of this Lambda as (hi, lo) pairs
  int one_warp_ok = 0;                // small Lambda may run smaller blocks (DeviceBasis::coupling_one_warp): one
                                      // warp (FP64) or two (FP32-bulk)
};
// Arguments of the electrostatic-potential kernel for one class (shgo_coupling.cu).
struct EspArgs {
  int64_t npp = 0, pp_base = 0;  // the class's primitive pairs
  const int* pp_pair = nullptr;
  const int* pair_a = nullptr;
  const double* shell_xyz = nullptr;
  const double* site_rot = nullptr;
  const int* pair_site = nullptr;
  const PPData* ppd = nullptr;
  const double* boys_tab = nullptr;
  const int* rmap = nullptr;     // R layout of this Lambda
  const double* gam = nullptr;   // adjoint blocks of the class, n_r(Lambda) per primitive pair
  int64_t npoints = 0;
  const double* points = nullptr;
  double* phi = nullptr;
  int nchunks = 0, nsplit = 0;   // blocks = nchunks x nsplit
};
cudaError_t launch_esp_fp64(int lam, const EspArgs& args, cudaStream_t stream);
// Gradient of the potential: args.phi receives 3 values per point; chunks of 16 points.
cudaError_t launch_esp_grad_fp64(int lam, const EspArgs& args, cudaStream_t stream);

// Launches the Lambda = lam instantiation with nucleus chunks of nch (16 or 32) on `grid` warps.
cudaError_t launch_coupling_fp64(int lam, int nch, const CouplingArgs& args, int grid, cudaStream_t stream);
size_t coupling_fp64_smem(int lam, int nch);
// Constants and launch attributes of the FP64 coupling kernels on the current device.
cudaError_t coupling_fp64_setup();

// Two-centre Coulomb integrals (a|b) of every class of `work` into out (layout of V, both triangles).
shgo_status launch_coulomb2c(const DeviceBasis& db, const DeviceTables& dt, const Tables& th,
                             const std::vector<ClassWork>& work, const MolView& mv, double* out, cudaStream_t stream,
                             std::string* err);

// Largest shell l of the four-centre electron-repulsion integrals (la + lb + lc + ld <= 16).
constexpr int kEriLmax = 4;

// Four-centre electron-repulsion integrals (ab|cd) of every quartet of pairs of `work` into out
// (nbf^4, row-major, all eight permutations written; out may be nullptr) and, with a density dens
// (nbf x nbf), accumulated into Jm[p][q] += (pq|rs) D_rs and Km[p][r] += (pq|rs) D_qs (zeroed by the caller;
// either may be nullptr).  Classes must have la <= kEriLmax.
shgo_status launch_eri(const DeviceBasis& db, const DeviceTables& dt, const Tables& th,
                       const std::vector<ClassWork>& work, int64_t nbf, double* out, const double* dens,
                       double* Jm, double* Km, cudaStream_t stream, std::string* err);

// FP32-bulk coupling (shgo_coupling_f32.cu): the Lambda = lam instantiation, compensated (pair
// arithmetic) or plain, on `grid` blocks of 64 threads; args.boys_ff and args.exp_ff must be set.
cudaError_t launch_coupling_f32(int lam, bool compensated, const CouplingArgs& args, int grid, cudaStream_t stream);
size_t coupling_f32_smem(int lam, bool compensated);
cudaError_t coupling_f32_setup();
// The tables those kernels read, as (hi, lo) FP32 pairs: the Boys grid, and exp(-g/16) for g < 2048.
std::vector<float2> boys_table_pairs(const std::vector<double>& boys);
std::vector<float2> exp_table_pairs();
std::vector<float2> pairs_of(const std::vector<double>& v);
// Work items of the FP32-bulk nucleus sums for every Lambda, aligned with Tables::rmap: per Lambda
// the first entry e of each pair (L, M, k), (L, M, k + 1), then each entry left over.
std::vector<int> coupling_f32_items(const std::vector<int>& rmap_off);

// Primitive pairs whose elementwise bound per unit of total nuclear charge is below this are skipped
// (k_pair_build); an element of V changes by at most kPrimSkip x sum |Z| per skipped pair.
constexpr double kPrimSkip = 1e-20;

// Per class of `work`: live primitive pairs, shell pairs with a live primitive pair, and (batches)
// the sum of the molecule's nucleus counts over live primitive pairs.  Blocking.
shgo_status live_counts(const DeviceBasis& db, const std::vector<ClassWork>& work, int64_t npairs, int64_t npp,
                        const int* pair_mol, const int64_t* mol_nc, std::vector<int64_t>& live_pp,
                        std::vector<int64_t>& live_pairs, std::vector<double>& live_cent, std::string* err);

// Fills db.ppd for the npp primitive pairs (asynchronous on `stream`).
shgo_status launch_pair_build(const DeviceBasis& db, int64_t npp, cudaStream_t stream, std::string* err);

// Fills db.rotd for every ordered centre pair (asynchronous on `stream`).
shgo_status launch_pair_rotations(const DeviceBasis& db, const DeviceTables& dt, cudaStream_t stream, std::string* err);

// Launch shape of one class: nucleus chunk of the coupling kernel (16 or 32) and threads per
// block of the pair kernel (32, 64 or 128); 0 = the default rule.
struct ClassTune {
  int nch = 0;
  int threads = 0;
};

// All molecules of a batch: one launch per class and kernel, classes concurrent on the pool.
shgo_status launch_batched(const DeviceBasis& db, const DeviceTables& dt, const std::vector<ClassWork>& work,
                           const MolView& mv, double nuclei_per_pair, const double* centers, const double* charges,
                           double* out, const std::vector<ClassTune>* tune, cudaStream_t stream, std::string* err);

// Times the candidate shapes of every class on the real work (synchronises the stream).
shgo_status autotune_batched(const DeviceBasis& db, const DeviceTables& dt, const std::vector<ClassWork>& work,
                             const MolView& mv, const double* centers, const double* charges, double* out,
                             std::vector<ClassTune>* tune, cudaStream_t stream, std::string* err);

struct ScreenBasis;
shgo_status launch_screen_features(const ScreenBasis& sb, const double* centers, const double* charges,
                                   const int* triples, int64_t n, float* X, cudaStream_t s);

// Device view of a basis for the screening kernels.
struct ScreenBasis {
  const double* shell_xyz = nullptr;
  const int* shell_l = nullptr;
  const int* shell_nprim = nullptr;
  const int* shell_poff = nullptr;
  const double* prim_exp = nullptr;
  const double* prim_coef = nullptr;
  const int* pair_a = nullptr;
  const int* pair_b = nullptr;
  const int* pair_mol = nullptr;       // batch: molecule of each pair
  const int64_t* mol_c0 = nullptr;
  const int64_t* mol_nc = nullptr;
  int64_t ncenters = 0;                // one molecule: nuclei of the call
  const int64_t* mask_off = nullptr;   // per pair, first triple of the pair in the mask
  const int64_t* clist_off = nullptr;  // per pair (+1), first kept nucleus in the list
};

}  // namespace shgo

struct shgo_mlp;
namespace shgo {
shgo_status launch_screen_pairs(const ScreenBasis& sb, int64_t npairs, const double* centers, const double* charges,
                                const shgo_mlp* mlp, float cut, int pass, uint8_t* mask, int64_t* counts,
                                int* clist, cudaStream_t s);
}  // namespace shgo
