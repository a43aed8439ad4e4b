// C ABI of the library: argument checks, primitive normalisation (Eq. 1), class-sorted shell
// and primitive-pair lists, device buffers, and the host-side table views.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "shgo_internal.h"
#include "shgo_math.h"
#include "../../include/shgo_mlp.h"

using namespace shgo;

namespace {
thread_local std::string g_last_error;

shgo_status fail(shgo_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

// N(l, alpha)^-2 = int S_lm^2 e^{-2 alpha r^2} d^3r = pi^{3/2} (2l-1)!! / (2^l (2 alpha)^{l+3/2})
// Normalisation N(l, alpha) of a primitive, N^-2 = pi^{3/2} (2l-1)!! / (2^l (2 alpha)^{l+3/2}).
// Double precision: the host's long double may be a software binary128 type, far slower, and the
// factor needs no more than double accuracy.
double prim_norm(int l, double alpha) {
  double df = 1;
  for (int k = 2 * l - 1; k > 1; k -= 2) df *= k;
  const double n2 = 5.5683279968317078453 * df / (std::ldexp(1.0, l) * std::pow(2.0 * alpha, l + 1.5));
  return 1.0 / std::sqrt(n2);
}
}  // namespace

namespace shgo {
// Lets the allocation-free entry point (its own translation unit) report through shgo_last_error.
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace shgo

struct shgo_basis {
  int device = 0;
  int n_shells = 0;
  int64_t nbf = 0;
  int64_t npairs = 0;
  std::vector<ClassWork> work;
  DeviceBasis d;
  const DeviceTables* tabs = nullptr;
  std::vector<void*> allocations;
  // batches (shgo_batch_create): per molecule basis size, offset of its V block, nuclei
  bool batch = false;
  int n_mol = 1;
  std::vector<int64_t> mol_nbf, mol_out, mol_c0, mol_nc;
  int64_t out_size = 0, total_centers = 0;
  std::vector<double> class_pair_cent, class_pp_cent;  // per class: sum over pairs / primitive pairs of nuclei
  // per class, after the primitive-pair bound: live primitive pairs, shell pairs with one, and (batches)
  // the sum of nuclei over live primitive pairs
  // filled on first use by the statistics calls (class_model), not at creation
  std::vector<int64_t> live_pp, live_pairs;
  std::vector<double> live_cent;
  bool live_ready = false;
  std::mutex live_mu;
  int64_t ppcount = 0;
  int* pair_mol = nullptr;
  int64_t *mol_c0_d = nullptr, *mol_nc_d = nullptr, *mol_out_d = nullptr, *mol_ld_d = nullptr;
  std::vector<ClassTune> tune;
  bool tuned = false;
  std::vector<int64_t> h_ppoff;  // per pair first primitive pair, plus the total
  std::vector<int> h_pair_a, h_pair_b, h_pair_mol;
  // screening state (shgo_screen_build)
  uint8_t* scr_mask = nullptr;
  int64_t* scr_mask_off = nullptr;
  int64_t* scr_counts = nullptr;
  int64_t* scr_clist_off = nullptr;
  int* scr_clist = nullptr;
  int64_t scr_ntrip = 0, scr_ncenters = -1;
  cudaGraphExec_t graph = nullptr;
  const void* graph_key[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaStream_t capture_stream = nullptr;
  // device status of the last call: the control block's error word, copied after every call into
  // pinned host memory, and the event that marks that copy (shgo_basis_sync)
  int* h_err = nullptr;
  cudaEvent_t done_ev = nullptr;
  // single-basis calls: the previous call's key (graph_key) and time limit, for graph replay
  bool single_key_set = false;
  unsigned long long single_limit = ~0ull;
  // block-sparse output (SHGO_FLAG_BLOCK_SPARSE): per pair the offset of its block, or -1
  bool sparse = false;
  int64_t sparse_nblocks = 0, sparse_ndoubles = 0;
  std::vector<int64_t> h_blk_off;
  int64_t* d_blk_off = nullptr;
  // one shard of a basis split over devices (shgo_basis_create_shard)
  int shard_index = 0, shard_count = 1;
  // density-contracted gradient: per shell its (pair, side) entries, CSR, built on the first such call
  int64_t* d_shell_off = nullptr;
  int64_t* d_shell_list = nullptr;
  std::mutex grad_mu;
};

namespace {
// Packed host image of per-basis arrays (each at a 256-byte aligned offset), followed by device-only
// regions that kernels fill; the whole arena is one allocation and the image one copy.
class HostImage {
 public:
  template <typename T>
  size_t put(const T* src, size_t n) {
    const size_t off = align(bytes_.size());
    bytes_.resize(off + sizeof(T) * n);
    if (n) std::memcpy(bytes_.data() + off, src, sizeof(T) * n);
    return off;
  }
  template <typename T>
  size_t put(const std::vector<T>& v) {
    return put(v.data(), v.size());
  }
  // Device-only region after the image (call after every put).
  size_t reserve(size_t n) {
    const size_t off = align(std::max(total_, bytes_.size()));
    total_ = off + std::max<size_t>(n, 1);
    return off;
  }
  const unsigned char* data() const { return bytes_.data(); }
  size_t size() const { return bytes_.size(); }
  size_t total() const { return std::max<size_t>(std::max(total_, bytes_.size()), 256); }

 private:
  static size_t align(size_t x) { return (x + 255) & ~(size_t)255; }
  std::vector<unsigned char> bytes_;
  size_t total_ = 0;
};

// Per-device memory pool for basis arrays: stream-ordered allocations that keep their memory after a
// basis is freed (release threshold = unlimited), so creating and freeing bases repeatedly does not go
// back to the CUDA driver each time.  All pool operations are ordered on the legacy default stream and the
// basis build synchronises before use on other streams.
cudaError_t pool_alloc(int device, void** p, size_t bytes) {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    if (!pools[device]) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = device;
      cudaError_t e = cudaMemPoolCreate(&pools[device], &props);
      if (e != cudaSuccess) return e;
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pools[device], cudaMemPoolAttrReleaseThreshold, &keep);
    }
    pool = pools[device];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, 0);
}

// Pinned host words for the bases' device status, carved from page-locked slabs that live until the
// process exits (pinning memory per basis would cost more than building the basis).
std::mutex g_pin_mu;
std::vector<int*> g_pin_free;

cudaError_t pinned_status_word(int** p) {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  if (g_pin_free.empty()) {
    constexpr int kSlab = 1024;
    int* slab = nullptr;
    const cudaError_t e = cudaMallocHost((void**)&slab, sizeof(int) * kSlab);
    if (e != cudaSuccess) return e;
    for (int i = kSlab - 1; i >= 0; --i) g_pin_free.push_back(slab + i);
  }
  *p = g_pin_free.back();
  g_pin_free.pop_back();
  **p = 0;
  return cudaSuccess;
}

void release_status_word(int* p) {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.push_back(p);
}

void release(shgo_basis* b) {
  if (!b) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  if (b->graph) cudaGraphExecDestroy(b->graph);
  cudaFree(b->scr_mask);
  cudaFree(b->scr_mask_off);
  cudaFree(b->scr_counts);
  cudaFree(b->scr_clist_off);
  cudaFree(b->scr_clist);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  if (b->done_ev) cudaEventDestroy(b->done_ev);
  if (b->h_err) release_status_word(b->h_err);
  for (void* p : b->allocations) cudaFreeAsync(p, 0);
  cudaStreamSynchronize(0);
  cudaSetDevice(prev);
  delete b;
}
}  // namespace

extern "C" {

const char* shgo_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace {

// Shard of every shell pair when one basis's pairs are split over `count` shards (one per device): inside each
// class the pairs, in the library's pair order, are cut by their cumulative primitive-pair count (the cost of a
// pair of one class is its primitive-pair count times the nuclei, the same for all of them), pair q going to
// shard floor(count (start_q + npp_q / 2) / npp_class).  Every shard gets about 1/count of every class, so the
// shards' costs and their mixes of classes match.
void shard_of_pairs(const std::vector<ClassWork>& work, const std::vector<int64_t>& ppoff, int count,
                    std::vector<int>& shard) {
  shard.assign(ppoff.empty() ? 0 : ppoff.size() - 1, 0);
  for (const ClassWork& w : work) {
    const double tot = (double)w.npp;
    for (int q = w.pair_base; q < w.pair_base + w.npairs; ++q) {
      const double mid = (double)(ppoff[q] - w.pp_base) + 0.5 * (double)(ppoff[q + 1] - ppoff[q]);
      int k = tot > 0 ? (int)((double)count * mid / tot) : 0;
      shard[q] = std::min(std::max(k, 0), count - 1);
    }
  }
}

// Shells of n_mol molecules (consecutive runs of mol_nshells shells; n_mol = 0 means one molecule
// whose nuclei are given per call), validated, normalised and turned into class-sorted pair lists.
// shard_count > 1 (single bases only): keep the pairs of shard shard_index (shard_of_pairs).
shgo_status build_basis(int32_t n_shells, const int32_t* l, const int32_t* n_prim, const double* exponents,
                        const double* coefs, const double* shell_xyz, const shgo_options* opt, int32_t n_mol,
                        const int32_t* mol_nshells, const int64_t* mol_ncenters, shgo_basis** out,
                        int32_t shard_index = 0, int32_t shard_count = 1) {
  g_last_error.clear();
  if (!out) return fail(SHGO_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (shard_count < 1 || shard_index < 0 || shard_index >= shard_count)
    return fail(SHGO_ERR_INVALID_ARG, "shard index outside 0..shard_count-1");
  if (shard_count > 1 && n_mol > 0) return fail(SHGO_ERR_INVALID_ARG, "a batch is split by molecules, not shards");
  if (n_shells < 0) return fail(SHGO_ERR_INVALID_ARG, "n_shells < 0");
  if (n_shells > 0 && (!l || !n_prim || !exponents || !coefs || !shell_xyz))
    return fail(SHGO_ERR_INVALID_ARG, "NULL basis array");
  if (opt && opt->precision != SHGO_PREC_FP64 && opt->precision != SHGO_PREC_FP32_BULK &&
      opt->precision != SHGO_PREC_FP32_PLAIN)
    return fail(SHGO_ERR_INVALID_ARG, "unknown precision mode");
  const int32_t flags = opt ? opt->flags : 0;
  if (flags & ~(SHGO_FLAG_BLOCK_SPARSE | SHGO_FLAG_NO_PRIM_BOUND)) return fail(SHGO_ERR_INVALID_ARG, "unknown option flag");
  if ((flags & SHGO_FLAG_BLOCK_SPARSE) && n_mol > 0)
    return fail(SHGO_ERR_INVALID_ARG, "block-sparse output is for single bases, not batches");
  const bool batch = n_mol > 0;
  if (n_mol < 0) return fail(SHGO_ERR_INVALID_ARG, "n_mol < 0");
  if (batch) {
    if (!mol_nshells || !mol_ncenters) return fail(SHGO_ERR_INVALID_ARG, "NULL molecule arrays");
    int64_t tot = 0;
    for (int m = 0; m < n_mol; ++m) {
      if (mol_nshells[m] < 0 || mol_ncenters[m] < 0) return fail(SHGO_ERR_INVALID_ARG, "negative molecule size");
      tot += mol_nshells[m];
    }
    if (tot != n_shells) return fail(SHGO_ERR_INVALID_ARG, "molecule shell counts do not add up to n_shells");
  }
  int64_t nprim_total = 0;
  for (int s = 0; s < n_shells; ++s) {
    if (l[s] < 0) return fail(SHGO_ERR_INVALID_ARG, "negative l in shell " + std::to_string(s));
    if (l[s] > kLmax) return fail(SHGO_ERR_UNSUPPORTED_L, "l > 8 in shell " + std::to_string(s));
    if (n_prim[s] < 1 || n_prim[s] > 64)
      return fail(SHGO_ERR_INVALID_ARG, "n_prim outside 1..64 in shell " + std::to_string(s));
    for (int c = 0; c < 3; ++c)
      if (!std::isfinite(shell_xyz[3 * s + c])) return fail(SHGO_ERR_INVALID_ARG, "non-finite shell centre");
    nprim_total += n_prim[s];
  }
  for (int64_t i = 0; i < nprim_total; ++i) {
    if (!(exponents[i] > 0) || !std::isfinite(exponents[i]))
      return fail(SHGO_ERR_INVALID_ARG, "exponent must be finite and > 0");
    if (!std::isfinite(coefs[i])) return fail(SHGO_ERR_INVALID_ARG, "non-finite contraction coefficient");
  }
  int device = 0;
  if (opt && opt->device >= 0) {
    device = opt->device;
  } else if (cudaGetDevice(&device) != cudaSuccess) {
    return fail(SHGO_ERR_CUDA, "no CUDA device");
  }
  if (cudaSetDevice(device) != cudaSuccess) return fail(SHGO_ERR_CUDA, "cudaSetDevice failed");

  auto* b = new shgo_basis();
  b->device = device;
  b->n_shells = n_shells;
  b->d.precision = opt ? opt->precision : SHGO_PREC_FP64;
  b->d.prim_bound = (flags & SHGO_FLAG_NO_PRIM_BOUND) ? 0 : 1;
  b->d.coupling_one_warp = 1;
  b->sparse = (flags & SHGO_FLAG_BLOCK_SPARSE) != 0;
  b->batch = batch;
  const int nm = batch ? n_mol : 1;
  b->n_mol = nm;
  std::string err;

  // molecule of each shell
  std::vector<int> shell_mol(n_shells, 0), mol_s0(nm + 1, 0);
  if (batch) {
    for (int m = 0; m < nm; ++m) mol_s0[m + 1] = mol_s0[m] + mol_nshells[m];
    for (int m = 0; m < nm; ++m)
      for (int s = mol_s0[m]; s < mol_s0[m + 1]; ++s) shell_mol[s] = m;
  } else {
    mol_s0[1] = n_shells;
  }

  // primitive offsets, normalised coefficients (Eq. 1 normalisation, contracted renormalisation)
  std::vector<int> poff(n_shells + 1, 0);
  for (int s = 0; s < n_shells; ++s) poff[s + 1] = poff[s] + n_prim[s];
  std::vector<double> pexp(exponents, exponents + nprim_total), pcoef(nprim_total);
  for (int s = 0; s < n_shells; ++s) {
    const int ls = l[s];
    for (int i = 0; i < n_prim[s]; ++i) pcoef[poff[s] + i] = coefs[poff[s] + i] * prim_norm(ls, exponents[poff[s] + i]);
    // <phi|phi> = sum_ij d_i d_j (2 sqrt(a_i a_j)/(a_i + a_j))^{l+3/2} / (N_i N_j) with d = c N
    double self = 0;
    for (int i = 0; i < n_prim[s]; ++i)
      for (int j = 0; j < n_prim[s]; ++j) {
        const double ai = exponents[poff[s] + i], aj = exponents[poff[s] + j];
        const double ov = std::pow(2 * std::sqrt(ai * aj) / (ai + aj), ls + 1.5);
        self += coefs[poff[s] + i] * coefs[poff[s] + j] * ov;
      }
    if (!(self > 0)) {
      release(b);
      return fail(SHGO_ERR_NUMERIC, "contracted shell " + std::to_string(s) + " has zero norm");
    }
    const double scale = 1.0 / std::sqrt(self);
    for (int i = 0; i < n_prim[s]; ++i) pcoef[poff[s] + i] *= scale;
  }
  // function offsets inside each molecule's V block
  std::vector<int64_t> foff(n_shells + 1, 0);
  b->mol_nbf.assign(nm, 0);
  for (int s = 0; s < n_shells; ++s) {
    foff[s] = b->mol_nbf[shell_mol[s]];
    b->mol_nbf[shell_mol[s]] += 2 * l[s] + 1;
  }
  foff[n_shells] = 0;
  b->mol_out.assign(nm, 0);
  b->mol_c0.assign(nm, 0);
  b->mol_nc.assign(nm, 0);
  int64_t acc_out = 0, acc_c = 0;
  for (int m = 0; m < nm; ++m) {
    b->mol_out[m] = acc_out;
    acc_out += b->mol_nbf[m] * b->mol_nbf[m];
    b->mol_c0[m] = acc_c;
    b->mol_nc[m] = batch ? mol_ncenters[m] : 0;
    acc_c += b->mol_nc[m];
  }
  b->out_size = acc_out;
  b->total_centers = acc_c;
  b->nbf = batch ? 0 : b->mol_nbf[0];
  for (int m = 0; m < nm; ++m) b->nbf = batch ? b->nbf + b->mol_nbf[m] : b->nbf;

  // class-sorted pairs (la >= lb), molecule after molecule inside a class, and their primitive pairs
  std::vector<std::vector<std::vector<int>>> by_l(nm, std::vector<std::vector<int>>(kLmax + 1));
  for (int s = 0; s < n_shells; ++s) by_l[shell_mol[s]][l[s]].push_back(s);
  std::vector<int> pa, pb, pmol;
  std::vector<int64_t> ppoff;
  std::vector<int> pp_pair, pp_ij;
  int64_t ppcount = 0;
  {
    // sizes first, then the lists filled by index
    int64_t np_total = 0, npp_total = 0;
    for (int m = 0; m < nm; ++m)
      for (int la = 0; la <= kLmax; ++la)
        for (int lb = 0; lb <= la; ++lb) {
          const auto& A = by_l[m][la];
          const auto& B = by_l[m][lb];
          if (la == lb) {
            int64_t run = 0;
            for (const int x : A) {
              run += n_prim[x];
              npp_total += (int64_t)n_prim[x] * run;  // y <= x
            }
            np_total += (int64_t)A.size() * ((int64_t)A.size() + 1) / 2;
          } else {
            int64_t sa = 0, sb = 0;
            for (const int x : A) sa += n_prim[x];
            for (const int y : B) sb += n_prim[y];
            np_total += (int64_t)A.size() * (int64_t)B.size();
            npp_total += sa * sb;
          }
        }
    pa.resize(np_total);
    pb.resize(np_total);
    pmol.resize(np_total);
    ppoff.resize(np_total);
    pp_pair.resize(npp_total);
    pp_ij.resize(npp_total);
  }
  int64_t q = 0;
  for (int la = 0; la <= kLmax; ++la)
    for (int lb = 0; lb <= la; ++lb) {
      ClassWork w{la, lb, 0, (int)q, 0, ppcount};
      double pc = 0, ppc = 0;
      for (int m = 0; m < nm; ++m) {
        const auto& A = by_l[m][la];
        const auto& B = by_l[m][lb];
        const double nc = (double)b->mol_nc[m];
        for (size_t x = 0; x < A.size(); ++x) {
          const size_t ylim = (la == lb) ? x + 1 : B.size();
          const int sa = A[x], npa = n_prim[sa];
          for (size_t y = 0; y < ylim; ++y, ++q) {
            const int sb = B[y], npb = n_prim[sb];
            pa[q] = sa;
            pb[q] = sb;
            pmol[q] = m;
            ppoff[q] = ppcount;
            int* ppp = pp_pair.data() + ppcount;
            int* ppi = pp_ij.data() + ppcount;
            for (int i = 0; i < npa; ++i)
              for (int j = 0; j < npb; ++j) {
                *ppp++ = (int)q;
                *ppi++ = (i << 8) | j;
              }
            ppcount += (int64_t)npa * npb;
            ppc += nc * npa * npb;
          }
          pc += nc * (double)ylim;
          w.npairs += (int)ylim;
        }
      }
      w.npp = ppcount - w.pp_base;
      if (w.npairs > 0) {
        b->work.push_back(w);
        b->class_pair_cent.push_back(pc);
        b->class_pp_cent.push_back(ppc);
      }
    }
  if (shard_count > 1) {
    // keep this shard's pairs (and their primitive pairs), renumbered in the same order
    std::vector<int64_t> off_all(ppoff.begin(), ppoff.end());
    off_all.push_back(ppcount);
    std::vector<int> shard;
    shard_of_pairs(b->work, off_all, shard_count, shard);
    std::vector<int> pa2, pb2, pm2, ppp2, ppi2;
    std::vector<int64_t> ppoff2;
    std::vector<ClassWork> work2;
    std::vector<double> pc2, ppc2;
    for (size_t wi = 0; wi < b->work.size(); ++wi) {
      const ClassWork& w = b->work[wi];
      ClassWork v{w.la, w.lb, 0, (int)pa2.size(), 0, (int64_t)ppp2.size()};
      for (int q = w.pair_base; q < w.pair_base + w.npairs; ++q) {
        if (shard[q] != shard_index) continue;
        const int nq = (int)pa2.size();
        pa2.push_back(pa[q]);
        pb2.push_back(pb[q]);
        pm2.push_back(pmol[q]);
        ppoff2.push_back((int64_t)ppp2.size());
        for (int64_t x = off_all[q]; x < off_all[q + 1]; ++x) {
          ppp2.push_back(nq);
          ppi2.push_back(pp_ij[x]);
        }
        ++v.npairs;
      }
      v.npp = (int64_t)ppp2.size() - v.pp_base;
      if (v.npairs > 0) {
        work2.push_back(v);
        pc2.push_back(0.0);
        ppc2.push_back(0.0);
      }
    }
    pa.swap(pa2);
    pb.swap(pb2);
    pmol.swap(pm2);
    ppoff.swap(ppoff2);
    pp_pair.swap(ppp2);
    pp_ij.swap(ppi2);
    ppcount = (int64_t)pp_pair.size();
    b->work.swap(work2);
    b->class_pair_cent.swap(pc2);
    b->class_pp_cent.swap(ppc2);
    b->shard_index = shard_index;
    b->shard_count = shard_count;
  }
  b->npairs = (int64_t)pa.size();
  b->h_pair_a = pa;
  b->h_pair_b = pb;
  b->h_pair_mol = pmol;
  std::vector<int> pair_site, site_rep;
  std::vector<double> site_rot;
  build_site_pairs(shell_xyz, pa, pb, pair_site, site_rep, site_rot);
  b->d.n_sites = (int)site_rep.size();
  for (int s = 0; s < n_shells; ++s) b->d.rot_lmax = std::max(b->d.rot_lmax, (int)l[s]);
  const int64_t rotlen = (int64_t)site_rep.size() * rot_block(b->d.rot_lmax);
  int64_t rlen = 0, max_pair_r = 0;
  for (const auto& w : b->work) rlen += w.npp * n_r(w.la + w.lb);
  b->h_ppoff.assign(ppoff.begin(), ppoff.end());
  b->h_ppoff.push_back(ppcount);
  for (const auto& w : b->work)
    for (int q = w.pair_base; q < w.pair_base + w.npairs; ++q)
      max_pair_r = std::max(max_pair_r, (b->h_ppoff[q + 1] - b->h_ppoff[q]) * (int64_t)n_r(w.la + w.lb));
  int64_t cap = kRbufCapDoubles;
  if (const char* env = std::getenv("SHGO_RBUF_CAP_DOUBLES")) cap = std::max<int64_t>(1, std::atoll(env));
  if (rlen > cap) {
    // bounded buffer: one region per pool stream, classes processed in chunks of shell pairs
    b->d.region = std::max(cap / kPoolStreamsPublic, max_pair_r);
    rlen = b->d.region * kPoolStreamsPublic;
  }
  b->d.h_ppoff = b->h_ppoff.data();
  // Work-queue orders of a batch: inside each class, the primitive pairs and shell pairs of molecules with
  // more nuclei first (their cost per primitive pair grows with the nucleus count); a single molecule's
  // work is uniform per class and keeps index order.
  std::vector<int> cp_items, pr_items;
  if (batch) {
    std::vector<int> mol_order(nm);
    for (int m = 0; m < nm; ++m) mol_order[m] = m;
    std::stable_sort(mol_order.begin(), mol_order.end(),
                     [&](int x, int y) { return b->mol_nc[x] > b->mol_nc[y]; });
    std::vector<int> rank(nm);
    for (int k = 0; k < nm; ++k) rank[mol_order[k]] = k;
    cp_items.resize(ppcount);
    pr_items.resize(pa.size());
    for (const ClassWork& w : b->work) {
      // counting sort of the class's pairs by molecule rank (pairs of one molecule are contiguous)
      std::vector<int64_t> pair_start(nm + 1, 0), pp_start(nm + 1, 0);
      for (int q = w.pair_base; q < w.pair_base + w.npairs; ++q) {
        pair_start[rank[pmol[q]] + 1] += 1;
        pp_start[rank[pmol[q]] + 1] += b->h_ppoff[q + 1] - b->h_ppoff[q];
      }
      for (int k = 0; k < nm; ++k) {
        pair_start[k + 1] += pair_start[k];
        pp_start[k + 1] += pp_start[k];
      }
      for (int q = w.pair_base; q < w.pair_base + w.npairs; ++q) {
        const int r = rank[pmol[q]];
        pr_items[w.pair_base + pair_start[r]++] = q - w.pair_base;
        const int64_t p0 = b->h_ppoff[q], p1 = b->h_ppoff[q + 1];
        for (int64_t x = p0; x < p1; ++x) cp_items[w.pp_base + pp_start[r]++] = (int)(x - w.pp_base);
      }
    }
  }

  // one host image of every per-basis array, one device arena (image + device-built data), one copy
  std::vector<int> poffv(poff.begin(), poff.end() - 1);
  HostImage im;
  const size_t o_xyz = im.put(shell_xyz, 3 * (size_t)n_shells);
  const size_t o_l = im.put(l, (size_t)n_shells);
  const size_t o_np = im.put(n_prim, (size_t)n_shells);
  const size_t o_poff = im.put(poffv);
  const size_t o_foff = im.put(foff);
  const size_t o_exp = im.put(pexp);
  const size_t o_coef = im.put(pcoef);
  const size_t o_pa = im.put(pa);
  const size_t o_pb = im.put(pb);
  const size_t o_ppoff = im.put(ppoff);
  const size_t o_srot = im.put(site_rot);
  const size_t o_psite = im.put(pair_site);
  const size_t o_srep = im.put(site_rep);
  const size_t o_pppair = im.put(pp_pair);
  const size_t o_ppij = im.put(pp_ij);
  size_t o_pmol = 0, o_c0 = 0, o_nc = 0, o_out = 0, o_ld = 0;
  if (batch) {
    o_pmol = im.put(pmol);
    o_c0 = im.put(b->mol_c0);
    o_nc = im.put(b->mol_nc);
    o_out = im.put(b->mol_out);
    o_ld = im.put(b->mol_nbf);
  }
  const size_t o_cpit = batch ? im.put(cp_items) : 0;
  const size_t o_prit = batch ? im.put(pr_items) : 0;
  const size_t host_bytes = im.size();
  const size_t o_ppd = im.reserve(sizeof(PPData) * (size_t)ppcount);
  const size_t o_ctrl = im.reserve(ctrl_bytes(b->work.size()));
  const size_t o_rotd = im.reserve(sizeof(double) * (size_t)rotlen);
  shgo_status st = SHGO_OK;
  unsigned char* base = nullptr;
  {
    cudaError_t e = pool_alloc(device, (void**)&base, im.total());
    if (e != cudaSuccess) {
      st = e == cudaErrorMemoryAllocation ? SHGO_ERR_OOM : SHGO_ERR_CUDA;
      err = std::string("allocating basis arrays: ") + cudaGetErrorString(e);
    } else {
      b->allocations.push_back(base);
      e = cudaMemcpyAsync(base, im.data(), host_bytes, cudaMemcpyHostToDevice, 0);
      if (e != cudaSuccess) {
        st = SHGO_ERR_CUDA;
        err = std::string("copying the basis arrays: ") + cudaGetErrorString(e);
      }
    }
  }
  if (st == SHGO_OK) {
    b->d.shell_xyz = reinterpret_cast<double*>(base + o_xyz);
    b->d.shell_l = reinterpret_cast<int*>(base + o_l);
    b->d.shell_nprim = reinterpret_cast<int*>(base + o_np);
    b->d.shell_poff = reinterpret_cast<int*>(base + o_poff);
    b->d.shell_foff = reinterpret_cast<int64_t*>(base + o_foff);
    b->d.prim_exp = reinterpret_cast<double*>(base + o_exp);
    b->d.prim_coef = reinterpret_cast<double*>(base + o_coef);
    b->d.pair_a = reinterpret_cast<int*>(base + o_pa);
    b->d.pair_b = reinterpret_cast<int*>(base + o_pb);
    b->d.pair_ppoff = reinterpret_cast<int64_t*>(base + o_ppoff);
    b->d.site_rot = reinterpret_cast<double*>(base + o_srot);
    b->d.pair_site = reinterpret_cast<int*>(base + o_psite);
    b->d.site_rep = reinterpret_cast<int*>(base + o_srep);
    b->d.pp_pair = reinterpret_cast<int*>(base + o_pppair);
    b->d.pp_ij = reinterpret_cast<int*>(base + o_ppij);
    b->d.ppd = reinterpret_cast<PPData*>(base + o_ppd);
    b->d.rotd = reinterpret_cast<double*>(base + o_rotd);
    b->d.ctrl = base + o_ctrl;
    if (batch) {
      b->d.cp_items = reinterpret_cast<const int*>(base + o_cpit);
      b->d.pr_items = reinterpret_cast<const int*>(base + o_prit);
    }
    if (batch) {
      b->pair_mol = reinterpret_cast<int*>(base + o_pmol);
      b->mol_c0_d = reinterpret_cast<int64_t*>(base + o_c0);
      b->mol_nc_d = reinterpret_cast<int64_t*>(base + o_nc);
      b->mol_out_d = reinterpret_cast<int64_t*>(base + o_out);
      b->mol_ld_d = reinterpret_cast<int64_t*>(base + o_ld);
    }
  }
  if (st == SHGO_OK && (pinned_status_word(&b->h_err) != cudaSuccess ||
                        cudaEventCreateWithFlags(&b->done_ev, cudaEventDisableTiming) != cudaSuccess)) {
    st = SHGO_ERR_CUDA;
    err = "cannot create the status word or its event";
  }
  if (batch && st == SHGO_OK && cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    st = SHGO_ERR_CUDA;
    err = "cannot create the capture stream";
  }
  if (st == SHGO_OK) {
    b->d.rbuf_len = rlen;
    cudaError_t e = pool_alloc(device, (void**)&b->d.rbuf, sizeof(double) * (size_t)(rlen > 0 ? rlen : 1));
    if (e != cudaSuccess) {
      st = e == cudaErrorMemoryAllocation ? SHGO_ERR_OOM : SHGO_ERR_CUDA;
      err = std::string("allocating the coupling buffer: ") + cudaGetErrorString(e);
    } else {
      b->allocations.push_back(b->d.rbuf);
    }
  }
  if (st == SHGO_OK) st = device_tables(device, &b->tabs, &err);
  if (st == SHGO_OK) st = launch_pair_build(b->d, ppcount, 0, &err);
  if (st == SHGO_OK) st = launch_pair_rotations(b->d, *b->tabs, 0, &err);
  if (st == SHGO_OK && cudaDeviceSynchronize() != cudaSuccess) {
    st = SHGO_ERR_CUDA;
    err = "primitive-pair and pair-frame build failed";
  }
  b->ppcount = ppcount;
  if (st == SHGO_OK && b->sparse) {
    // block-sparse layout: pairs with a kept primitive pair, in pair order
    const int64_t np = (int64_t)pa.size();
    uint8_t* live = nullptr;
    cudaError_t e = pool_alloc(device, (void**)&live, (size_t)std::max<int64_t>(np, 1));
    if (e == cudaSuccess) {
      b->allocations.push_back(live);
      st = launch_pair_live(b->d, np, ppcount, live, 0, &err);
      std::vector<uint8_t> h(np);
      if (st == SHGO_OK && np) e = cudaMemcpy(h.data(), live, (size_t)np, cudaMemcpyDeviceToHost);
      b->h_blk_off.assign(np, -1);
      int64_t off = 0, nblk = 0;
      for (int64_t q = 0; q < np && e == cudaSuccess; ++q)
        if (h[q]) {
          b->h_blk_off[q] = off;
          off += (int64_t)(2 * l[pa[q]] + 1) * (2 * l[pb[q]] + 1);
          ++nblk;
        }
      b->sparse_nblocks = nblk;
      b->sparse_ndoubles = off;
      if (e == cudaSuccess) e = pool_alloc(device, (void**)&b->d_blk_off, sizeof(int64_t) * (size_t)std::max<int64_t>(np, 1));
      if (e == cudaSuccess) {
        b->allocations.push_back(b->d_blk_off);
        if (np) e = cudaMemcpy(b->d_blk_off, b->h_blk_off.data(), sizeof(int64_t) * (size_t)np, cudaMemcpyHostToDevice);
      }
    }
    if (e != cudaSuccess && st == SHGO_OK) {
      st = e == cudaErrorMemoryAllocation ? SHGO_ERR_OOM : SHGO_ERR_CUDA;
      err = std::string("block-sparse layout: ") + cudaGetErrorString(e);
    }
  }
  if (st != SHGO_OK) {
    release(b);
    return fail(st, err);
  }
  *out = b;
  return SHGO_OK;
}

}  // namespace

namespace {
// Per class wi of a basis: out[0] shell triples, out[1] unused, out[2] algorithmic flops of the
// coupling kernel (S2), out[3] flops of the pair kernel (S3-S5), out[4] primitive triples, out[5]
// integrals (shell triples x (2la+1)(2lb+1)).  Flops count an FMA as two.
// The per-class live counts behind the flop model, computed on first use (a kernel and a copy back).
shgo_status ensure_live_counts(const shgo_basis* cb, std::string* err) {
  shgo_basis* b = const_cast<shgo_basis*>(cb);
  std::lock_guard<std::mutex> lk(b->live_mu);
  if (b->live_ready) return SHGO_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  const shgo_status st = live_counts(b->d, b->work, b->npairs, b->ppcount, b->batch ? b->pair_mol : nullptr,
                                     b->batch ? b->mol_nc_d : nullptr, b->live_pp, b->live_pairs, b->live_cent, err);
  if (prev != b->device) cudaSetDevice(prev);
  b->live_ready = st == SHGO_OK;
  return st;
}

// Algorithmic FP64 operations of the coupling kernel of order lam per primitive triple: geometry 9; |d|^2, T,
// 1/|d|, |d| and the unit vector 11; Boys: Horner over kBoysK Taylor terms (5 per term), exp 1, downward
// recursion 3 per order; Z |d|^n F_n 2 Lambda + 1; (p |d|)^j / j! 2 per j; the beta running sums 2 per entry
// beyond the first of each L; the unit-vector harmonic recursion 6 l + 5 for level l + 1; the nucleus sum
// 2 per R entry.
double coupling_per_triple(int lam) {
  const double nB = n_beta(lam), nR = n_r(lam);
  double s_lm = 0.0;
  for (int l = 1; l < lam; ++l) s_lm += 6.0 * l + 5.0;
  const double boys = 5.0 * kBoysK + 1 + 3.0 * lam;
  return 9 + 11 + boys + (2.0 * lam + 1) + 2.0 * (lam / 2) + 2.0 * (nB - (lam + 1)) + s_lm + 2.0 * nR;
}

// Per (primitive pair, point) of the potential's point pass: the coupling kernel's per-nucleus tables and
// the sum grouped by radial row, one multiply-add per R' entry and one per radial row.
double esp_per_point(int lam) { return coupling_per_triple(lam) - 2.0 * n_r(lam) + 2.0 * (n_r(lam) + n_beta(lam)); }

// Per (primitive pair, point) of the gradient's point pass: the frame offset (20), Boys values to order
// lam + 1, T^k/k!, the radial rows B and -2p T^k/k! F (4 per row), the solid-harmonic polynomials with their
// gradients (26 per column recursion step, 3 per first step, 22 per step of the diagonal chain, 5 for r^2),
// the sums (per R' entry two products and four multiply-adds: a form grouped by harmonic row needs fewer
// operations but ran slower, having less independent work per thread), the offset term (6) and the rotation
// back to the molecular frame (18).
double esp_grad_per_point(int lam) {
  double harm = 5.0;
  for (int am = 0; am <= lam; ++am) {
    const double cols = am == 0 ? 1.0 : 2.0;
    if (am + 1 <= lam) harm += 3.0 * cols;
    harm += 26.0 * cols * std::max(0, lam - am - 1);
    if (am >= 1 && am < lam) harm += 22.0;
  }
  const double boys = 5.0 * kBoysK + 1 + 3.0 * (lam + 1);
  return 20.0 + boys + (lam / 2) + 4.0 * n_beta(lam) + harm + 10.0 * n_r(lam) + 24.0;
}

// The Gaunt coupling of one primitive pair into a (lbra, lket) block: 2 per nonzero coefficient of the class
// stored as (max, min).
double gaunt_flops(const Tables& t, int lbra, int lket) {
  return 2.0 * t.g_nnz[class_id(std::max(lbra, lket), std::min(lbra, lket))];
}

// Per shell pair: the translation of a (lbra, lket) block along the pair axis (diagonal in m) and its
// rotation back to the molecular frame.
double block_flops(int lbra, int lket) {
  const int nWa = (lbra + 1) * (lbra + 1);
  const double na = 2 * lbra + 1, nb = 2 * lket + 1;
  double zt = 0, vt = 0;
  for (int mb = -lket; mb <= lket; ++mb) zt += 2.0 * (lket - std::abs(mb) + 1) * nWa;
  for (int ma = -lbra; ma <= lbra; ++ma) vt += 2.0 * (lbra - std::abs(ma) + 1) * nb;
  return zt + vt + 2.0 * na * nb * nb + 2.0 * na * na * nb;
}

// One pass of the pair kernel over a (lbra, lket) block: per primitive pair the Gaunt coupling and 4 per W
// entry (the primitive factor and the accumulation); per shell pair the translation and rotation.
double pair_pass_flops(const Tables& t, int lbra, int lket, double live_pp, double live_pairs) {
  const double nW = (double)(lbra + 1) * (lbra + 1) * (lket + 1) * (lket + 1);
  return (gaunt_flops(t, lbra, lket) + 4.0 * nW) * live_pp + block_flops(lbra, lket) * live_pairs;
}

// Nonzero terms of the raising (which = 0) or the p-free field table (which = 1) of order lam, all components.
double deriv_table_nnz(const Tables& t, int lam, int which) {
  const std::vector<GTerm>& v = which == 0 ? t.d_raise : t.d_field;
  double n = 0;
  const size_t b = (size_t)t.d_xoff[lam] * 3 * kDerivSlots, e = (size_t)t.d_xoff[lam + 1] * 3 * kDerivSlots;
  for (size_t i = b; i < e; ++i) n += v[i].coef != 0.0 ? 1.0 : 0.0;
  return n;
}

void class_model(const shgo_basis* basis, size_t wi, int64_t n_centers, double* out) {
  const Tables& t = tables_host();
  const ClassWork& w = basis->work[wi];
  // nuclei seen by the class: per call for one molecule, per molecule for a batch.  Shell triples
  // count every pair (the output is complete); the work counts only live primitive pairs (those not
  // dropped by K_AB underflow or the per-basis bound) and shell pairs with at least one.
  const double pair_cent = basis->batch ? basis->class_pair_cent[wi] : (double)w.npairs * (double)n_centers;
  const double live_pp = (double)basis->live_pp[wi], live_pairs = (double)basis->live_pairs[wi];
  const double pp_cent = basis->batch ? basis->live_cent[wi] : live_pp * (double)n_centers;
  const int la = w.la, lb = w.lb, lam = la + lb;
  const double f0 = coupling_per_triple(lam) * pp_cent + 2.0 * n_r(lam) * live_pp;
  const double f1 = pair_pass_flops(t, la, lb, live_pp, live_pairs);
  const double na = 2 * la + 1, nb = 2 * lb + 1;
  out[0] = pair_cent;
  out[1] = 0;
  out[2] = f0;
  out[3] = f1;
  out[4] = basis->batch ? basis->class_pp_cent[wi] : (double)w.npp * (double)n_centers;
  out[5] = pair_cent * na * nb;
}
}  // namespace

namespace {
// After a call that launched kernels: the device error word into the basis's pinned status word, and the
// event that marks the copy (read by shgo_basis_sync).
cudaError_t status_readback(const shgo_basis* b, cudaStream_t s) {
  return cudaMemcpyAsync(b->h_err, b->d.ctrl, sizeof(int), cudaMemcpyDeviceToHost, s);
}
// A call without a time limit cannot change the error word, so only limited calls copy it.
cudaError_t finish_call(const shgo_basis* b, cudaStream_t s) {
  cudaError_t e = b->d.limit_ns != ~0ull ? status_readback(b, s) : cudaSuccess;
  if (e == cudaSuccess) e = cudaEventRecord(b->done_ev, s);
  return e;
}
}  // namespace

extern "C" {

shgo_status shgo_basis_create(int32_t n_shells, const int32_t* l, const int32_t* n_prim, const double* exponents,
                              const double* coefs, const double* shell_xyz, const shgo_options* opt,
                              shgo_basis** out) {
  return build_basis(n_shells, l, n_prim, exponents, coefs, shell_xyz, opt, 0, nullptr, nullptr, out);
}

shgo_status shgo_basis_create_shard(int32_t n_shells, const int32_t* l, const int32_t* n_prim,
                                    const double* exponents, const double* coefs, const double* shell_xyz,
                                    const shgo_options* opt, int32_t shard_index, int32_t shard_count,
                                    shgo_basis** out) {
  return build_basis(n_shells, l, n_prim, exponents, coefs, shell_xyz, opt, 0, nullptr, nullptr, out, shard_index,
                     shard_count);
}

shgo_status shgo_host_shard_of_pairs(int32_t n_shells, const int32_t* l, const int32_t* n_prim, int32_t shard_count,
                                     int64_t* npairs, int32_t* shard) {
  g_last_error.clear();
  if (n_shells < 0 || shard_count < 1 || !npairs || (n_shells > 0 && (!l || !n_prim)))
    return fail(SHGO_ERR_INVALID_ARG, "bad arguments");
  for (int s = 0; s < n_shells; ++s)
    if (l[s] < 0 || l[s] > kLmax || n_prim[s] < 1 || n_prim[s] > 64) return fail(SHGO_ERR_INVALID_ARG, "bad shell");
  // the library's pair order for one molecule (class by class, la >= lb, then shell index) and its
  // primitive-pair offsets
  std::vector<std::vector<int>> by_l(kLmax + 1);
  for (int s = 0; s < n_shells; ++s) by_l[l[s]].push_back(s);
  std::vector<ClassWork> work;
  std::vector<int64_t> ppoff;
  int64_t pp = 0;
  for (int la = 0; la <= kLmax; ++la)
    for (int lb = 0; lb <= la; ++lb) {
      ClassWork w{la, lb, 0, (int)ppoff.size(), 0, pp};
      const auto& A = by_l[la];
      const auto& B = by_l[lb];
      for (size_t x = 0; x < A.size(); ++x)
        for (size_t y = 0; y < ((la == lb) ? x + 1 : B.size()); ++y) {
          ppoff.push_back(pp);
          pp += (int64_t)n_prim[A[x]] * n_prim[B[y]];
          ++w.npairs;
        }
      w.npp = pp - w.pp_base;
      if (w.npairs > 0) work.push_back(w);
    }
  const int64_t np = (int64_t)ppoff.size();
  ppoff.push_back(pp);
  if (shard && *npairs >= np) {
    std::vector<int> sh;
    shard_of_pairs(work, ppoff, shard_count, sh);
    for (int64_t q = 0; q < np; ++q) shard[q] = sh[q];
  }
  *npairs = np;
  return SHGO_OK;
}

shgo_status shgo_batch_create(int32_t n_mol, const int32_t* mol_nshells, const int64_t* mol_ncenters, int32_t n_shells,
                              const int32_t* l, const int32_t* n_prim, const double* exponents, const double* coefs,
                              const double* shell_xyz, const shgo_options* opt, shgo_basis** out) {
  if (n_mol < 1) {
    g_last_error = "n_mol must be >= 1";
    return SHGO_ERR_INVALID_ARG;
  }
  return build_basis(n_shells, l, n_prim, exponents, coefs, shell_xyz, opt, n_mol, mol_nshells, mol_ncenters, out);
}

shgo_status shgo_batch_layout(const shgo_basis* batch, int64_t* mol_nbf, int64_t* mol_out_offset) {
  if (!batch || !batch->batch) return fail(SHGO_ERR_INVALID_ARG, "not a batch");
  for (int m = 0; m < batch->n_mol; ++m) {
    if (mol_nbf) mol_nbf[m] = batch->mol_nbf[m];
    if (mol_out_offset) mol_out_offset[m] = batch->mol_out[m];
  }
  return SHGO_OK;
}

int64_t shgo_batch_out_size(const shgo_basis* batch) { return batch && batch->batch ? batch->out_size : -1; }

shgo_status shgo_nuclear_attraction_batched(shgo_basis* batch, const double* centers, const double* charges,
                                            double* out, void* stream) {
  g_last_error.clear();
  if (!batch || !batch->batch) return fail(SHGO_ERR_INVALID_ARG, "not a batch");
  if (batch->total_centers > 0 && (!centers || !charges)) return fail(SHGO_ERR_INVALID_ARG, "NULL centers/charges");
  if (batch->out_size > 0 && !out) return fail(SHGO_ERR_INVALID_ARG, "out is NULL");
  if (batch->work.empty()) return SHGO_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != batch->device) cudaSetDevice(batch->device);
  MolView mv;
  mv.pair_mol = batch->pair_mol;
  mv.c0 = batch->mol_c0_d;
  mv.nc = batch->mol_nc_d;
  mv.out_off = batch->mol_out_d;
  mv.ld = batch->mol_ld_d;
  mv.ncenters = batch->total_centers;
  const double npp_cent = batch->npairs > 0 ? (double)batch->total_centers / batch->n_mol : 0.0;
  std::string err;
  shgo_status st = SHGO_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (!batch->tuned) {
    // first call: tune the launch shape of every class on the real work (its output is exact)
    st = autotune_batched(batch->d, *batch->tabs, batch->work, mv, centers, charges, out, &batch->tune, s, &err);
    if (st == SHGO_OK && batch->d.limit_ns != ~0ull && status_readback(batch, s) != cudaSuccess) {
      st = SHGO_ERR_CUDA;
      err = "status read-back failed";
    }
    if (st == SHGO_OK) batch->tuned = true;
  } else {
    const void* key[4] = {centers, charges, out, reinterpret_cast<const void*>((uintptr_t)batch->d.limit_ns)};
    if (!batch->graph || std::memcmp(key, batch->graph_key, sizeof(key)) != 0) {
      // capture the whole batch (all classes, both kernels, fork/join over the stream pool) once
      if (batch->graph) {
        cudaGraphExecDestroy(batch->graph);
        batch->graph = nullptr;
      }
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(batch->capture_stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        st = launch_batched(batch->d, *batch->tabs, batch->work, mv, npp_cent, centers, charges, out, &batch->tune,
                            batch->capture_stream, &err);
        if (st == SHGO_OK && batch->d.limit_ns != ~0ull) e = status_readback(batch, batch->capture_stream);
        const cudaError_t e2 = cudaStreamEndCapture(batch->capture_stream, &g);
        if (e == cudaSuccess) e = e2;
      }
      if (e == cudaSuccess && st == SHGO_OK) e = cudaGraphInstantiate(&batch->graph, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess || st != SHGO_OK) {
        if (st == SHGO_OK) {
          st = SHGO_ERR_CUDA;
          err = std::string("graph capture: ") + cudaGetErrorString(e);
        }
        batch->graph = nullptr;
      } else {
        std::memcpy(batch->graph_key, key, sizeof(key));
      }
    }
    if (st == SHGO_OK) {
      const cudaError_t e = cudaGraphLaunch(batch->graph, s);
      if (e != cudaSuccess) {
        st = SHGO_ERR_CUDA;
        err = std::string("graph launch: ") + cudaGetErrorString(e);
      }
    }
  }
  if (st == SHGO_OK) cudaEventRecord(batch->done_ev, s);
  if (prev != batch->device) cudaSetDevice(prev);
  if (st != SHGO_OK) return fail(st, err);
  return SHGO_OK;
}

namespace {
shgo_status esp_call(const shgo_basis* basis, const double* density, const shgo_centers* points, double* phi,
                     void* stream, bool gradient) {
  g_last_error.clear();
  if (!basis) return fail(SHGO_ERR_INVALID_ARG, "basis is NULL");
  if (basis->batch) return fail(SHGO_ERR_INVALID_ARG, "the potential takes a single basis, not a batch");
  if (basis->d.region > 0) return fail(SHGO_ERR_INVALID_ARG, "the potential needs the whole coupling buffer");
  if (!points || points->n < 0) return fail(SHGO_ERR_INVALID_ARG, "points is NULL or negative count");
  if (points->n > 0 && (!points->xyz || !phi)) return fail(SHGO_ERR_INVALID_ARG, "NULL points or phi");
  if (basis->nbf > 0 && !density) return fail(SHGO_ERR_INVALID_ARG, "density is NULL");
  if (points->n == 0) return SHGO_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != basis->device) cudaSetDevice(basis->device);
  std::string err;
  const shgo_status st = launch_esp(basis->d, *basis->tabs, basis->work, basis->nbf, density, points->n, points->xyz,
                                    phi, basis->d.rbuf, gradient, (cudaStream_t)stream, &err);
  if (prev != basis->device) cudaSetDevice(prev);
  if (st != SHGO_OK) return fail(st, err);
  return SHGO_OK;
}
}  // namespace

namespace {
shgo_status deriv_call(const shgo_basis* basis, const shgo_centers* centers, const double* charges, double* out,
                       void* stream, bool field) {
  g_last_error.clear();
  if (!basis) return fail(SHGO_ERR_INVALID_ARG, "basis is NULL");
  if (basis->batch) return fail(SHGO_ERR_INVALID_ARG, "derivative integrals take a single basis, not a batch");
  if (!centers || centers->n < 0) return fail(SHGO_ERR_INVALID_ARG, "centers is NULL or negative count");
  if (centers->n > 0 && (!centers->xyz || !charges)) return fail(SHGO_ERR_INVALID_ARG, "NULL centers/charges");
  if (basis->nbf > 0 && !out) return fail(SHGO_ERR_INVALID_ARG, "out is NULL");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != basis->device) cudaSetDevice(basis->device);
  std::string err;
  const shgo_status st = launch_nuclear_deriv(basis->d, *basis->tabs, basis->work, basis->nbf, centers->n,
                                              centers->xyz, charges, out, field, (cudaStream_t)stream, &err);
  if (prev != basis->device) cudaSetDevice(prev);
  if (st != SHGO_OK) return fail(st, err);
  return SHGO_OK;
}
}  // namespace

shgo_status shgo_nuclear_attraction_deriv(const shgo_basis* basis, const shgo_centers* centers,
                                          const double* charges, double* out, void* stream) {
  return deriv_call(basis, centers, charges, out, stream, false);
}

shgo_status shgo_nuclear_attraction_gradient(const shgo_basis* basis, const double* density,
                                             const shgo_centers* centers, const double* charges, double* grad,
                                             void* stream) {
  g_last_error.clear();
  if (!basis) return fail(SHGO_ERR_INVALID_ARG, "basis is NULL");
  if (basis->batch) return fail(SHGO_ERR_INVALID_ARG, "the gradient takes a single basis, not a batch");
  if (!centers || centers->n < 0) return fail(SHGO_ERR_INVALID_ARG, "centers is NULL or negative count");
  if (centers->n > 0 && (!centers->xyz || !charges)) return fail(SHGO_ERR_INVALID_ARG, "NULL centers/charges");
  if (basis->n_shells > 0 && (!grad || !density)) return fail(SHGO_ERR_INVALID_ARG, "grad or density is NULL");
  if (basis->n_shells == 0) return SHGO_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != basis->device) cudaSetDevice(basis->device);
  shgo_basis* mb = const_cast<shgo_basis*>(basis);
  std::string err;
  shgo_status st = SHGO_OK;
  {
    // each shell's (pair, side) entries in pair order, once per basis
    std::lock_guard<std::mutex> lk(mb->grad_mu);
    if (!mb->d_shell_off) {
      const int ns = basis->n_shells;
      const int64_t np = basis->npairs;
      std::vector<int64_t> off(ns + 1, 0), list;
      for (int64_t q = 0; q < np; ++q) {
        off[basis->h_pair_a[q] + 1] += 1;
        if (basis->h_pair_b[q] != basis->h_pair_a[q]) off[basis->h_pair_b[q] + 1] += 1;
      }
      for (int i = 0; i < ns; ++i) off[i + 1] += off[i];
      list.resize(off[ns]);
      std::vector<int64_t> pos(off.begin(), off.end() - 1);
      for (int64_t q = 0; q < np; ++q) {
        list[pos[basis->h_pair_a[q]]++] = 2 * q;
        if (basis->h_pair_b[q] != basis->h_pair_a[q]) list[pos[basis->h_pair_b[q]]++] = 2 * q + 1;
      }
      int64_t *doff = nullptr, *dlist = nullptr;
      cudaError_t e = pool_alloc(basis->device, (void**)&doff, sizeof(int64_t) * off.size());
      if (e == cudaSuccess) e = pool_alloc(basis->device, (void**)&dlist, sizeof(int64_t) * std::max<size_t>(list.size(), 1));
      if (e == cudaSuccess) e = cudaMemcpy(doff, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice);
      if (e == cudaSuccess && !list.empty())
        e = cudaMemcpy(dlist, list.data(), sizeof(int64_t) * list.size(), cudaMemcpyHostToDevice);
      if (doff) mb->allocations.push_back(doff);
      if (dlist) mb->allocations.push_back(dlist);
      if (e != cudaSuccess) {
        st = e == cudaErrorMemoryAllocation ? SHGO_ERR_OOM : SHGO_ERR_CUDA;
        err = std::string("gradient lists: ") + cudaGetErrorString(e);
      } else {
        mb->d_shell_off = doff;
        mb->d_shell_list = dlist;
      }
    }
  }
  if (st == SHGO_OK) {
    DerivContraction c;
    c.P = density;
    c.n_shells = basis->n_shells;
    c.shell_off = mb->d_shell_off;
    c.shell_list = mb->d_shell_list;
    c.grad = grad;
    st = launch_nuclear_deriv(basis->d, *basis->tabs, basis->work, basis->nbf, centers->n, centers->xyz, charges,
                              nullptr, false, (cudaStream_t)stream, &err, &c);
  }
  if (prev != basis->device) cudaSetDevice(prev);
  if (st != SHGO_OK) return fail(st, err);
  return SHGO_OK;
}

shgo_status shgo_nuclear_field(const shgo_basis* basis, const shgo_centers* centers, const double* charges,
                               double* out, void* stream) {
  return deriv_call(basis, centers, charges, out, stream, true);
}

shgo_status shgo_esp(const shgo_basis* basis, const double* density, const shgo_centers* points, double* phi,
                     void* stream) {
  return esp_call(basis, density, points, phi, stream, false);
}

shgo_status shgo_esp_gradient(const shgo_basis* basis, const double* density, const shgo_centers* points,
                              double* grad, void* stream) {
  return esp_call(basis, density, points, grad, stream, true);
}

shgo_status shgo_overlap(const shgo_basis* basis, double* out, void* stream) {
  g_last_error.clear();
  if (!basis) return fail(SHGO_ERR_INVALID_ARG, "basis is NULL");
  if (!out && (basis->batch ? basis->out_size : basis->nbf) > 0) return fail(SHGO_ERR_INVALID_ARG, "out is NULL");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != basis->device) cudaSetDevice(basis->device);
  MolView mv;
  if (basis->batch) {
    mv.pair_mol = basis->pair_mol;
    mv.c0 = basis->mol_c0_d;
    mv.nc = basis->mol_nc_d;
    mv.out_off = basis->mol_out_d;
    mv.ld = basis->mol_ld_d;
  }
  mv.nbf = basis->nbf;
  std::string err;
  const shgo_status st = launch_overlap(basis->d, *basis->tabs, basis->work, mv, out, (cudaStream_t)stream, &err);
  if (prev != basis->device) cudaSetDevice(prev);
  if (st != SHGO_OK) return fail(st, err);
  return SHGO_OK;
}

shgo_status shgo_coulomb_2c(const shgo_basis* basis, double* out, void* stream) {
  g_last_error.clear();
  if (!basis) return fail(SHGO_ERR_INVALID_ARG, "basis is NULL");
  if (!out && (basis->batch ? basis->out_size : basis->nbf) > 0) return fail(SHGO_ERR_INVALID_ARG, "out is NULL");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != basis->device) cudaSetDevice(basis->device);
  MolView mv;
  if (basis->batch) {
    mv.pair_mol = basis->pair_mol;
    mv.c0 = basis->mol_c0_d;
    mv.nc = basis->mol_nc_d;
    mv.out_off = basis->mol_out_d;
    mv.ld = basis->mol_ld_d;
  }
  mv.nbf = basis->nbf;
  std::string err;
  const shgo_status st = launch_coulomb2c(basis->d, *basis->tabs, tables_host(), basis->work, mv, out,
                                          (cudaStream_t)stream, &err);
  if (prev != basis->device) cudaSetDevice(prev);
  if (st != SHGO_OK) return fail(st, err);
  return SHGO_OK;
}

shgo_status shgo_eri(const shgo_basis* basis, double* out, void* stream) {
  g_last_error.clear();
  if (!basis) return fail(SHGO_ERR_INVALID_ARG, "basis is NULL");
  if (basis->shard_count > 1) return fail(SHGO_ERR_INVALID_ARG, "four-centre integrals need every shell pair, not a shard");
  if (basis->batch) return fail(SHGO_ERR_INVALID_ARG, "electron-repulsion integrals take a single basis, not a batch");
  if (basis->nbf > 40000) return fail(SHGO_ERR_INVALID_ARG, "nbf^4 output too large");
  for (const ClassWork& w : basis->work)
    if (w.la > kEriLmax) return fail(SHGO_ERR_UNSUPPORTED_L, "electron-repulsion integrals support l <= 4");
  if (!out && basis->nbf > 0) return fail(SHGO_ERR_INVALID_ARG, "out is NULL");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != basis->device) cudaSetDevice(basis->device);
  std::string err;
  const shgo_status st = launch_eri(basis->d, *basis->tabs, tables_host(), basis->work, basis->nbf, out, nullptr,
                                    nullptr, nullptr, (cudaStream_t)stream, &err);
  if (prev != basis->device) cudaSetDevice(prev);
  if (st != SHGO_OK) return fail(st, err);
  return SHGO_OK;
}

shgo_status shgo_eri_jk(const shgo_basis* basis, const double* density, double* J, double* K, void* stream) {
  g_last_error.clear();
  if (!basis) return fail(SHGO_ERR_INVALID_ARG, "basis is NULL");
  if (basis->shard_count > 1) return fail(SHGO_ERR_INVALID_ARG, "four-centre integrals need every shell pair, not a shard");
  if (basis->batch) return fail(SHGO_ERR_INVALID_ARG, "electron-repulsion integrals take a single basis, not a batch");
  for (const ClassWork& w : basis->work)
    if (w.la > kEriLmax) return fail(SHGO_ERR_UNSUPPORTED_L, "electron-repulsion integrals support l <= 4");
  if (basis->nbf > 0 && (!density || (!J && !K))) return fail(SHGO_ERR_INVALID_ARG, "NULL density or no output");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != basis->device) cudaSetDevice(basis->device);
  std::string err;
  shgo_status st = SHGO_OK;
  const size_t bytes = sizeof(double) * (size_t)basis->nbf * (size_t)basis->nbf;
  cudaError_t e = cudaSuccess;
  if (J && bytes) e = cudaMemsetAsync(J, 0, bytes, (cudaStream_t)stream);
  if (e == cudaSuccess && K && bytes) e = cudaMemsetAsync(K, 0, bytes, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    st = SHGO_ERR_CUDA;
    err = std::string("clearing J, K: ") + cudaGetErrorString(e);
  } else {
    st = launch_eri(basis->d, *basis->tabs, tables_host(), basis->work, basis->nbf, nullptr, density, J, K,
                    (cudaStream_t)stream, &err);
  }
  if (prev != basis->device) cudaSetDevice(prev);
  if (st != SHGO_OK) return fail(st, err);
  return SHGO_OK;
}

int64_t shgo_basis_nbf(const shgo_basis* basis) { return basis ? basis->nbf : -1; }
int64_t shgo_basis_npairs(const shgo_basis* basis) { return basis ? basis->npairs : -1; }

shgo_status shgo_sparse_layout(const shgo_basis* basis, int64_t* nblocks, int64_t* ndoubles, int64_t* offset) {
  g_last_error.clear();
  if (!basis) return fail(SHGO_ERR_INVALID_ARG, "basis is NULL");
  if (!basis->sparse) return fail(SHGO_ERR_INVALID_ARG, "the basis was not created with SHGO_FLAG_BLOCK_SPARSE");
  if (nblocks) *nblocks = basis->sparse_nblocks;
  if (ndoubles) *ndoubles = basis->sparse_ndoubles;
  if (offset) std::copy(basis->h_blk_off.begin(), basis->h_blk_off.end(), offset);
  return SHGO_OK;
}

shgo_status shgo_nuclear_attraction(const shgo_basis* basis, const shgo_centers* centers, const double* charges,
                                    double* out, void* stream) {
  g_last_error.clear();
  if (!basis) return fail(SHGO_ERR_INVALID_ARG, "basis is NULL");
  if (!centers || centers->n < 0) return fail(SHGO_ERR_INVALID_ARG, "centers is NULL or negative count");
  if (centers->n > 0 && (!centers->xyz || !charges)) return fail(SHGO_ERR_INVALID_ARG, "NULL centers/charges");
  if (basis->nbf > 0 && !out) return fail(SHGO_ERR_INVALID_ARG, "out is NULL");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != basis->device) cudaSetDevice(basis->device);
  std::string err;
  shgo_status st = SHGO_OK;
  // A call that repeats the previous call's pointers, nucleus count and time limit replays the previous
  // call's launch sequence, captured into a CUDA graph on the first repetition.
  shgo_basis* mb = const_cast<shgo_basis*>(basis);
  const cudaStream_t s = (cudaStream_t)stream;
  const void* key[4] = {centers->xyz, charges, out,
                        reinterpret_cast<const void*>((uintptr_t)(centers->n * 1000003 + (int64_t)(basis->d.limit_ns & 0xffffff)))};
  const bool work = basis->nbf > 0 && centers->n > 0;
  const bool repeat = work && mb->single_key_set && std::memcmp(key, mb->graph_key, sizeof(key)) == 0 &&
                      mb->single_limit == basis->d.limit_ns;
  auto direct = [&](cudaStream_t on) {
    return launch_nuclear_attraction(basis->d, *basis->tabs, basis->work, basis->nbf, centers->n, centers->xyz,
                                     charges, out, on, &err, nullptr, true,
                                     basis->sparse ? basis->d_blk_off : nullptr, basis->sparse_ndoubles);
  };
  if (repeat) {
    if (!mb->graph) {
      cudaError_t e = mb->capture_stream ? cudaSuccess
                                         : cudaStreamCreateWithFlags(&mb->capture_stream, cudaStreamNonBlocking);
      cudaGraph_t g = nullptr;
      if (e == cudaSuccess) e = cudaStreamBeginCapture(mb->capture_stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        st = direct(mb->capture_stream);
        e = cudaStreamEndCapture(mb->capture_stream, &g);
      }
      if (e == cudaSuccess && st == SHGO_OK) e = cudaGraphInstantiate(&mb->graph, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess || st != SHGO_OK) {
        mb->graph = nullptr;
        if (st == SHGO_OK) {
          st = SHGO_ERR_CUDA;
          err = std::string("graph capture: ") + cudaGetErrorString(e);
        }
      }
    }
    if (st == SHGO_OK) {
      const cudaError_t e = cudaGraphLaunch(mb->graph, s);
      if (e != cudaSuccess) {
        st = SHGO_ERR_CUDA;
        err = std::string("graph launch: ") + cudaGetErrorString(e);
      }
    }
  } else {
    if (mb->graph) {
      cudaGraphExecDestroy(mb->graph);
      mb->graph = nullptr;
    }
    std::memcpy(mb->graph_key, key, sizeof(key));
    mb->single_key_set = work;
    mb->single_limit = basis->d.limit_ns;
    st = direct(s);
  }
  if (st == SHGO_OK && work && finish_call(basis, s) != cudaSuccess) {
    st = SHGO_ERR_CUDA;
    err = "status read-back failed";
  }
  if (prev != basis->device) cudaSetDevice(prev);
  if (st != SHGO_OK) return fail(st, err);
  return SHGO_OK;
}

shgo_status shgo_basis_set_time_limit(shgo_basis* basis, double seconds) {
  g_last_error.clear();
  if (!basis) return fail(SHGO_ERR_INVALID_ARG, "basis is NULL");
  if (!(seconds >= 0)) return fail(SHGO_ERR_INVALID_ARG, "time limit must be >= 0 (infinity = none)");
  basis->d.limit_ns = std::isinf(seconds) || seconds >= 1.8e10 ? ~0ull : (unsigned long long)(seconds * 1e9);
  return SHGO_OK;
}

shgo_status shgo_basis_sync(const shgo_basis* basis) {
  g_last_error.clear();
  if (!basis) return fail(SHGO_ERR_INVALID_ARG, "basis is NULL");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != basis->device) cudaSetDevice(basis->device);
  const cudaError_t e = cudaEventSynchronize(basis->done_ev);
  if (prev != basis->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return fail(SHGO_ERR_CUDA, std::string("waiting for the basis: ") + cudaGetErrorString(e));
  const int v = *basis->h_err;
  if (v != 0) {
    // clear the word on both sides; the basis's last call has completed, and calls on one basis are ordered
    *basis->h_err = 0;
    if (prev != basis->device) cudaSetDevice(basis->device);
    const cudaError_t ec = cudaMemset(basis->d.ctrl, 0, sizeof(int));
    if (prev != basis->device) cudaSetDevice(prev);
    if (ec != cudaSuccess) return fail(SHGO_ERR_CUDA, std::string("clearing the status: ") + cudaGetErrorString(ec));
    if (v == SHGO_ERR_TIMEOUT)
      return fail(SHGO_ERR_TIMEOUT, "a launch of the last call reached the basis's time limit; its output is incomplete");
    return fail(SHGO_ERR_CUDA, "device status word " + std::to_string(v));
  }
  return SHGO_OK;
}

shgo_status shgo_nuclear_attraction_timed(const shgo_basis* basis, const shgo_centers* centers,
                                          const double* charges, double* out, void* stream, double* phase_ms) {
  g_last_error.clear();
  if (!basis || !phase_ms) return fail(SHGO_ERR_INVALID_ARG, "basis or phase_ms is NULL");
  if (!centers || centers->n < 0) return fail(SHGO_ERR_INVALID_ARG, "centers is NULL or negative count");
  if (centers->n > 0 && (!centers->xyz || !charges)) return fail(SHGO_ERR_INVALID_ARG, "NULL centers/charges");
  if (basis->nbf > 0 && !out) return fail(SHGO_ERR_INVALID_ARG, "out is NULL");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != basis->device) cudaSetDevice(basis->device);
  cudaEvent_t ev[3];
  for (auto& e : ev) cudaEventCreate(&e);
  std::string err;
  shgo_status st = launch_nuclear_attraction(basis->d, *basis->tabs, basis->work, basis->nbf, centers->n,
                                             centers->xyz, charges, out, (cudaStream_t)stream, &err, ev, true,
                                             basis->sparse ? basis->d_blk_off : nullptr, basis->sparse_ndoubles);
  if (st == SHGO_OK && basis->nbf > 0 && centers->n > 0) finish_call(basis, (cudaStream_t)stream);
  if (st == SHGO_OK) {
    cudaError_t e = cudaEventSynchronize(ev[2]);
    float t0 = 0, t1 = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t0, ev[0], ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t1, ev[1], ev[2]);
    if (e != cudaSuccess) {
      st = SHGO_ERR_CUDA;
      err = cudaGetErrorString(e);
    }
    phase_ms[0] = t0;
    phase_ms[1] = t1;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (prev != basis->device) cudaSetDevice(prev);
  if (st != SHGO_OK) return fail(st, err);
  return SHGO_OK;
}

int64_t shgo_basis_launches(const shgo_basis* basis) { return basis ? launches_per_call(basis->work, basis->nbf) : -1; }

shgo_status shgo_basis_flops(const shgo_basis* basis, int64_t n_centers, double* flops, double* triples) {
  if (!basis || !flops || !triples || n_centers < 0) return fail(SHGO_ERR_INVALID_ARG, "bad arguments");
  {
    std::string err;
    const shgo_status st = ensure_live_counts(basis, &err);
    if (st != SHGO_OK) return fail(st, err);
  }
  flops[0] = flops[1] = triples[0] = triples[1] = 0;
  for (size_t wi = 0; wi < basis->work.size(); ++wi) {
    double c[6];
    class_model(basis, wi, n_centers, c);
    flops[0] += c[2];
    flops[1] += c[3];
    triples[0] += c[0];
    triples[1] += c[4];
  }
  return SHGO_OK;
}

shgo_status shgo_basis_deriv_flops(const shgo_basis* basis, int64_t n_centers, int32_t field, double* flops) {
  if (!basis || !flops || n_centers < 0 || basis->batch) return fail(SHGO_ERR_INVALID_ARG, "bad arguments");
  {
    std::string err;
    const shgo_status st = ensure_live_counts(basis, &err);
    if (st != SHGO_OK) return fail(st, err);
  }
  const Tables& t = tables_host();
  flops[0] = flops[1] = 0;
  for (size_t wi = 0; wi < basis->work.size(); ++wi) {
    const ClassWork& w = basis->work[wi];
    const int la = w.la, lb = w.lb, lam = la + lb;
    const double live_pp = (double)basis->live_pp[wi], live_pairs = (double)basis->live_pairs[wi];
    flops[0] += coupling_per_triple(lam + 1) * live_pp * (double)n_centers + 2.0 * n_r(lam + 1) * live_pp;
    const double na = 2 * la + 1, nb = 2 * lb + 1;
    if (field) {
      // three differentiated blocks (raising, p-free terms, one combining FMA per entry), then Q^T per entry
      const double tr = 2.0 * (deriv_table_nnz(t, lam, 0) + deriv_table_nnz(t, lam, 1)) + 2.0 * 3 * n_r(lam);
      flops[1] += tr * live_pp + 3.0 * pair_pass_flops(t, la, lb, live_pp, live_pairs) + 18.0 * na * nb * w.npairs;
      continue;
    }
    // per primitive pair: the raising of the three axes; the Gaunt coupling of the three raised blocks and of
    // the unraised one (the pair-axis offsets of both centres on z); per W entry and centre 4 for x and y and
    // 6 for z.  Per shell pair: translation and rotation of the six raised blocks; then the lowered classes.
    const double nW = (double)(la + 1) * (la + 1) * (lb + 1) * (lb + 1);
    flops[1] += (2.0 * deriv_table_nnz(t, lam, 0) + 4.0 * gaunt_flops(t, la, lb) + 2.0 * 14.0 * nW) * live_pp +
                6.0 * block_flops(la, lb) * live_pairs;
    if (la > 0) flops[1] += pair_pass_flops(t, la - 1, lb, live_pp, live_pairs);
    if (lb > 0) flops[1] += pair_pass_flops(t, la, lb - 1, live_pp, live_pairs);
    // combine: per element and component 6 (the frame rotation) + 2 (2l - 1) (lowered), for both orientations
    flops[1] += 3.0 * na * nb * w.npairs * (2.0 * 6.0 + 2.0 * (2 * la - 1) + 2.0 * (2 * lb - 1));
  }
  return SHGO_OK;
}

shgo_status shgo_basis_esp_flops(const shgo_basis* basis, int64_t n_points, int32_t gradient, double* flops) {
  if (!basis || !flops || n_points < 0 || basis->batch) return fail(SHGO_ERR_INVALID_ARG, "bad arguments");
  {
    std::string err;
    const shgo_status st = ensure_live_counts(basis, &err);
    if (st != SHGO_OK) return fail(st, err);
  }
  const Tables& t = tables_host();
  flops[0] = flops[1] = 0;
  for (size_t wi = 0; wi < basis->work.size(); ++wi) {
    const ClassWork& w = basis->work[wi];
    const int lam = w.la + w.lb;
    const double live_pp = (double)basis->live_pp[wi], live_pairs = (double)basis->live_pairs[wi];
    // the adjoint pass is the pair kernel's operation count read backwards, plus the R' scale
    flops[0] += pair_pass_flops(t, w.la, w.lb, live_pp, live_pairs) + 2.0 * n_r(lam) * live_pp;
    flops[1] += (gradient ? esp_grad_per_point(lam) : esp_per_point(lam)) * live_pp * (double)n_points;
  }
  return SHGO_OK;
}

int32_t shgo_basis_nclasses(const shgo_basis* basis) { return basis ? (int32_t)basis->work.size() : -1; }

shgo_status shgo_basis_class_stats(const shgo_basis* basis, int64_t n_centers, int32_t c, int32_t* la_lb,
                                   double* stats) {
  if (!basis || !la_lb || !stats || n_centers < 0 || c < 0 || c >= (int32_t)basis->work.size())
    return fail(SHGO_ERR_INVALID_ARG, "bad arguments");
  {
    std::string err;
    const shgo_status st = ensure_live_counts(basis, &err);
    if (st != SHGO_OK) return fail(st, err);
  }
  double m[6];
  class_model(basis, (size_t)c, n_centers, m);
  la_lb[0] = basis->work[c].la;
  la_lb[1] = basis->work[c].lb;
  stats[0] = m[0];
  stats[1] = m[5];
  stats[2] = m[2];
  stats[3] = m[3];
  return SHGO_OK;
}

shgo_status shgo_nuclear_attraction_class_timed(const shgo_basis* basis, const shgo_centers* centers,
                                                const double* charges, double* out, void* stream, double* ms) {
  g_last_error.clear();
  if (!basis || !ms) return fail(SHGO_ERR_INVALID_ARG, "basis or ms is NULL");
  if (!centers || centers->n < 0) return fail(SHGO_ERR_INVALID_ARG, "centers is NULL or negative count");
  if (centers->n > 0 && (!centers->xyz || !charges)) return fail(SHGO_ERR_INVALID_ARG, "NULL centers/charges");
  if ((basis->batch ? basis->out_size : basis->nbf) > 0 && !out) return fail(SHGO_ERR_INVALID_ARG, "out is NULL");
  if (basis->d.region > 0) return fail(SHGO_ERR_INVALID_ARG, "class timing needs the whole coupling buffer");
  if (basis->batch && centers->n != basis->total_centers)
    return fail(SHGO_ERR_INVALID_ARG, "a batch takes all its molecules' nuclei");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != basis->device) cudaSetDevice(basis->device);
  MolView mv;
  if (basis->batch) {
    mv.pair_mol = basis->pair_mol;
    mv.c0 = basis->mol_c0_d;
    mv.nc = basis->mol_nc_d;
    mv.out_off = basis->mol_out_d;
    mv.ld = basis->mol_ld_d;
  }
  mv.ncenters = centers->n;
  mv.nbf = basis->nbf;
  mv.blk_off = basis->sparse ? basis->d_blk_off : nullptr;
  std::string err;
  const shgo_status st = launch_class_timed(basis->d, *basis->tabs, basis->work, mv, centers->xyz, charges, out,
                                            (cudaStream_t)stream, ms, &err);
  if (prev != basis->device) cudaSetDevice(prev);
  if (st != SHGO_OK) return fail(st, err);
  return SHGO_OK;
}

void shgo_free(shgo_basis* basis) { release(basis); }

shgo_status shgo_host_solid_harmonics(int32_t l, int64_t npts, const double* xyz, double* out) {
  if (l < 0 || l > kHarmMax || npts < 0 || (npts > 0 && (!xyz || !out)))
    return fail(SHGO_ERR_INVALID_ARG, "bad arguments");
  const HarmCoef& hc = harm_coef_host();
  std::vector<double> buf(n_harm(l));
  for (int64_t p = 0; p < npts; ++p) {
    solid_harmonics(l, xyz[3 * p], xyz[3 * p + 1], xyz[3 * p + 2], buf.data(), 1, hc.a, hc.b, hc.c);
    for (int m = -l; m <= l; ++m) out[p * (2 * l + 1) + m + l] = buf[harm_index(l, m)];
  }
  return SHGO_OK;
}

double shgo_host_gaunt(int32_t l1, int32_t m1, int32_t l2, int32_t m2, int32_t L, int32_t M) {
  if (l1 < 0 || l2 < 0 || l1 > kLmax || l2 > kLmax || L < 0) return 0.0;
  return gaunt_real(l1, m1, l2, m2, L, M);
}

double shgo_host_translation(int32_t la, int32_t ma, int32_t l1, int32_t m1, int32_t nu) {
  if (la < 0 || la > kLmax) return 0.0;
  return translation_real(la, ma, l1, m1, nu);
}

double shgo_host_laplacian_coef(int32_t L, int32_t k, int32_t j) {
  if (L < 0 || L > kLamMax || k < 0 || k > kC2K || j < 0 || j > k) return 0.0;
  return tables_host().c2_a[((size_t)L * (kC2K + 1) + k) * (kC2K + 1) + j];
}

double shgo_host_eri_eps(int32_t L, int32_t k, int32_t n) {
  if (L < 0 || L > kLamMax || k < 0 || k > kC2K || n < 0 || n > k) return 0.0;
  return tables_host().eri_eps[((size_t)L * (kC2K + 1) + k) * (kC2K + 1) + n];
}

shgo_status shgo_host_deriv_transform(int32_t lam, int32_t comp, double p, const double* r1, double* raised,
                                      double* field) {
  if (lam < 0 || lam > kLamMax || comp < 0 || comp > 2 || !r1 || !raised || !field)
    return fail(SHGO_ERR_INVALID_ARG, "bad arguments");
  const Tables& t = tables_host();
  for (int e = 0; e < n_r(lam); ++e) {
    const GTerm* tr = &t.d_raise[((size_t)(t.d_xoff[lam] + e) * 3 + comp) * kDerivSlots];
    const GTerm* tf = &t.d_field[((size_t)(t.d_xoff[lam] + e) * 3 + comp) * kDerivSlots];
    double s = 0.0, f = 0.0;
    for (int k = 0; k < kDerivSlots; ++k) {
      s += tr[k].coef * r1[tr[k].ridx];
      f += tf[k].coef * r1[tf[k].ridx];
    }
    raised[e] = s;
    field[e] = f - 2.0 * p * s;
  }
  return SHGO_OK;
}

shgo_status shgo_host_deriv_lowering(int32_t l, int32_t comp, int32_t m, double* w) {
  if (l < 1 || l > kLmax || comp < 0 || comp > 2 || m < -l || m > l || !w)
    return fail(SHGO_ERR_INVALID_ARG, "bad arguments");
  const Tables& t = tables_host();
  for (int k = 0; k < 2 * l - 1; ++k) w[k] = t.d_low[t.d_low_off[l] + ((size_t)comp * (2 * l + 1) + m + l) * (2 * l - 1) + k];
  return SHGO_OK;
}

shgo_status shgo_host_boys(int32_t nmax, double T, double* F) {
  if (nmax < 0 || nmax > kLamMax + 1 || !F || !(T >= 0) || !std::isfinite(T))
    return fail(SHGO_ERR_INVALID_ARG, "bad arguments");
  boys_host(nmax, T, F);
  return SHGO_OK;
}


// ---------------------------------------------------------------------------------------------
// Learned screening (include/shgo_mlp.h)
// ---------------------------------------------------------------------------------------------
static ScreenBasis screen_view(const shgo_basis* b, int64_t n_centers) {
  ScreenBasis sb;
  sb.shell_xyz = b->d.shell_xyz;
  sb.shell_l = b->d.shell_l;
  sb.shell_nprim = b->d.shell_nprim;
  sb.shell_poff = b->d.shell_poff;
  sb.prim_exp = b->d.prim_exp;
  sb.prim_coef = b->d.prim_coef;
  sb.pair_a = b->d.pair_a;
  sb.pair_b = b->d.pair_b;
  sb.pair_mol = b->batch ? b->pair_mol : nullptr;
  sb.mol_c0 = b->batch ? b->mol_c0_d : nullptr;
  sb.mol_nc = b->batch ? b->mol_nc_d : nullptr;
  sb.ncenters = n_centers;
  sb.mask_off = b->scr_mask_off;
  sb.clist_off = b->scr_clist_off;
  return sb;
}

shgo_status shgo_pair_shells(const shgo_basis* basis, int32_t* shell_a, int32_t* shell_b) {
  if (!basis || !shell_a || !shell_b) return fail(SHGO_ERR_INVALID_ARG, "NULL argument");
  for (int64_t q = 0; q < basis->npairs; ++q) {
    shell_a[q] = basis->h_pair_a[q];
    shell_b[q] = basis->h_pair_b[q];
  }
  return SHGO_OK;
}

shgo_status shgo_screen_features(const shgo_basis* basis, const double* centers, const double* charges,
                                 const int32_t* triples, int64_t n, float* X, void* stream) {
  if (!basis || n < 0 || (n > 0 && (!centers || !charges || !triples || !X)))
    return fail(SHGO_ERR_INVALID_ARG, "bad arguments");
  return launch_screen_features(screen_view(basis, 0), centers, charges, triples, n, X, (cudaStream_t)stream);
}

shgo_status shgo_screen_build(shgo_basis* basis, const shgo_mlp* mlp, const double* centers, const double* charges,
                              int64_t n_centers, double log10_threshold, double log10_margin, int64_t* kept,
                              int64_t* skipped) {
  g_last_error.clear();
  if (!basis || !mlp) return fail(SHGO_ERR_INVALID_ARG, "NULL basis or network");
  const int64_t nc_total = basis->batch ? basis->total_centers : n_centers;
  if (nc_total < 0 || (nc_total > 0 && (!centers || !charges))) return fail(SHGO_ERR_INVALID_ARG, "bad nuclei");
  cudaFree(basis->scr_mask);
  cudaFree(basis->scr_mask_off);
  cudaFree(basis->scr_counts);
  cudaFree(basis->scr_clist_off);
  cudaFree(basis->scr_clist);
  basis->scr_mask = nullptr;
  basis->scr_mask_off = basis->scr_counts = basis->scr_clist_off = nullptr;
  basis->scr_clist = nullptr;
  const int64_t np = basis->npairs;
  std::vector<int64_t> moff(np + 1, 0);
  for (int64_t q = 0; q < np; ++q)
    moff[q + 1] = moff[q] + (basis->batch ? basis->mol_nc[basis->h_pair_mol[q]] : n_centers);
  const int64_t ntrip = moff[np];
  cudaError_t e = cudaSuccess;
  e = cudaMalloc((void**)&basis->scr_mask_off, sizeof(int64_t) * (np + 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&basis->scr_counts, sizeof(int64_t) * (np + 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&basis->scr_clist_off, sizeof(int64_t) * (np + 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&basis->scr_mask, ntrip > 0 ? ntrip : 1);
  if (e == cudaSuccess) e = cudaMemcpy(basis->scr_mask_off, moff.data(), sizeof(int64_t) * (np + 1), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? SHGO_ERR_OOM : SHGO_ERR_CUDA, cudaGetErrorString(e));
  const float cut = (float)(log10_threshold - log10_margin);
  ScreenBasis sb = screen_view(basis, n_centers);
  shgo_status st = launch_screen_pairs(sb, np, centers, charges, mlp, cut, 0, basis->scr_mask, basis->scr_counts,
                                       nullptr, 0);
  if (st != SHGO_OK) return st;
  std::vector<int64_t> counts(np), coff(np + 1, 0);
  if (np > 0 && cudaMemcpy(counts.data(), basis->scr_counts, sizeof(int64_t) * np, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(SHGO_ERR_CUDA, "screen counts copy failed");
  for (int64_t q = 0; q < np; ++q) coff[q + 1] = coff[q] + counts[q];
  e = cudaMemcpy(basis->scr_clist_off, coff.data(), sizeof(int64_t) * (np + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)&basis->scr_clist, sizeof(int) * (coff[np] > 0 ? coff[np] : 1));
  if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? SHGO_ERR_OOM : SHGO_ERR_CUDA, cudaGetErrorString(e));
  sb.clist_off = basis->scr_clist_off;
  st = launch_screen_pairs(sb, np, centers, charges, mlp, cut, 1, basis->scr_mask, basis->scr_counts,
                           basis->scr_clist, 0);
  if (st != SHGO_OK) return st;
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(SHGO_ERR_CUDA, cudaGetErrorString(e));
  basis->scr_ntrip = ntrip;
  basis->scr_ncenters = n_centers;
  if (kept) *kept = coff[np];
  if (skipped) *skipped = ntrip - coff[np];
  return SHGO_OK;
}

shgo_status shgo_screen_mask(const shgo_basis* basis, uint8_t* mask) {
  if (!basis || !mask || !basis->scr_mask) return fail(SHGO_ERR_INVALID_ARG, "no screening built");
  if (basis->scr_ntrip > 0 &&
      cudaMemcpy(mask, basis->scr_mask, (size_t)basis->scr_ntrip, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(SHGO_ERR_CUDA, "mask copy failed");
  return SHGO_OK;
}

shgo_status shgo_nuclear_attraction_screened(shgo_basis* basis, const double* centers, const double* charges,
                                             int64_t n_centers, double* out, void* stream) {
  g_last_error.clear();
  if (!basis || !basis->scr_clist) return fail(SHGO_ERR_INVALID_ARG, "no screening built for this basis");
  if (!basis->batch && n_centers != basis->scr_ncenters)
    return fail(SHGO_ERR_INVALID_ARG, "nucleus count differs from the screening build");
  if (!out && (basis->batch ? basis->out_size : basis->nbf) > 0) return fail(SHGO_ERR_INVALID_ARG, "out is NULL");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != basis->device) cudaSetDevice(basis->device);
  MolView mv;
  if (basis->batch) {
    mv.pair_mol = basis->pair_mol;
    mv.c0 = basis->mol_c0_d;
    mv.nc = basis->mol_nc_d;
    mv.out_off = basis->mol_out_d;
    mv.ld = basis->mol_ld_d;
  }
  mv.ncenters = basis->batch ? basis->total_centers : n_centers;
  mv.nbf = basis->nbf;
  mv.clist = basis->scr_clist;
  mv.clist_off = basis->scr_clist_off;
  mv.blk_off = basis->sparse ? basis->d_blk_off : nullptr;
  const double per_pair = basis->npairs > 0 ? (double)basis->scr_ntrip / (double)basis->npairs : 0.0;
  std::string err;
  shgo_status st = launch_batched(basis->d, *basis->tabs, basis->work, mv, per_pair, centers, charges, out,
                                  basis->tuned ? &basis->tune : nullptr, (cudaStream_t)stream, &err);
  if (st == SHGO_OK) finish_call(basis, (cudaStream_t)stream);
  if (prev != basis->device) cudaSetDevice(prev);
  if (st != SHGO_OK) return fail(st, err);
  return SHGO_OK;
}

}  // extern "C"
