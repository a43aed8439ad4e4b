// shgo_nuclear_attraction_noalloc: the nuclear-attraction matrix without any device allocation.
//
// Some callers cannot call cudaMalloc: a host process whose device memory is owned by an external
// pool manager that forbids foreign allocations, or code that must not enter the CUDA allocator
// while it runs.  shgo_basis_create allocates (shell arrays, pair lists, the per-primitive-pair
// coupling buffer, and on first use the constant tables), so such callers get this one entry
// point instead.  Everything it needs on the device lives in one file-scope static array of
// kNoallocScratchBytes (SHGO_NOALLOC_SCRATCH_BYTES), which every GPU that loads the library keeps
// until the process exits:
//   [ constant tables, copied in once per device ][ this call's shells, pair lists and coupling buffer ]
// The kernels are the ones shgo_nuclear_attraction launches; only their buffers differ.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_set>
#include <vector>

#include "shgo_internal.h"

namespace shgo {
shgo_status upload_constants(std::string* err);  // shgo_kernels.cu
void set_last_error(const std::string& msg);     // shgo_api.cpp (read by shgo_last_error)
}

using namespace shgo;

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)SHGO_NOALLOC_SCRATCH_BYTES;

// The scratch.  In host code this name is only a stand-in for the device array: its device address
// comes from cudaGetSymbolAddress at set-up and is what the kernels receive.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

struct NoallocDevice {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_noalloc_scratch on this device
  size_t tables_end = 0;          // first byte after the tables
  DeviceTables tabs;
};
std::mutex g_noalloc_mu;
NoallocDevice g_noalloc_dev[64];

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

// Byte layout of a list of arrays packed back to back, each 256-byte aligned.
struct Packer {
  size_t used = 0;
  size_t add(size_t bytes) {
    const size_t off = used;
    used = align256(used + bytes);
    return off;
  }
};

// Once per device, with that device current: the scratch address, the tables and the constants.
shgo_status noalloc_setup(int device, NoallocDevice** out, std::string* err) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoallocDevice& d = g_noalloc_dev[device];
  if (d.ready) {
    *out = &d;
    return SHGO_OK;
  }
  void* ptr = nullptr;
  // The CUDA driver loads this file's module, and with it commits the array's device memory, when the
  // module is first used on the device, which is here; no room for it then is an out-of-memory error.
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) {
    *err = std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();  // not a sticky error: clear it so the caller's next CUDA call does not report it
      return SHGO_ERR_OOM;
    }
    return SHGO_ERR_CUDA;
  }
  d.base = static_cast<unsigned char*>(ptr);
  const Tables& t = tables_host();
  Packer pk;
  const size_t o_boys = pk.add(t.boys.size() * sizeof(double));
  const size_t o_etab = pk.add(t.etab.size() * sizeof(double));
  const size_t o_eoff = pk.add(t.eoff.size() * sizeof(int));
  const size_t o_rowinfo = pk.add(t.g_rowinfo.size() * sizeof(int));
  const size_t o_grp = pk.add(t.g_grp.size() * sizeof(int));
  const size_t o_terms = pk.add(t.g_terms.size() * sizeof(GTerm));
  const size_t o_rmap = pk.add(t.rmap.size() * sizeof(int));
  const size_t o_rnorm = pk.add(t.rnorm.size() * sizeof(double));
  const size_t o_rotptr = pk.add(t.rot_ptr.size() * sizeof(int));
  const size_t o_rotterms = pk.add(t.rot_terms.size() * sizeof(GTerm));
  if (pk.used > kNoallocScratchBytes) {
    *err = "constant tables do not fit the static scratch";
    return SHGO_ERR_OOM;
  }
  struct Piece {
    size_t off;
    const void* src;
    size_t bytes;
  } pieces[] = {{o_boys, t.boys.data(), t.boys.size() * sizeof(double)},
                {o_etab, t.etab.data(), t.etab.size() * sizeof(double)},
                {o_eoff, t.eoff.data(), t.eoff.size() * sizeof(int)},
                {o_rowinfo, t.g_rowinfo.data(), t.g_rowinfo.size() * sizeof(int)},
                {o_grp, t.g_grp.data(), t.g_grp.size() * sizeof(int)},
                {o_terms, t.g_terms.data(), t.g_terms.size() * sizeof(GTerm)},
                {o_rmap, t.rmap.data(), t.rmap.size() * sizeof(int)},
                {o_rnorm, t.rnorm.data(), t.rnorm.size() * sizeof(double)},
                {o_rotptr, t.rot_ptr.data(), t.rot_ptr.size() * sizeof(int)},
                {o_rotterms, t.rot_terms.data(), t.rot_terms.size() * sizeof(GTerm)}};
  for (const Piece& p : pieces) {
    e = cudaMemcpy(d.base + p.off, p.src, p.bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      *err = std::string("copying tables into the scratch: ") + cudaGetErrorString(e);
      return SHGO_ERR_CUDA;
    }
  }
  shgo_status st = upload_constants(err);
  if (st != SHGO_OK) return st;
  d.tabs.boys = reinterpret_cast<double*>(d.base + o_boys);
  d.tabs.etab = reinterpret_cast<double*>(d.base + o_etab);
  d.tabs.eoff = reinterpret_cast<int*>(d.base + o_eoff);
  d.tabs.g_rowinfo = reinterpret_cast<int*>(d.base + o_rowinfo);
  d.tabs.g_grp = reinterpret_cast<int*>(d.base + o_grp);
  d.tabs.g_terms = reinterpret_cast<GTerm*>(d.base + o_terms);
  d.tabs.rmap = reinterpret_cast<int*>(d.base + o_rmap);
  d.tabs.rnorm = reinterpret_cast<double*>(d.base + o_rnorm);
  d.tabs.rot_ptr = reinterpret_cast<int*>(d.base + o_rotptr);
  d.tabs.rot_terms = reinterpret_cast<GTerm*>(d.base + o_rotterms);
  d.tables_end = pk.used;
  d.ready = true;
  *out = &d;
  return SHGO_OK;
}

shgo_status noalloc_fail(shgo_status s, const std::string& msg) {
  set_last_error(msg);
  return s;
}

// N(l, alpha) of Eq. 1: N^-2 = pi^{3/2} (2l-1)!! / (2^l (2 alpha)^{l+3/2}).
// The same expressions as the basis build, so both entry points normalise identically.
double noalloc_prim_norm(int l, double alpha) {
  double df = 1;
  for (int k = 2 * l - 1; k > 1; k -= 2) df *= k;
  const double n2 = 5.5683279968317078453 * df / (std::ldexp(1.0, l) * std::pow(2.0 * alpha, l + 1.5));
  return 1.0 / std::sqrt(n2);
}

}  // namespace

extern "C" shgo_status shgo_nuclear_attraction_noalloc(int32_t n_shells, const int32_t* l, const int32_t* n_prim,
                                                       const double* exponents, const double* coefs,
                                                       const double* shell_xyz, const shgo_centers* centers,
                                                       const double* charges, double* out, void* stream) {
  set_last_error("");
  if (n_shells < 0) return noalloc_fail(SHGO_ERR_INVALID_ARG, "n_shells < 0");
  if (n_shells > 0 && (!l || !n_prim || !exponents || !coefs || !shell_xyz))
    return noalloc_fail(SHGO_ERR_INVALID_ARG, "NULL basis array");
  if (!centers || centers->n < 0) return noalloc_fail(SHGO_ERR_INVALID_ARG, "centers is NULL or negative count");
  if (centers->n > 0 && (!centers->xyz || !charges)) return noalloc_fail(SHGO_ERR_INVALID_ARG, "NULL centers/charges");
  int64_t nprim_total = 0, nbf = 0;
  int count_l[kLmax + 1] = {0};
  for (int s = 0; s < n_shells; ++s) {
    if (l[s] < 0) return noalloc_fail(SHGO_ERR_INVALID_ARG, "negative l");
    if (l[s] > kLmax) return noalloc_fail(SHGO_ERR_UNSUPPORTED_L, "l > 8");
    if (n_prim[s] < 1 || n_prim[s] > 64) return noalloc_fail(SHGO_ERR_INVALID_ARG, "n_prim outside 1..64");
    for (int c = 0; c < 3; ++c)
      if (!std::isfinite(shell_xyz[3 * s + c])) return noalloc_fail(SHGO_ERR_INVALID_ARG, "non-finite shell centre");
    nprim_total += n_prim[s];
    nbf += 2 * l[s] + 1;
    ++count_l[l[s]];
  }
  for (int64_t i = 0; i < nprim_total; ++i)
    if (!(exponents[i] > 0) || !std::isfinite(exponents[i]) || !std::isfinite(coefs[i]))
      return noalloc_fail(SHGO_ERR_INVALID_ARG, "exponents must be finite and > 0, coefficients finite");
  if (nbf > 0 && !out) return noalloc_fail(SHGO_ERR_INVALID_ARG, "out is NULL");

  // Scratch needed by this call, before anything is built: shells, pairs, primitive pairs, coupling buffer.
  int64_t npairs = 0, npp = 0, rlen = 0;
  {
    std::vector<int64_t> prim_sum(kLmax + 1, 0);
    for (int s = 0; s < n_shells; ++s) prim_sum[l[s]] += n_prim[s];
    for (int la = 0; la <= kLmax; ++la)
      for (int lb = 0; lb <= la; ++lb) {
        int64_t pairs, pps;
        if (la == lb) {
          pairs = (int64_t)count_l[la] * (count_l[la] + 1) / 2;
          int64_t sq = 0;
          for (int s = 0; s < n_shells; ++s)
            if (l[s] == la) sq += (int64_t)n_prim[s] * n_prim[s];
          pps = (prim_sum[la] * prim_sum[la] + sq) / 2;
        } else {
          pairs = (int64_t)count_l[la] * count_l[lb];
          pps = prim_sum[la] * prim_sum[lb];
        }
        npairs += pairs;
        npp += pps;
        rlen += pps * n_r(la + lb);
      }
  }
  Packer pk;
  const size_t o_xyz = pk.add(sizeof(double) * 3 * (size_t)n_shells);
  const size_t o_l = pk.add(sizeof(int) * (size_t)n_shells);
  const size_t o_np = pk.add(sizeof(int) * (size_t)n_shells);
  const size_t o_poff = pk.add(sizeof(int) * (size_t)n_shells);
  const size_t o_foff = pk.add(sizeof(int64_t) * (size_t)(n_shells + 1));
  const size_t o_exp = pk.add(sizeof(double) * (size_t)nprim_total);
  const size_t o_coef = pk.add(sizeof(double) * (size_t)nprim_total);
  const size_t o_pa = pk.add(sizeof(int) * (size_t)npairs);
  const size_t o_pb = pk.add(sizeof(int) * (size_t)npairs);
  const size_t o_ppoff = pk.add(sizeof(int64_t) * (size_t)npairs);
  const size_t o_srot = pk.add(sizeof(double) * 9 * (size_t)npairs);
  const size_t o_pppair = pk.add(sizeof(int) * (size_t)npp);
  const size_t o_ppij = pk.add(sizeof(int) * (size_t)npp);
  const size_t o_psite = pk.add(sizeof(int) * (size_t)npairs);
  const size_t o_srep = pk.add(sizeof(int) * (size_t)npairs);
  const size_t host_bytes = pk.used;
  // rotation blocks: one per ordered pair of distinct centre positions
  int lmax_b = 0;
  for (int s = 0; s < n_shells; ++s) lmax_b = std::max(lmax_b, (int)l[s]);
  int64_t npos = 0;
  {
    std::unordered_set<std::string> pos;
    for (int s = 0; s < n_shells; ++s) pos.emplace(reinterpret_cast<const char*>(shell_xyz + 3 * s), 3 * sizeof(double));
    npos = (int64_t)pos.size();
  }
  const int64_t rotlen = std::min(npairs, npos * npos) * rot_block(lmax_b);
  const size_t o_ppd = pk.add(sizeof(PPData) * (size_t)npp);
  const size_t o_rotd = pk.add(sizeof(double) * (size_t)rotlen);
  const size_t o_rbuf = pk.add(sizeof(double) * (size_t)rlen);
  const size_t need = pk.used;

  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= 64)
    return noalloc_fail(SHGO_ERR_CUDA, "no current CUDA device");
  NoallocDevice* nd = nullptr;
  std::string err;
  shgo_status st = noalloc_setup(device, &nd, &err);
  if (st != SHGO_OK) return noalloc_fail(st, err);
  if (need > kNoallocScratchBytes - nd->tables_end)
    return noalloc_fail(SHGO_ERR_INVALID_ARG,
                        "problem needs " + std::to_string(need) + " bytes of scratch; the static maximum for "
                        "shells, pairs and coupling buffer is " + std::to_string(kNoallocScratchBytes - nd->tables_end));
  if (nbf == 0) return SHGO_OK;

  // Host image of the shell and pair arrays (same layout and order as shgo_basis_create builds).
  std::vector<unsigned char> img(host_bytes, 0);
  auto put = [&](size_t off, const void* src, size_t bytes) {
    if (bytes) std::memcpy(img.data() + off, src, bytes);
  };
  std::vector<int> poff(n_shells, 0);
  for (int s = 1; s < n_shells; ++s) poff[s] = poff[s - 1] + n_prim[s - 1];
  std::vector<int64_t> foff(n_shells + 1, 0);
  for (int s = 0; s < n_shells; ++s) foff[s + 1] = foff[s] + 2 * l[s] + 1;
  std::vector<double> pcoef(nprim_total);
  for (int s = 0; s < n_shells; ++s) {
    double self = 0;
    for (int i = 0; i < n_prim[s]; ++i)
      for (int j = 0; j < n_prim[s]; ++j) {
        const double ai = exponents[poff[s] + i], aj = exponents[poff[s] + j];
        const double ov = std::pow(2 * std::sqrt(ai * aj) / (ai + aj), l[s] + 1.5);
        self += coefs[poff[s] + i] * coefs[poff[s] + j] * ov;
      }
    if (!(self > 0)) return noalloc_fail(SHGO_ERR_NUMERIC, "a contracted shell has zero norm");
    const double scale = 1.0 / std::sqrt(self);
    for (int i = 0; i < n_prim[s]; ++i)
      pcoef[poff[s] + i] = coefs[poff[s] + i] * noalloc_prim_norm(l[s], exponents[poff[s] + i]) * scale;
  }
  std::vector<std::vector<int>> by_l(kLmax + 1);
  for (int s = 0; s < n_shells; ++s) by_l[l[s]].push_back(s);
  std::vector<int> pa, pb, pp_pair, pp_ij;
  std::vector<int64_t> ppoff;
  pa.reserve(npairs);
  pb.reserve(npairs);
  ppoff.reserve(npairs);
  pp_pair.reserve(npp);
  pp_ij.reserve(npp);
  std::vector<ClassWork> work;
  int64_t ppcount = 0;
  for (int la = 0; la <= kLmax; ++la)
    for (int lb = 0; lb <= la; ++lb) {
      ClassWork w{la, lb, 0, (int)pa.size(), 0, ppcount};
      for (size_t x = 0; x < by_l[la].size(); ++x) {
        const size_t ylim = (la == lb) ? x + 1 : by_l[lb].size();
        for (size_t y = 0; y < ylim; ++y) {
          const int sa = by_l[la][x], sb = by_l[lb][y];
          pa.push_back(sa);
          pb.push_back(sb);
          ppoff.push_back(ppcount);
          for (int i = 0; i < n_prim[sa]; ++i)
            for (int j = 0; j < n_prim[sb]; ++j) {
              pp_pair.push_back((int)pa.size() - 1);
              pp_ij.push_back((i << 8) | j);
            }
          ppcount += (int64_t)n_prim[sa] * n_prim[sb];
          ++w.npairs;
        }
      }
      w.npp = ppcount - w.pp_base;
      if (w.npairs > 0) work.push_back(w);
    }
  put(o_xyz, shell_xyz, sizeof(double) * 3 * (size_t)n_shells);
  put(o_l, l, sizeof(int) * (size_t)n_shells);
  put(o_np, n_prim, sizeof(int) * (size_t)n_shells);
  put(o_poff, poff.data(), sizeof(int) * poff.size());
  put(o_foff, foff.data(), sizeof(int64_t) * foff.size());
  put(o_exp, exponents, sizeof(double) * (size_t)nprim_total);
  put(o_coef, pcoef.data(), sizeof(double) * pcoef.size());
  put(o_pa, pa.data(), sizeof(int) * pa.size());
  put(o_pb, pb.data(), sizeof(int) * pb.size());
  put(o_ppoff, ppoff.data(), sizeof(int64_t) * ppoff.size());
  put(o_pppair, pp_pair.data(), sizeof(int) * pp_pair.size());
  put(o_ppij, pp_ij.data(), sizeof(int) * pp_ij.size());
  std::vector<int> pair_site, site_rep;
  std::vector<double> site_rot;
  build_site_pairs(shell_xyz, pa, pb, pair_site, site_rep, site_rot);
  put(o_psite, pair_site.data(), sizeof(int) * pair_site.size());
  put(o_srep, site_rep.data(), sizeof(int) * site_rep.size());
  put(o_srot, site_rot.data(), sizeof(double) * site_rot.size());

  unsigned char* region = nd->base + nd->tables_end;
  cudaStream_t s = (cudaStream_t)stream;
  // Pageable source: the copy is ordered after earlier work on `stream` and the host image may be
  // released when the call returns.
  cudaError_t e = cudaMemcpyAsync(region, img.data(), host_bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return noalloc_fail(SHGO_ERR_CUDA, std::string("copying the basis: ") + cudaGetErrorString(e));
  DeviceBasis db;
  db.shell_xyz = reinterpret_cast<double*>(region + o_xyz);
  db.shell_l = reinterpret_cast<int*>(region + o_l);
  db.shell_nprim = reinterpret_cast<int*>(region + o_np);
  db.shell_poff = reinterpret_cast<int*>(region + o_poff);
  db.shell_foff = reinterpret_cast<int64_t*>(region + o_foff);
  db.prim_exp = reinterpret_cast<double*>(region + o_exp);
  db.prim_coef = reinterpret_cast<double*>(region + o_coef);
  db.pair_a = reinterpret_cast<int*>(region + o_pa);
  db.pair_b = reinterpret_cast<int*>(region + o_pb);
  db.pair_ppoff = reinterpret_cast<int64_t*>(region + o_ppoff);
  db.site_rot = reinterpret_cast<double*>(region + o_srot);
  db.pp_pair = reinterpret_cast<int*>(region + o_pppair);
  db.pp_ij = reinterpret_cast<int*>(region + o_ppij);
  db.rbuf = reinterpret_cast<double*>(region + o_rbuf);
  db.rbuf_len = rlen;
  db.ppd = reinterpret_cast<PPData*>(region + o_ppd);
  db.rotd = reinterpret_cast<double*>(region + o_rotd);
  db.pair_site = reinterpret_cast<int*>(region + o_psite);
  db.site_rep = reinterpret_cast<int*>(region + o_srep);
  db.n_sites = (int)site_rep.size();
  db.rot_lmax = lmax_b;
  st = launch_pair_build(db, npp, s, &err);
  if (st == SHGO_OK) st = launch_pair_rotations(db, nd->tabs, s, &err);
  if (st != SHGO_OK) return noalloc_fail(st, err);
  st = launch_nuclear_attraction(db, nd->tabs, work, nbf, centers->n, centers->xyz, charges, out, s, &err, nullptr,
                                 /*concurrent=*/false);
  if (st != SHGO_OK) return noalloc_fail(st, err);
  return SHGO_OK;
}
