// The screening network: a 16 -> 64 -> 64 -> 1 multilayer perceptron with SiLU activations that
// predicts log10 max|V block| of one (shell pair, nucleus) triple.  Weights are BF16 in the forward
// pass (rounded from FP32 master weights after every update), all accumulation is FP32.  Training
// (forward, backward, Adam) runs in the kernels below.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "shgo_internal.h"
#include "shgo_mlp.h"

namespace shgo {
void set_last_error(const std::string& msg);  // shgo_api.cpp
}

using namespace shgo;

namespace {

constexpr int kIn = SHGO_MLP_IN, kH = SHGO_MLP_HIDDEN;
// parameter layout (FP32 master / BF16 copy): W1[kH][kIn], b1[kH], W2[kH][kH], b2[kH], W3[kH], b3
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH, kNParam = kOffB3 + 1;
static_assert(kNParam == SHGO_MLP_NPARAM, "parameter count");

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
  const float s = 1.f / (1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

// Weights are staged in shared memory as FP32 values of the BF16 copy.
__device__ void stage_weights(const __nv_bfloat16* __restrict__ wq, const float* __restrict__ bias_src, float* sw) {
  for (int i = threadIdx.x; i < kNParam; i += blockDim.x) sw[i] = __bfloat162float(wq[i]);
  (void)bias_src;
}

// ---------------------------------------------------------------------------------------------
// Tensor-core inference: one warp evaluates 32 samples with mma.sync m16n8k16 (BF16 inputs, FP32
// accumulation).  The weights are BF16 already; each FP32 activation is split into a BF16 high part
// and a BF16 low part (x = hi + lo to about 2^-16 relative) and both are multiplied, so the result
// follows the FP32-activation forward pass to ~1e-5 instead of BF16 rounding of the activations.
// Fragment layout of m16n8k16 (g = lane / 4, t = lane % 4): A rows g and g + 8, columns 2t, 2t + 1
// and 2t + 8, 2t + 9; B columns g, rows 2t, 2t + 1 and 2t + 8, 2t + 9; C/D rows g and g + 8,
// columns 2t, 2t + 1.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo_col, float hi_col) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo_col, hi_col);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// hi/lo BF16 split of two FP32 values (the lower column first).
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const float h0 = __bfloat162float(__float2bfloat16_rn(x0)), h1 = __bfloat162float(__float2bfloat16_rn(x1));
  hi = pack_bf16(h0, h1);
  lo = pack_bf16(x0 - h0, x1 - h1);
}

__device__ __forceinline__ uint32_t ldw2(const __nv_bfloat16* w, int i) {  // i even
  return *reinterpret_cast<const uint32_t*>(w + i);
}

// Outputs of 32 standardised samples xs[32][kIn] (shared, this warp's) into ys[32] (shared).
// Every lane of the warp must call it.
__device__ void mlp_eval_warp(const __nv_bfloat16* __restrict__ wq, const float* xs, float* ys) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float out[2][2];  // [m tile][row g, g + 8] partial sums over this thread's columns
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    // layer 1: A = x (16 samples x 16 features), one k step
    const float* r0 = xs + (16 * mt + g) * kIn;
    const float* r1 = xs + (16 * mt + g + 8) * kIn;
    uint32_t ah[4], al[4];
    split2(r0[2 * t], r0[2 * t + 1], ah[0], al[0]);
    split2(r1[2 * t], r1[2 * t + 1], ah[1], al[1]);
    split2(r0[2 * t + 8], r0[2 * t + 9], ah[2], al[2]);
    split2(r1[2 * t + 8], r1[2 * t + 9], ah[3], al[3]);
    // hidden layer 1 (64 = 8 n tiles), SiLU, then split into the A fragments of layer 2
    uint32_t h2h[4][4], h2l[4][4];  // [k step][fragment register]
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int j = 8 * nt + g;  // output unit held as B column
      const uint32_t b0 = ldw2(wq, kOffW1 + j * kIn + 2 * t), b1 = ldw2(wq, kOffW1 + j * kIn + 2 * t + 8);
      const float bias0 = __bfloat162float(wq[kOffB1 + 8 * nt + 2 * t]);
      const float bias1 = __bfloat162float(wq[kOffB1 + 8 * nt + 2 * t + 1]);
      float d[4] = {bias0, bias1, bias0, bias1};
      mma_bf16(d, ah, b0, b1);
      mma_bf16(d, al, b0, b1);
      // D tile nt covers hidden units 8 nt .. 8 nt + 7 = columns of k step nt / 2
      const int kk = nt >> 1, half = nt & 1;
      split2(silu(d[0]), silu(d[1]), h2h[kk][2 * half], h2l[kk][2 * half]);
      split2(silu(d[2]), silu(d[3]), h2h[kk][2 * half + 1], h2l[kk][2 * half + 1]);
    }
    // hidden layer 2 and the output unit
    float o0 = 0.f, o1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int j = 8 * nt + g;
      const float bias0 = __bfloat162float(wq[kOffB2 + 8 * nt + 2 * t]);
      const float bias1 = __bfloat162float(wq[kOffB2 + 8 * nt + 2 * t + 1]);
      float d[4] = {bias0, bias1, bias0, bias1};
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t b0 = ldw2(wq, kOffW2 + j * kH + 16 * kk + 2 * t);
        const uint32_t b1 = ldw2(wq, kOffW2 + j * kH + 16 * kk + 2 * t + 8);
        mma_bf16(d, h2h[kk], b0, b1);
        mma_bf16(d, h2l[kk], b0, b1);
      }
      const float w30 = __bfloat162float(wq[kOffW3 + 8 * nt + 2 * t]);
      const float w31 = __bfloat162float(wq[kOffW3 + 8 * nt + 2 * t + 1]);
      o0 = fmaf(w31, silu(d[1]), fmaf(w30, silu(d[0]), o0));
      o1 = fmaf(w31, silu(d[3]), fmaf(w30, silu(d[2]), o1));
    }
    out[mt][0] = o0;
    out[mt][1] = o1;
  }
  // sum the four threads of each row
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float v = out[mt][h];
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      out[mt][h] = v;
    }
  if (t == 0) {
    const float b3 = __bfloat162float(wq[kOffB3]);
    ys[g] = out[0][0] + b3;
    ys[g + 8] = out[0][1] + b3;
    ys[16 + g] = out[1][0] + b3;
    ys[24 + g] = out[1][1] + b3;
  }
  __syncwarp();
}

// Inference: one warp per 32 samples on the tensor cores.
__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ X, int64_t n,
                                                     const __nv_bfloat16* __restrict__ wq,
                                                     const float* __restrict__ norm,  // mean[16], 1/sd[16]
                                                     float* __restrict__ y) {
  __shared__ float sxs[4][32 * kIn];
  __shared__ float sys[4][32];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int64_t warp = blockIdx.x * 4ll + wi, nwarps = (int64_t)gridDim.x * 4;
  for (int64_t base = warp * 32; base < n; base += nwarps * 32) {
    const int64_t s = base + lane;
#pragma unroll
    for (int k = 0; k < kIn; ++k) sxs[wi][lane * kIn + k] = s < n ? (X[s * kIn + k] - norm[k]) * norm[kIn + k] : 0.f;
    __syncwarp();
    mlp_eval_warp(wq, sxs[wi], sys[wi]);
    if (s < n) y[s] = sys[wi][lane];
    __syncwarp();
  }
}

// One training pass over n samples: loss = sum_s w_s (y_s - t_s)^2 / n with w_s = under_weight when
// the prediction is below the target (under-prediction is what causes false skips), 1 otherwise.
// Gradients are accumulated into grad (FP32, zeroed by the caller); the loss sum into loss[0].
constexpr int kTB = 64;  // samples (threads) per block
__global__ void __launch_bounds__(kTB) k_mlp_train(const float* __restrict__ X, const float* __restrict__ T,
                                                   int64_t n, const __nv_bfloat16* __restrict__ wq,
                                                   const float* __restrict__ norm, float under_weight,
                                                   float* __restrict__ grad, float* __restrict__ loss) {
  extern __shared__ float sm[];
  float* sw = sm;                       // kNParam
  float* snorm = sw + kNParam;          // 2 kIn
  float* sx = snorm + 2 * kIn;          // [kTB][kIn] normalised inputs
  float* sa1 = sx + kTB * kIn;          // [kTB][kH] layer-1 activations
  float* sd1 = sa1 + kTB * kH;          // [kTB][kH] d loss / d z1
  float* sa2 = sd1 + kTB * kH;          // [kTB][kH] layer-2 activations
  float* sd2 = sa2 + kTB * kH;          // [kTB][kH] d loss / d z2
  float* sdy = sd2 + kTB * kH;          // [kTB]
  stage_weights(wq, nullptr, sw);
  for (int i = threadIdx.x; i < 2 * kIn; i += blockDim.x) snorm[i] = norm[i];
  __syncthreads();
  const float inv_n = 1.f / (float)n;
  float block_loss = 0.f;
  for (int64_t base = blockIdx.x * (int64_t)kTB; base < n; base += (int64_t)gridDim.x * kTB) {
    const int t = threadIdx.x;
    const int64_t s = base + t;
    const bool live = s < n;
    // forward with saved activations
    float z1[kH];
    for (int k = 0; k < kIn; ++k) sx[t * kIn + k] = live ? (X[s * kIn + k] - snorm[k]) * snorm[kIn + k] : 0.f;
    for (int j = 0; j < kH; ++j) {
      float z = sw[kOffB1 + j];
      for (int k = 0; k < kIn; ++k) z = fmaf(sw[kOffW1 + j * kIn + k], sx[t * kIn + k], z);
      z1[j] = z;
      sa1[t * kH + j] = silu(z);
    }
    float out = sw[kOffB3];
    for (int j = 0; j < kH; ++j) {
      float z = sw[kOffB2 + j];
      for (int k = 0; k < kH; ++k) z = fmaf(sw[kOffW2 + j * kH + k], sa1[t * kH + k], z);
      sa2[t * kH + j] = silu(z);
      sd2[t * kH + j] = z;  // z2 for now
      out = fmaf(sw[kOffW3 + j], sa2[t * kH + j], out);
    }
    float dy = 0.f;
    if (live) {
      const float r = out - T[s];
      const float w = r < 0.f ? under_weight : 1.f;
      block_loss += w * r * r;
      dy = 2.f * w * r * inv_n;
    }
    sdy[t] = dy;
    // backward through the per-sample activations
    for (int j = 0; j < kH; ++j) sd2[t * kH + j] = dy * sw[kOffW3 + j] * silu_grad(sd2[t * kH + j]);
    for (int k = 0; k < kH; ++k) {
      float acc = 0.f;
      for (int j = 0; j < kH; ++j) acc = fmaf(sw[kOffW2 + j * kH + k], sd2[t * kH + j], acc);
      sd1[t * kH + k] = acc * silu_grad(z1[k]);
    }
    __syncthreads();
    // weight gradients: sums over this block's samples, one parameter slice per thread
    for (int p = threadIdx.x; p < kNParam; p += blockDim.x) {
      float g = 0.f;
      if (p < kOffB1) {
        const int j = p / kIn, k = p % kIn;
        for (int u = 0; u < kTB; ++u) g = fmaf(sd1[u * kH + j], sx[u * kIn + k], g);
      } else if (p < kOffW2) {
        const int j = p - kOffB1;
        for (int u = 0; u < kTB; ++u) g += sd1[u * kH + j];
      } else if (p < kOffB2) {
        const int q = p - kOffW2, j = q / kH, k = q % kH;
        for (int u = 0; u < kTB; ++u) g = fmaf(sd2[u * kH + j], sa1[u * kH + k], g);
      } else if (p < kOffW3) {
        const int j = p - kOffB2;
        for (int u = 0; u < kTB; ++u) g += sd2[u * kH + j];
      } else if (p < kOffB3) {
        const int j = p - kOffW3;
        for (int u = 0; u < kTB; ++u) g = fmaf(sdy[u], sa2[u * kH + j], g);
      } else {
        for (int u = 0; u < kTB; ++u) g += sdy[u];
      }
      if (g != 0.f) atomicAdd(grad + p, g);
    }
    __syncthreads();
  }
  // block loss
  __shared__ float red[kTB];
  red[threadIdx.x] = block_loss;
  __syncthreads();
  for (int o = kTB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] * inv_n);
}

// Adam on the FP32 master weights, then the BF16 copy; clears the gradient.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       __nv_bfloat16* __restrict__ wq, int np, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    w[i] = wi;
    wq[i] = __float2bfloat16_rn(wi);
    g[i] = 0.f;
  }
}

__global__ void k_quantize(const float* __restrict__ w, __nv_bfloat16* __restrict__ wq, int np) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x)
    wq[i] = __float2bfloat16_rn(w[i]);
}

size_t train_smem() { return sizeof(float) * (kNParam + 2 * kIn + kTB * kIn + 4 * kTB * kH + kTB); }

shgo_status fail_mlp(shgo_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

// ---------------------------------------------------------------------------------------------
// Features of (shell pair, nucleus) triples.  Pair-level quantities first (once per pair in the
// screening kernel), then the nucleus-dependent ones; training and screening call the same code.
// ---------------------------------------------------------------------------------------------
struct PairFeat {
  float f[16];                 // pair-level entries filled, nucleus-level ones set by nucleus_features
  double Pmin[3], pmin, A[3], B[3];
};

// lane / nlanes split the primitive-pair sum of the overlap scale over the lanes of a warp
// (nlanes = 32: every lane of the warp must call, and all receive the full sum).
__device__ void pair_features(const ScreenBasis& sb, int pr, PairFeat& pf, int lane = 0, int nlanes = 1) {
  const int a = sb.pair_a[pr], b = sb.pair_b[pr];
  const int la = sb.shell_l[a], lb = sb.shell_l[b];
  const int pa = sb.shell_poff[a], pb = sb.shell_poff[b], na = sb.shell_nprim[a], nb = sb.shell_nprim[b];
  double amin = 1e300, amax = 0, bmin = 1e300, bmax = 0, ca = 0, cb = 0;
  for (int i = 0; i < na; ++i) {
    amin = fmin(amin, sb.prim_exp[pa + i]);
    amax = fmax(amax, sb.prim_exp[pa + i]);
    ca += fabs(sb.prim_coef[pa + i]);
  }
  for (int j = 0; j < nb; ++j) {
    bmin = fmin(bmin, sb.prim_exp[pb + j]);
    bmax = fmax(bmax, sb.prim_exp[pb + j]);
    cb += fabs(sb.prim_coef[pb + j]);
  }
  double ab2 = 0;
  for (int c = 0; c < 3; ++c) {
    pf.A[c] = sb.shell_xyz[3 * a + c];
    pf.B[c] = sb.shell_xyz[3 * b + c];
    ab2 += (pf.B[c] - pf.A[c]) * (pf.B[c] - pf.A[c]);
  }
  double ovl = 0;
  for (int ij = lane; ij < na * nb; ij += nlanes) {
    const int i = ij / nb, j = ij - (ij / nb) * nb;
    const double ea = sb.prim_exp[pa + i], eb = sb.prim_exp[pb + j], p = ea + eb;
    const double sp = 3.14159265358979323846 / p;
    ovl += fabs(sb.prim_coef[pa + i] * sb.prim_coef[pb + j]) * exp(-ea * eb / p * ab2) * sp * sqrt(sp);
  }
  if (nlanes == 32)
    for (int o = 16; o > 0; o >>= 1) ovl += __shfl_xor_sync(0xffffffffu, ovl, o);
  const double pmin = amin + bmin;
  pf.pmin = pmin;
  for (int c = 0; c < 3; ++c) pf.Pmin[c] = (amin * pf.A[c] + bmin * pf.B[c]) / pmin;
  pf.f[0] = (float)la;
  pf.f[1] = (float)lb;
  pf.f[2] = (float)log10(amin);
  pf.f[3] = (float)log10(bmin);
  pf.f[4] = (float)log10(amax);
  pf.f[5] = (float)log10(bmax);
  pf.f[6] = (float)sqrt(ab2);
  pf.f[7] = (float)(-amin * bmin / pmin * ab2 * 0.43429448190325182765);
  pf.f[11] = (float)log10(ca + 1e-300);
  pf.f[12] = (float)log10(cb + 1e-300);
  pf.f[15] = (float)log10(ovl + 1e-300);
}

// Nucleus-dependent features in FP32 (only the coordinate differences are formed in FP64): they
// are network inputs, and FP64 square roots and logarithms are costly on GB300 (sm_103a).
__device__ void nucleus_features(const PairFeat& pf, const double* C, double Z, float* x) {
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = pf.f[k];
  float pc2 = 0.f, ac2 = 0.f, bc2 = 0.f;
  for (int c = 0; c < 3; ++c) {
    const float dp = (float)(pf.Pmin[c] - C[c]), da = (float)(pf.A[c] - C[c]), db = (float)(pf.B[c] - C[c]);
    pc2 = fmaf(dp, dp, pc2);
    ac2 = fmaf(da, da, ac2);
    bc2 = fmaf(db, db, bc2);
  }
  x[8] = sqrtf(pc2);
  x[9] = log10f(fmaf((float)pf.pmin, pc2, 1.f));
  x[10] = log10f(fmaxf((float)Z, 1e-30f));
  x[13] = sqrtf(ac2);
  x[14] = sqrtf(bc2);
}

__global__ void k_screen_features(ScreenBasis sb, const double* __restrict__ centers,
                                  const double* __restrict__ charges, const int* __restrict__ triples, int64_t n,
                                  float* __restrict__ X) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int pr = triples[2 * t], c = triples[2 * t + 1];
    PairFeat pf;
    pair_features(sb, pr, pf);
    float x[16];
    nucleus_features(pf, centers + 3 * (int64_t)c, charges[c], x);
    for (int k = 0; k < 16; ++k) X[t * 16 + k] = x[k];
  }
}

// One warp per shell pair: predict every nucleus of the pair's molecule.  Pass 0 writes the keep
// mask (1 byte per triple) and the kept count of the pair; pass 1 writes the kept nucleus indices
// in order at the pair's offset.
__global__ void __launch_bounds__(128) k_screen_pairs(ScreenBasis sb, int64_t npairs, const double* __restrict__ centers,
                                                     const double* __restrict__ charges,
                                                     const __nv_bfloat16* __restrict__ wq,
                                                     const float* __restrict__ norm, float cut, int pass,
                                                     uint8_t* __restrict__ mask, int64_t* __restrict__ counts,
                                                     int* __restrict__ clist) {
  __shared__ float snorm[2 * kIn];
  __shared__ float sxs[4][32 * kIn];
  __shared__ float sys[4][32];
  if (pass == 0) {
    for (int i = threadIdx.x; i < 2 * kIn; i += blockDim.x) snorm[i] = norm[i];
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int64_t warp = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t pr = warp; pr < npairs; pr += nwarps) {
    int64_t c0, nc;
    if (sb.pair_mol) {
      const int m = sb.pair_mol[pr];
      c0 = sb.mol_c0[m];
      nc = sb.mol_nc[m];
    } else {
      c0 = 0;
      nc = sb.ncenters;
    }
    const int64_t moff = sb.mask_off[pr];
    if (pass == 0) {
      PairFeat pf;
      pair_features(sb, (int)pr, pf, lane, 32);
      int64_t kept = 0;
      for (int64_t k0 = 0; k0 < nc; k0 += 32) {
        const int64_t k = k0 + lane;
        float x[16];
        if (k < nc) {
          nucleus_features(pf, centers + 3 * (c0 + k), charges[c0 + k], x);
#pragma unroll
          for (int q = 0; q < kIn; ++q) x[q] = (x[q] - snorm[q]) * snorm[kIn + q];
        } else {
#pragma unroll
          for (int q = 0; q < kIn; ++q) x[q] = 0.f;
        }
#pragma unroll
        for (int q = 0; q < kIn; ++q) sxs[wi][lane * kIn + q] = x[q];
        __syncwarp();
        mlp_eval_warp(wq, sxs[wi], sys[wi]);  // all lanes
        const bool keep = k < nc && sys[wi][lane] >= cut;
        if (k < nc) mask[moff + k] = keep ? 1 : 0;
        kept += __popc(__ballot_sync(0xffffffffu, keep));
        __syncwarp();
      }
      if (lane == 0) counts[pr] = kept;
    } else {
      int64_t w = sb.clist_off[pr];
      for (int64_t k0 = 0; k0 < nc; k0 += 32) {
        const int64_t k = k0 + lane;
        const bool keep = k < nc && mask[moff + k];
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) clist[w + __popc(bal & ((1u << lane) - 1u))] = (int)(c0 + k);
        w += __popc(bal);
      }
    }
  }
}

}  // namespace

namespace shgo {
shgo_status launch_screen_features(const ScreenBasis& sb, const double* centers, const double* charges,
                                   const int* triples, int64_t n, float* X, cudaStream_t s) {
  if (n == 0) return SHGO_OK;
  const int64_t blocks = std::min<int64_t>((n + 127) / 128, 152 * 16);
  k_screen_features<<<(int)blocks, 128, 0, s>>>(sb, centers, charges, triples, n, X);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SHGO_OK : fail_mlp(SHGO_ERR_CUDA, cudaGetErrorString(e));
}

shgo_status launch_screen_pairs(const ScreenBasis& sb, int64_t npairs, const double* centers, const double* charges,
                                const shgo_mlp* mlp, float cut, int pass, uint8_t* mask, int64_t* counts,
                                int* clist, cudaStream_t s);
}  // namespace shgo

struct shgo_mlp {
  int device = 0;
  float* w = nullptr;  // FP32 master
  float* g = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* norm = nullptr;  // mean[16], 1/sd[16]
  float* loss = nullptr;
  __nv_bfloat16* wq = nullptr;
  int64_t step = 0;
};

extern "C" {

shgo_status shgo_mlp_create(const float* params, const float* feature_mean, const float* feature_sd,
                            shgo_mlp** out) {
  if (!out || !params || !feature_mean || !feature_sd) return fail_mlp(SHGO_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  auto* M = new shgo_mlp();
  cudaGetDevice(&M->device);
  cudaError_t e = cudaSuccess;
  float** bufs[] = {&M->w, &M->g, &M->m, &M->v};
  for (float** b : bufs)
    if (e == cudaSuccess) e = cudaMalloc((void**)b, sizeof(float) * kNParam);
  if (e == cudaSuccess) e = cudaMalloc((void**)&M->norm, sizeof(float) * 2 * kIn);
  if (e == cudaSuccess) e = cudaMalloc((void**)&M->loss, sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&M->wq, sizeof(__nv_bfloat16) * kNParam);
  std::vector<float> nrm(2 * kIn);
  for (int k = 0; k < kIn; ++k) {
    if (!(feature_sd[k] > 0.f)) e = e == cudaSuccess ? cudaErrorInvalidValue : e;
    nrm[k] = feature_mean[k];
    nrm[kIn + k] = feature_sd[k] > 0.f ? 1.f / feature_sd[k] : 0.f;
  }
  if (e == cudaSuccess) e = cudaMemcpy(M->w, params, sizeof(float) * kNParam, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(M->norm, nrm.data(), sizeof(float) * 2 * kIn, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(M->g, 0, sizeof(float) * kNParam);
  if (e == cudaSuccess) e = cudaMemset(M->m, 0, sizeof(float) * kNParam);
  if (e == cudaSuccess) e = cudaMemset(M->v, 0, sizeof(float) * kNParam);
  if (e == cudaSuccess) {
    k_quantize<<<(kNParam + 255) / 256, 256>>>(M->w, M->wq, kNParam);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    shgo_mlp_free(M);
    return fail_mlp(e == cudaErrorInvalidValue ? SHGO_ERR_INVALID_ARG : SHGO_ERR_CUDA,
                    std::string("mlp create: ") + cudaGetErrorString(e));
  }
  *out = M;
  return SHGO_OK;
}

void shgo_mlp_free(shgo_mlp* mlp) {
  if (!mlp) return;
  cudaDeviceSynchronize();
  cudaFree(mlp->w);
  cudaFree(mlp->g);
  cudaFree(mlp->m);
  cudaFree(mlp->v);
  cudaFree(mlp->norm);
  cudaFree(mlp->loss);
  cudaFree(mlp->wq);
  delete mlp;
}

shgo_status shgo_mlp_get_params(const shgo_mlp* mlp, float* params) {
  if (!mlp || !params) return fail_mlp(SHGO_ERR_INVALID_ARG, "NULL argument");
  if (cudaMemcpy(params, mlp->w, sizeof(float) * kNParam, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail_mlp(SHGO_ERR_CUDA, "copy of the parameters failed");
  return SHGO_OK;
}

shgo_status shgo_mlp_forward(const shgo_mlp* mlp, const float* X, int64_t n, float* y, void* stream) {
  if (!mlp || n < 0 || (n > 0 && (!X || !y))) return fail_mlp(SHGO_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return SHGO_OK;
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, mlp->device);
  const int64_t blocks = std::min<int64_t>((n + 127) / 128, (int64_t)nsm * 8);
  k_mlp_forward<<<(int)blocks, 128, 0, (cudaStream_t)stream>>>(X, n, mlp->wq, mlp->norm, y);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SHGO_OK : fail_mlp(SHGO_ERR_CUDA, cudaGetErrorString(e));
}

static shgo_status run_train(shgo_mlp* mlp, const float* X, const float* T, int64_t n, float under_weight,
                             cudaStream_t s) {
  const size_t sm = train_smem();
  ensure_max_dynamic_smem((const void*)k_mlp_train, (int)sm);
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, mlp->device);
  const int64_t blocks = std::min<int64_t>((n + kTB - 1) / kTB, (int64_t)nsm * 2);
  cudaMemsetAsync(mlp->loss, 0, sizeof(float), s);
  k_mlp_train<<<(int)blocks, kTB, sm, s>>>(X, T, n, mlp->wq, mlp->norm, under_weight, mlp->g, mlp->loss);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SHGO_OK : fail_mlp(SHGO_ERR_CUDA, cudaGetErrorString(e));
}

shgo_status shgo_mlp_gradients(shgo_mlp* mlp, const float* X, const float* T, int64_t n, float under_weight,
                               float* grad, float* loss) {
  if (!mlp || n <= 0 || !X || !T || !grad || !loss) return fail_mlp(SHGO_ERR_INVALID_ARG, "bad arguments");
  cudaMemset(mlp->g, 0, sizeof(float) * kNParam);
  shgo_status st = run_train(mlp, X, T, n, under_weight, 0);
  if (st != SHGO_OK) return st;
  if (cudaMemcpy(grad, mlp->g, sizeof(float) * kNParam, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(loss, mlp->loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail_mlp(SHGO_ERR_CUDA, "copy of the gradients failed");
  cudaMemset(mlp->g, 0, sizeof(float) * kNParam);
  return SHGO_OK;
}

shgo_status shgo_mlp_train_step(shgo_mlp* mlp, const float* X, const float* T, int64_t n, float under_weight,
                                float lr, float* loss, void* stream) {
  if (!mlp || n <= 0 || !X || !T) return fail_mlp(SHGO_ERR_INVALID_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  shgo_status st = run_train(mlp, X, T, n, under_weight, s);
  if (st != SHGO_OK) return st;
  mlp->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f / (1.f - std::pow(b1, (float)mlp->step));
  const float c2 = 1.f / (1.f - std::pow(b2, (float)mlp->step));
  k_adam<<<(kNParam + 255) / 256, 256, 0, s>>>(mlp->w, mlp->g, mlp->m, mlp->v, mlp->wq, kNParam, lr, b1, b2, 1e-8f,
                                               c1, c2);
  if (loss) {
    if (cudaMemcpyAsync(loss, mlp->loss, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail_mlp(SHGO_ERR_CUDA, "loss copy failed");
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SHGO_OK : fail_mlp(SHGO_ERR_CUDA, cudaGetErrorString(e));
}

}  // extern "C"

namespace shgo {
shgo_status launch_screen_pairs(const ScreenBasis& sb, int64_t npairs, const double* centers, const double* charges,
                                const shgo_mlp* mlp, float cut, int pass, uint8_t* mask, int64_t* counts,
                                int* clist, cudaStream_t s) {
  if (npairs == 0) return SHGO_OK;
  const int64_t blocks = std::min<int64_t>((npairs + 3) / 4, 152 * 8);
  k_screen_pairs<<<(int)blocks, 128, 0, s>>>(sb, npairs, centers, charges, mlp->wq, mlp->norm, cut, pass, mask,
                                              counts, clist);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SHGO_OK : fail_mlp(SHGO_ERR_CUDA, cudaGetErrorString(e));
}
}  // namespace shgo
