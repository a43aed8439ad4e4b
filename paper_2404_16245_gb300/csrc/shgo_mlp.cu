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
//
// Tensor cores in a fixed order.  A block is one warp; it takes tiles of 32 samples (tiles b, b + grid, ...)
// and runs every product on mma.sync m16n8k16 (BF16 inputs, FP32 accumulation): the forward layers as in
// inference (activations split into BF16 high and low parts, weights BF16 as used), the backward product
// D2 W2 the same way, and the weight gradients D2^T A1 and D1^T X with both operands split (high x high +
// high x low + low x high: FP32-level accuracy).  The block's gradient and loss accumulate in shared memory
// in tile order and go to the block's slot of `part`; k_mlp_reduce adds the slots in block order.  Every
// sum has a fixed order, so two passes over the same samples give the same bits.
constexpr int kTS = 32;  // samples per tile (one warp)
constexpr int kTrainFloats = kTS * kIn + 4 * kTS * kH + 2 * kTS + kNParam + 2 * kIn + 4;

size_t train_smem() { return sizeof(float) * (size_t)kTrainFloats + sizeof(__nv_bfloat16) * kH * kH; }

// A fragment of rows r0.. and columns c0.. of a row-major FP32 matrix M (row stride ld), split.
__device__ __forceinline__ void load_a_split(const float* M, int ld, int r0, int c0, int g, int t, uint32_t* hi,
                                             uint32_t* lo) {
  const float* p0 = M + (r0 + g) * ld + c0;
  const float* p1 = M + (r0 + g + 8) * ld + c0;
  split2(p0[2 * t], p0[2 * t + 1], hi[0], lo[0]);
  split2(p1[2 * t], p1[2 * t + 1], hi[1], lo[1]);
  split2(p0[2 * t + 8], p0[2 * t + 9], hi[2], lo[2]);
  split2(p1[2 * t + 8], p1[2 * t + 9], hi[3], lo[3]);
}

// A fragment of a transpose, A[m][k] = M[k0 + k][m0 + m] (M row-major, row stride ld), split.
__device__ __forceinline__ void load_at_split(const float* M, int ld, int m0, int k0, int g, int t, uint32_t* hi,
                                              uint32_t* lo) {
  const float* c0 = M + k0 * ld + m0;
  split2(c0[(2 * t) * ld + g], c0[(2 * t + 1) * ld + g], hi[0], lo[0]);
  split2(c0[(2 * t) * ld + g + 8], c0[(2 * t + 1) * ld + g + 8], hi[1], lo[1]);
  split2(c0[(2 * t + 8) * ld + g], c0[(2 * t + 9) * ld + g], hi[2], lo[2]);
  split2(c0[(2 * t + 8) * ld + g + 8], c0[(2 * t + 9) * ld + g + 8], hi[3], lo[3]);
}

// B fragment, B[k][n] = M[k0 + k][n0 + n] (M row-major, row stride ld), split.
__device__ __forceinline__ void load_b_split(const float* M, int ld, int k0, int n0, int g, int t, uint32_t* hi,
                                             uint32_t* lo) {
  const float* c0 = M + k0 * ld + n0 + g;
  split2(c0[(2 * t) * ld], c0[(2 * t + 1) * ld], hi[0], lo[0]);
  split2(c0[(2 * t + 8) * ld], c0[(2 * t + 9) * ld], hi[1], lo[1]);
}

// d += A B with both split: high x high + high x low + low x high.
__device__ __forceinline__ void mma3(float* d, const uint32_t* ah, const uint32_t* al, const uint32_t* bh,
                                     const uint32_t* bl) {
  mma_bf16(d, ah, bh[0], bh[1]);
  mma_bf16(d, ah, bl[0], bl[1]);
  mma_bf16(d, al, bh[0], bh[1]);
}

__global__ void __launch_bounds__(32) k_mlp_train(const float* __restrict__ X, const float* __restrict__ T,
                                                  int64_t n, const __nv_bfloat16* __restrict__ wq,
                                                  const float* __restrict__ norm, float under_weight,
                                                  float* __restrict__ part) {
  extern __shared__ __align__(16) float sm[];
  float* xs = sm;                       // [32][16] standardised inputs
  float* A1 = xs + kTS * kIn;           // [32][64] layer-1 activations
  float* S1 = A1 + kTS * kH;            // [32][64] silu'(z1), then D1 = d loss / d z1
  float* A2 = S1 + kTS * kH;            // [32][64] layer-2 activations
  float* S2 = A2 + kTS * kH;            // [32][64] silu'(z2), then D2 = d loss / d z2
  float* dyv = S2 + kTS * kH;           // [32] d loss / d y
  float* lterm = dyv + kTS;             // [32] loss term w (y - t)^2 of each sample
  float* acc = lterm + kTS;             // [kNParam] this block's gradient
  float* snorm = acc + kNParam;         // mean[16], 1/sd[16]
  float* sloss = snorm + 2 * kIn;       // [1] this block's loss sum
  __nv_bfloat16* w2t = reinterpret_cast<__nv_bfloat16*>(sm + kTrainFloats);  // w2t[k][j] = W2[j][k]
  const int lane = threadIdx.x, g = lane >> 2, t = lane & 3;
  for (int i = lane; i < kNParam; i += 32) acc[i] = 0.f;
  for (int i = lane; i < 2 * kIn; i += 32) snorm[i] = norm[i];
  for (int i = lane; i < kH * kH; i += 32) w2t[(i % kH) * kH + i / kH] = wq[kOffW2 + i];
  if (lane == 0) sloss[0] = 0.f;
  __syncwarp();
  const float inv_n = 1.f / (float)n;
  const int64_t ntiles = (n + kTS - 1) / kTS;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t s0 = tile * kTS;
    {
      const int64_t s = s0 + lane;
#pragma unroll
      for (int k = 0; k < kIn; ++k) xs[lane * kIn + k] = s < n ? (X[s * kIn + k] - snorm[k]) * snorm[kIn + k] : 0.f;
    }
    __syncwarp();
    // forward, two m tiles of 16 samples; z1, z2 kept as activations and SiLU derivatives
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
      const int r0 = 16 * mt;
      uint32_t ah[4], al[4];
      load_a_split(xs, kIn, r0, 0, g, t, ah, al);
      uint32_t h2h[4][4], h2l[4][4];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int j = 8 * nt + g;
        const uint32_t b0 = ldw2(wq, kOffW1 + j * kIn + 2 * t), b1 = ldw2(wq, kOffW1 + j * kIn + 2 * t + 8);
        const float bias0 = __bfloat162float(wq[kOffB1 + 8 * nt + 2 * t]);
        const float bias1 = __bfloat162float(wq[kOffB1 + 8 * nt + 2 * t + 1]);
        float d[4] = {bias0, bias1, bias0, bias1};
        mma_bf16(d, ah, b0, b1);
        mma_bf16(d, al, b0, b1);
        float a[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = r0 + g + (q >> 1) * 8, c = 8 * nt + 2 * t + (q & 1);
          a[q] = silu(d[q]);
          A1[r * kH + c] = a[q];
          S1[r * kH + c] = silu_grad(d[q]);
        }
        const int kk = nt >> 1, half = nt & 1;
        split2(a[0], a[1], h2h[kk][2 * half], h2l[kk][2 * half]);
        split2(a[2], a[3], h2h[kk][2 * half + 1], h2l[kk][2 * half + 1]);
      }
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
        float a[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = r0 + g + (q >> 1) * 8, c = 8 * nt + 2 * t + (q & 1);
          a[q] = silu(d[q]);
          A2[r * kH + c] = a[q];
          S2[r * kH + c] = silu_grad(d[q]);
        }
        const int c = 8 * nt + 2 * t;
        const float w30 = __bfloat162float(wq[kOffW3 + c]), w31 = __bfloat162float(wq[kOffW3 + c + 1]);
        o0 = fmaf(w31, a[1], fmaf(w30, a[0], o0));
        o1 = fmaf(w31, a[3], fmaf(w30, a[2], o1));
      }
      o0 += __shfl_xor_sync(0xffffffffu, o0, 1);
      o0 += __shfl_xor_sync(0xffffffffu, o0, 2);
      o1 += __shfl_xor_sync(0xffffffffu, o1, 1);
      o1 += __shfl_xor_sync(0xffffffffu, o1, 2);
      if (t == 0) {
        const float b3 = __bfloat162float(wq[kOffB3]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = r0 + g + 8 * h;
          const int64_t s = s0 + r;
          float dy = 0.f, lt = 0.f;
          if (s < n) {
            const float res = (h ? o1 : o0) + b3 - T[s];
            const float w = res < 0.f ? under_weight : 1.f;
            lt = w * res * res;
            dy = 2.f * w * res * inv_n;
          }
          dyv[r] = dy;
          lterm[r] = lt;
        }
      }
    }
    __syncwarp();
    // D2 = (dy W3) * silu'(z2), in place of S2
    for (int e = lane; e < kTS * kH; e += 32) {
      const int r = e / kH, j = e % kH;
      S2[e] = dyv[r] * __bfloat162float(wq[kOffW3 + j]) * S2[e];
    }
    __syncwarp();
    // D1 = (D2 W2) * silu'(z1), in place of S1 (each thread rewrites the entries it reads)
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
      const int r0 = 16 * mt;
      uint32_t dh[4][4], dl[4][4];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) load_a_split(S2, kH, r0, 16 * kk, g, t, dh[kk], dl[kk]);
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        const int k = 8 * nt + g;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t b0 = ldw2(w2t, k * kH + 16 * kk + 2 * t), b1 = ldw2(w2t, k * kH + 16 * kk + 2 * t + 8);
          mma_bf16(d, dh[kk], b0, b1);
          mma_bf16(d, dl[kk], b0, b1);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = r0 + g + (q >> 1) * 8, c = 8 * nt + 2 * t + (q & 1);
          S1[r * kH + c] = d[q] * S1[r * kH + c];
        }
      }
    }
    __syncwarp();
    // gW2[j][k] += sum_r D2[r][j] A1[r][k]  and  gW1[j][k] += sum_r D1[r][j] x[r][k]
#pragma unroll 1
    for (int jm = 0; jm < 4; ++jm) {
      uint32_t ah[2][4], al[2][4], eh[2][4], el[2][4];
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        load_at_split(S2, kH, 16 * jm, 16 * ks, g, t, ah[ks], al[ks]);
        load_at_split(S1, kH, 16 * jm, 16 * ks, g, t, eh[ks], el[ks]);
      }
#pragma unroll 1
      for (int nt = 0; nt < 8; ++nt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          uint32_t bh[2], bl[2];
          load_b_split(A1, kH, 16 * ks, 8 * nt, g, t, bh, bl);
          mma3(d, ah[ks], al[ks], bh, bl);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = 16 * jm + g + (q >> 1) * 8, k = 8 * nt + 2 * t + (q & 1);
          acc[kOffW2 + j * kH + k] += d[q];
        }
      }
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          uint32_t bh[2], bl[2];
          load_b_split(xs, kIn, 16 * ks, 8 * nt, g, t, bh, bl);
          mma3(d, eh[ks], el[ks], bh, bl);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = 16 * jm + g + (q >> 1) * 8, k = 8 * nt + 2 * t + (q & 1);
          acc[kOffW1 + j * kIn + k] += d[q];
        }
      }
    }
    // bias and output gradients, summed over the tile's samples in order
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = lane + 32 * h;
      float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f;
      for (int r = 0; r < kTS; ++r) {
        gb1 += S1[r * kH + j];
        gb2 += S2[r * kH + j];
        gw3 = fmaf(dyv[r], A2[r * kH + j], gw3);
      }
      acc[kOffB1 + j] += gb1;
      acc[kOffB2 + j] += gb2;
      acc[kOffW3 + j] += gw3;
    }
    if (lane == 0) {
      float gb3 = 0.f, ls = 0.f;
      for (int r = 0; r < kTS; ++r) {
        gb3 += dyv[r];
        ls += lterm[r];
      }
      acc[kOffB3] += gb3;
      sloss[0] += ls;
    }
    __syncwarp();  // the tile's arrays are free for the next tile
  }
  float* slot = part + (int64_t)blockIdx.x * (kNParam + 1);
  for (int i = lane; i < kNParam; i += 32) slot[i] = acc[i];
  if (lane == 0) slot[kNParam] = sloss[0];
}

// grad[p] = sum over blocks b = 0, 1, ... of part[b][p] (fixed order); loss = sum of the blocks' loss sums / n.
__global__ void k_mlp_reduce(const float* __restrict__ part, int nblocks, float inv_n, float* __restrict__ grad,
                             float* __restrict__ loss) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p <= kNParam; p += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += part[(int64_t)b * (kNParam + 1) + p];
    if (p < kNParam)
      grad[p] = s;
    else
      *loss = s * inv_n;
  }
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
  float* part = nullptr;  // per training block: gradient partial sums and loss sum
  int max_blocks = 0;
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
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, M->device);
  M->max_blocks = 4 * nsm;
  if (e == cudaSuccess) e = cudaMalloc((void**)&M->part, sizeof(float) * (size_t)M->max_blocks * (kNParam + 1));
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
  cudaFree(mlp->part);
  delete mlp;
}

shgo_status shgo_mlp_get_params(const shgo_mlp* mlp, float* params) {
  if (!mlp || !params) return fail_mlp(SHGO_ERR_INVALID_ARG, "NULL argument");
  if (cudaMemcpy(params, mlp->w, sizeof(float) * kNParam, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail_mlp(SHGO_ERR_CUDA, "copy of the parameters failed");
  return SHGO_OK;
}

shgo_status shgo_mlp_get_state(const shgo_mlp* mlp, float* params, float* adam_m, float* adam_v, int64_t* step) {
  if (!mlp || !params || !adam_m || !adam_v || !step) return fail_mlp(SHGO_ERR_INVALID_ARG, "NULL argument");
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(params, mlp->w, sizeof(float) * kNParam, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(adam_m, mlp->m, sizeof(float) * kNParam, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(adam_v, mlp->v, sizeof(float) * kNParam, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail_mlp(SHGO_ERR_CUDA, std::string("saving the state: ") + cudaGetErrorString(e));
  *step = mlp->step;
  return SHGO_OK;
}

shgo_status shgo_mlp_set_state(shgo_mlp* mlp, const float* params, const float* adam_m, const float* adam_v,
                               int64_t step) {
  if (!mlp || !params || !adam_m || !adam_v || step < 0) return fail_mlp(SHGO_ERR_INVALID_ARG, "bad arguments");
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(mlp->w, params, sizeof(float) * kNParam, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(mlp->m, adam_m, sizeof(float) * kNParam, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(mlp->v, adam_v, sizeof(float) * kNParam, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(mlp->g, 0, sizeof(float) * kNParam);
  if (e == cudaSuccess) {
    k_quantize<<<(kNParam + 255) / 256, 256>>>(mlp->w, mlp->wq, kNParam);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) return fail_mlp(SHGO_ERR_CUDA, std::string("restoring the state: ") + cudaGetErrorString(e));
  mlp->step = step;
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

// Gradient (mlp->g) and loss (mlp->loss) of the loss over n samples, in a fixed order: the block count
// depends only on n and the device.
static shgo_status run_train(shgo_mlp* mlp, const float* X, const float* T, int64_t n, float under_weight,
                             cudaStream_t s) {
  const size_t sm = train_smem();
  ensure_max_dynamic_smem((const void*)k_mlp_train, (int)sm);
  const int blocks = (int)std::min<int64_t>((n + kTS - 1) / kTS, (int64_t)mlp->max_blocks);
  k_mlp_train<<<blocks, 32, sm, s>>>(X, T, n, mlp->wq, mlp->norm, under_weight, mlp->part);
  k_mlp_reduce<<<(kNParam + 256) / 256, 256, 0, s>>>(mlp->part, blocks, 1.f / (float)n, mlp->g, mlp->loss);
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
