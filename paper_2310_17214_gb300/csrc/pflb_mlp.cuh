// pflb_mlp.cuh -- the chemistry-surrogate MLP on tensor cores (sm_103a).
//
// Network 8 -> 64 -> 64 -> 64 -> 6, tanh hidden layers, linear output; BF16
// weights and activations as tensor-core operands, FP32 accumulation
// (mma.sync m16n8k16).  A warp carries 16 samples: the FP32 accumulator
// fragments of one layer are repacked in registers as the BF16 A fragments of
// the next layer.  Training keeps FP32 master weights; the backward pass
// computes dX = dZ W^T on tensor cores in the same register scheme and
// dW = X^T dZ on tensor cores from warp-staged BF16 copies.
//
// Parameter order (flat FP32): W1 (8x64, input-major), b1, W2, b2, W3, b3,
// W4 (64x6), b4 -- y = x W + b per layer.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace pflb {
namespace mlp {

constexpr int NL = 4;
__host__ __device__ constexpr int dim(int i) { return i == 0 ? 8 : (i == 4 ? 6 : 64); }
__host__ __device__ constexpr int pdim(int i) { return i == 0 ? 16 : (i == 4 ? 8 : 64); }
__host__ __device__ constexpr int woff(int l) {  // offset of W_l in the flat vector
  return l == 0 ? 0 : woff(l - 1) + dim(l - 1) * dim(l) + dim(l);
}
__host__ __device__ constexpr int boff(int l) { return woff(l) + dim(l) * dim(l + 1); }
constexpr int NPARAM = woff(NL);  // 9286
// padded BF16 weight tiles, one layout per direction
__host__ __device__ constexpr int poff(int l) {
  return l == 0 ? 0 : poff(l - 1) + pdim(l - 1) * pdim(l);
}
constexpr int NPAD = poff(NL);  // 9728
__host__ __device__ constexpr int pboff(int l) { return l == 0 ? 0 : pboff(l - 1) + pdim(l); }
constexpr int NPB = pboff(NL);  // 200 padded biases

// Device-side network: BF16 weights in the forward layout and the backward
// layout [in][out] (padded), FP32 biases (padded).  The forward layout is the
// order in which the tensor cores take B fragments: for layer l, n-tile j
// (8 outputs) and k-tile kk (16 inputs), 32 lanes x 4 values, lane (g, t)
// holding W[k][n] for n = 8 j + g and k = 16 kk + 2 t + {0, 1, 8, 9}; one
// 8-byte shared-memory load per lane and fragment, free of bank conflicts.
struct Net {
  const __nv_bfloat16* wf;  // NPAD
  const __nv_bfloat16* wb;  // NPAD
  const float* bias;        // NPB
  const float* theta;       // NPARAM FP32 master parameters (flat order above)
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float fast_tanh(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Shared-memory copy of the network for training (weights in both layouts).
struct SmemNet {
  __nv_bfloat16 wf[NPAD];
  __nv_bfloat16 wb[NPAD];
  float bias[NPB];
};
// Shared-memory copy for inference (forward layout only).
struct __align__(16) SmemFwd {
  __nv_bfloat16 wf[NPAD];
  float bias[NPB];
};
static_assert(NPAD * 2 % 16 == 0 && NPB * 4 % 16 == 0, "16-byte copies of the network");

__device__ __forceinline__ void load_words(uint32_t* dst, const uint32_t* src, int words) {
  for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
}
__device__ __forceinline__ void load_net(SmemNet& s, const Net& n) {
  load_words(reinterpret_cast<uint32_t*>(s.wf), reinterpret_cast<const uint32_t*>(n.wf), NPAD / 2);
  load_words(reinterpret_cast<uint32_t*>(s.wb), reinterpret_cast<const uint32_t*>(n.wb), NPAD / 2);
  load_words(reinterpret_cast<uint32_t*>(s.bias), reinterpret_cast<const uint32_t*>(n.bias), NPB);
}
// 16-byte copy of NV vectors by a block of BT threads, every load issued
// before the first store (a block loads the network once; a copy that waits
// on each load in turn costs microseconds per block)
template <int NV, int BT>
__device__ __forceinline__ void load_vec16(uint4* dst, const uint4* __restrict__ src) {
  constexpr int R = (NV + BT - 1) / BT;
  uint4 v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = threadIdx.x + r * BT;
    if (i < NV) v[r] = __ldg(src + i);
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = threadIdx.x + r * BT;
    if (i < NV) dst[i] = v[r];
  }
}
template <int BT = 256>
__device__ __forceinline__ void load_fwd(SmemFwd& s, const Net& n) {
  load_vec16<NPAD * 2 / 16, BT>(reinterpret_cast<uint4*>(s.wf), reinterpret_cast<const uint4*>(n.wf));
  load_vec16<NPB * 4 / 16, BT>(reinterpret_cast<uint4*>(s.bias),
                               reinterpret_cast<const uint4*>(n.bias));
}

// B fragment (b0, b1) of layer L, n-tile j, k-tile kk for this lane.
template <int L>
__device__ __forceinline__ uint2 b_frag(const __nv_bfloat16* wf, int j, int kk) {
  constexpr int KT = pdim(L) / 16;
  const int lane = threadIdx.x & 31;
  return *reinterpret_cast<const uint2*>(wf + poff(L) + ((j * KT + kk) * 32 + lane) * 4);
}

// One dense layer for 16 rows: acc[j] (n-tile j) = A x W + b.  `a` holds the
// A fragments of the layer input, k-tile kk at a[4 kk .. 4 kk + 3].
template <int L>
__device__ __forceinline__ void layer_fwd(const __nv_bfloat16* wf, const float* bias,
                                          const uint32_t* a, float acc[][4]) {
  constexpr int IN = pdim(L), OUT = pdim(L + 1);
  const int t = threadIdx.x & 3;
  const float* b = bias + pboff(L);
#pragma unroll
  for (int j = 0; j < OUT / 8; ++j) {
    acc[j][0] = acc[j][2] = b[8 * j + 2 * t];
    acc[j][1] = acc[j][3] = b[8 * j + 2 * t + 1];
#pragma unroll
    for (int kk = 0; kk < IN / 16; ++kk) {
      const uint2 w = b_frag<L>(wf, j, kk);
      mma16816(acc[j], a + 4 * kk, w.x, w.y);
    }
  }
}

// The same for two 16-row tiles sharing each B fragment.
template <int L>
__device__ __forceinline__ void layer_fwd2(const __nv_bfloat16* wf, const float* bias,
                                           const uint32_t* a0, const uint32_t* a1,
                                           float acc0[][4], float acc1[][4]) {
  constexpr int IN = pdim(L), OUT = pdim(L + 1);
  const int t = threadIdx.x & 3;
  const float* b = bias + pboff(L);
#pragma unroll
  for (int j = 0; j < OUT / 8; ++j) {
    acc0[j][0] = acc0[j][2] = acc1[j][0] = acc1[j][2] = b[8 * j + 2 * t];
    acc0[j][1] = acc0[j][3] = acc1[j][1] = acc1[j][3] = b[8 * j + 2 * t + 1];
#pragma unroll
    for (int kk = 0; kk < IN / 16; ++kk) {
      const uint2 w = b_frag<L>(wf, j, kk);
      mma16816(acc0[j], a0 + 4 * kk, w.x, w.y);
      mma16816(acc1[j], a1 + 4 * kk, w.x, w.y);
    }
  }
}

// Accumulator fragments (16 x 64, 8 n-tiles) -> A fragments (4 k-tiles), with
// an optional tanh.
template <bool TANH>
__device__ __forceinline__ void to_a(float acc[8][4], uint32_t* a) {
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (TANH) acc[j][e] = fast_tanh(acc[j][e]);
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    a[4 * kk + 0] = pack_bf16(acc[2 * kk][0], acc[2 * kk][1]);
    a[4 * kk + 1] = pack_bf16(acc[2 * kk][2], acc[2 * kk][3]);
    a[4 * kk + 2] = pack_bf16(acc[2 * kk + 1][0], acc[2 * kk + 1][1]);
    a[4 * kk + 3] = pack_bf16(acc[2 * kk + 1][2], acc[2 * kk + 1][3]);
  }
}

// A fragments of a 16 x 16 BF16 input tile (row stride `ld` elements).
__device__ __forceinline__ void x_frags(const __nv_bfloat16* x, int ld, uint32_t* a) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  a[0] = *reinterpret_cast<const uint32_t*>(x + g * ld + 2 * t);
  a[1] = *reinterpret_cast<const uint32_t*>(x + (g + 8) * ld + 2 * t);
  a[2] = *reinterpret_cast<const uint32_t*>(x + g * ld + 8 + 2 * t);
  a[3] = *reinterpret_cast<const uint32_t*>(x + (g + 8) * ld + 8 + 2 * t);
}

// Row stride (BF16 elements) of the inference input tiles: 24 keeps the A
// fragment loads free of bank conflicts.
constexpr int XLD = 24;

// Forward of 32 normalised samples; x = the warp's inputs as a BF16 [32][XLD]
// tile (features 8..15 zero) in shared memory.  out0 / out1: output fragments
// of rows 0..15 / 16..31 (rows g, g + 8; columns 2t, 2t + 1; columns 6, 7
// padding).
__device__ __forceinline__ void forward32(const SmemFwd& s, const __nv_bfloat16* x,
                                          float out0[4], float out1[4]) {
  uint32_t a0[16], a1[16];
  x_frags(x, XLD, a0);
  x_frags(x + 16 * XLD, XLD, a1);
  float c0[8][4], c1[8][4];
  layer_fwd2<0>(s.wf, s.bias, a0, a1, c0, c1);
  to_a<true>(c0, a0);
  to_a<true>(c1, a1);
  layer_fwd2<1>(s.wf, s.bias, a0, a1, c0, c1);
  to_a<true>(c0, a0);
  to_a<true>(c1, a1);
  layer_fwd2<2>(s.wf, s.bias, a0, a1, c0, c1);
  to_a<true>(c0, a0);
  to_a<true>(c1, a1);
  float o0[1][4], o1[1][4];
  layer_fwd2<3>(s.wf, s.bias, a0, a1, o0, o1);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    out0[e] = o0[0][e];
    out1[e] = o1[0][e];
  }
}

}  // namespace mlp
}  // namespace pflb
