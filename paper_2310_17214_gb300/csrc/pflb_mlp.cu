// pflb_mlp.cu -- training and inference kernels of the chemistry-surrogate MLP
// and their C ABI (pflb_mlp_*, declared in include/pflb.h).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/pflb.h"
#include "pflb_mlp.cuh"

using namespace pflb::mlp;

struct pflb_mlp {
  int device = 0;
  cudaStream_t stream = nullptr;
  float* theta = nullptr;  // FP32 master parameters
  float* m = nullptr;      // Adam moments
  float* v = nullptr;
  float* grad = nullptr;   // gradient accumulator
  double* loss = nullptr;  // loss accumulator
  __nv_bfloat16* wf = nullptr;
  __nv_bfloat16* wb = nullptr;
  float* bias = nullptr;
  long long t = 0;         // Adam step count
};

namespace {

constexpr int TW = 8;  // warps per block in the training kernel

struct WarpSmem {
  __nv_bfloat16 x[16 * 16];
  __nv_bfloat16 h[3][16 * 64];
  __nv_bfloat16 dz[16 * 64];
  __nv_bfloat16 dO[16 * 8];
};
struct TrainSmem {
  SmemNet net;
  float dW[NPARAM];
  WarpSmem w[TW];
  double loss;
};

// Padded BF16 copies of the FP32 parameters (both layouts) and biases.
__global__ void pack_kernel(const float* __restrict__ theta, __nv_bfloat16* __restrict__ wf,
                            __nv_bfloat16* __restrict__ wb, float* __restrict__ bias) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < NPAD + NPB;
       idx += gridDim.x * blockDim.x) {
    if (idx >= NPAD) {
      const int q = idx - NPAD;
      int l = 0;
      while (l < NL - 1 && q >= pboff(l + 1)) ++l;
      const int o = q - pboff(l);
      bias[q] = o < dim(l + 1) ? theta[boff(l) + o] : 0.f;
      continue;
    }
    int l = 0;
    while (l < NL - 1 && idx >= poff(l + 1)) ++l;
    const int r = idx - poff(l), IN = pdim(l), OUT = pdim(l + 1);
    // forward layout: B fragments in lane order (see Net)
    {
      const int e = r & 3, lane = (r >> 2) & 31, tile = r >> 7, KT = IN / 16;
      const int j = tile / KT, kk = tile % KT;
      const int o = 8 * j + (lane >> 2);
      const int i = 16 * kk + 2 * (lane & 3) + (e & 1) + (e >= 2 ? 8 : 0);
      const float w = (i < dim(l) && o < dim(l + 1)) ? theta[woff(l) + i * dim(l + 1) + o] : 0.f;
      wf[idx] = __float2bfloat16_rn(w);
    }
    // backward layout [in][out]
    {
      const int i = r / OUT, o = r % OUT;
      const float w = (i < dim(l) && o < dim(l + 1)) ? theta[woff(l) + i * dim(l + 1) + o] : 0.f;
      wb[idx] = __float2bfloat16_rn(w);
    }
  }
}

// Stage 16 normalised input rows (features 0..7) into a BF16 [16][16] tile.
__device__ __forceinline__ void stage_x(__nv_bfloat16* x16, const float* __restrict__ X,
                                        long long row0, long long n) {
  const int lane = threadIdx.x & 31;
  const int r = lane & 15, half = lane >> 4;
  const long long row = row0 + r;
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    const int col = half * 8 + f;
    float v = 0.f;
    if (col < 8 && row < n) v = X[row * 8 + col];
    x16[r * 16 + col] = __float2bfloat16_rn(v);
  }
}

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// dW_l += A^T dZ for 16 samples on tensor cores: A (16 x IN) and dZ (16 x OUT)
// are warp-staged BF16 tiles; accumulates into the block's FP32 copy.
template <int L>
__device__ __forceinline__ void grad_w(const __nv_bfloat16* A, const __nv_bfloat16* dZ, float* dW) {
  constexpr int IN = pdim(L), OUT = pdim(L + 1);
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  auto pk = [](__nv_bfloat16 lo, __nv_bfloat16 hi) {
    __nv_bfloat162 v;
    v.x = lo;
    v.y = hi;
    return *reinterpret_cast<uint32_t*>(&v);
  };
#pragma unroll
  for (int mt = 0; mt < IN / 16; ++mt) {
    uint32_t a[4];
    const int m0 = 16 * mt + g;
    a[0] = pk(A[(2 * t) * IN + m0], A[(2 * t + 1) * IN + m0]);
    a[1] = pk(A[(2 * t) * IN + m0 + 8], A[(2 * t + 1) * IN + m0 + 8]);
    a[2] = pk(A[(2 * t + 8) * IN + m0], A[(2 * t + 9) * IN + m0]);
    a[3] = pk(A[(2 * t + 8) * IN + m0 + 8], A[(2 * t + 9) * IN + m0 + 8]);
#pragma unroll
    for (int nt = 0; nt < OUT / 8; ++nt) {
      const int n0 = 8 * nt + g;
      const uint32_t b0 = pk(dZ[(2 * t) * OUT + n0], dZ[(2 * t + 1) * OUT + n0]);
      const uint32_t b1 = pk(dZ[(2 * t + 8) * OUT + n0], dZ[(2 * t + 9) * OUT + n0]);
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      mma16816(c, a, b0, b1);
      const int rows[2] = {16 * mt + g, 16 * mt + g + 8};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int mi = rows[e >> 1], ni = 8 * nt + 2 * t + (e & 1);
        if (mi < dim(L) && ni < dim(L + 1)) atomicAdd(&dW[woff(L) + mi * dim(L + 1) + ni], c[e]);
      }
    }
  }
}

// Bias gradient: column sums of the 16 x OUT fragment set (rows g, g + 8).
template <int L, int NT>
__device__ __forceinline__ void grad_b(const float acc[][4], float* dW) {
  const int lane = threadIdx.x & 31, t = lane & 3;
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    float s0 = acc[j][0] + acc[j][2], s1 = acc[j][1] + acc[j][3];
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if (lane < 4) {
      const int n0 = 8 * j + 2 * t;
      if (n0 < dim(L + 1)) atomicAdd(&dW[boff(L) + n0], s0);
      if (n0 + 1 < dim(L + 1)) atomicAdd(&dW[boff(L) + n0 + 1], s1);
    }
  }
}

// Store a 16 x 64 fragment set as a BF16 [16][64] tile.
__device__ __forceinline__ void store_tile(__nv_bfloat16* T, const float acc[8][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    *reinterpret_cast<uint32_t*>(T + g * 64 + 8 * j + 2 * t) = pack_bf16(acc[j][0], acc[j][1]);
    *reinterpret_cast<uint32_t*>(T + (g + 8) * 64 + 8 * j + 2 * t) = pack_bf16(acc[j][2], acc[j][3]);
  }
}

// dH = dZ_next W^T (dZ_next as A fragments, W from the backward layout), then
// dZ = dH (1 - H^2) with H read back from the warp's tile.
template <int L>
__device__ __forceinline__ void back_dx(const SmemNet& s, const uint32_t* a, const __nv_bfloat16* H,
                                        float acc[8][4]) {
  constexpr int IN = pdim(L), OUT = pdim(L + 1);  // W_L is IN x OUT; dX has IN = 64 columns
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const __nv_bfloat16* W = s.wb + poff(L);
#pragma unroll
  for (int j = 0; j < IN / 8; ++j) {
    acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < (OUT + 15) / 16; ++kk) {
      const __nv_bfloat16* wr = W + (8 * j + g) * OUT + 16 * kk + 2 * t;
      const uint32_t b0 = (16 * kk + 2 * t < OUT) ? *reinterpret_cast<const uint32_t*>(wr) : 0u;
      const uint32_t b1 = (16 * kk + 8 + 2 * t < OUT) ? *reinterpret_cast<const uint32_t*>(wr + 8) : 0u;
      mma16816(acc[j], a + 4 * kk, b0, b1);
    }
    const float h0 = bf(H[g * 64 + 8 * j + 2 * t]), h1 = bf(H[g * 64 + 8 * j + 2 * t + 1]);
    const float h2 = bf(H[(g + 8) * 64 + 8 * j + 2 * t]), h3 = bf(H[(g + 8) * 64 + 8 * j + 2 * t + 1]);
    acc[j][0] *= 1.f - h0 * h0;
    acc[j][1] *= 1.f - h1 * h1;
    acc[j][2] *= 1.f - h2 * h2;
    acc[j][3] *= 1.f - h3 * h3;
  }
}

// Forward + backward of mini-batch rows; accumulates the gradient of the mean
// squared error (scaled by inv_norm = 1 / (rows x 6)) and the loss.
__global__ void __launch_bounds__(TW * 32, 1)
grad_kernel(Net net, const float* __restrict__ X, const float* __restrict__ Y, long long n,
            float inv_norm, float* __restrict__ grad, double* __restrict__ loss) {
  extern __shared__ __align__(16) unsigned char smem[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem);
  load_net(S.net, net);
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) S.dW[i] = 0.f;
  if (threadIdx.x == 0) S.loss = 0.0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  WarpSmem& W = S.w[warp];
  const long long tiles = (n + 15) / 16;
  float lsum = 0.f;
  for (long long tile = (long long)blockIdx.x * TW + warp; tile < tiles;
       tile += (long long)gridDim.x * TW) {
    const long long row0 = tile * 16;
    stage_x(W.x, X, row0, n);
    __syncwarp();
    // forward, keeping H1..H3
    uint32_t a[16];
    x_frags(W.x, 16, a);
    float acc[8][4];
    layer_fwd<0>(S.net.wf, S.net.bias, a, acc);
    to_a<true>(acc, a);
    store_tile(W.h[0], acc);
    layer_fwd<1>(S.net.wf, S.net.bias, a, acc);
    to_a<true>(acc, a);
    store_tile(W.h[1], acc);
    layer_fwd<2>(S.net.wf, S.net.bias, a, acc);
    to_a<true>(acc, a);
    store_tile(W.h[2], acc);
    float o[1][4];
    layer_fwd<3>(S.net.wf, S.net.bias, a, o);
    // output gradient 2 (o - y) / (rows x 6)
    const long long rr[2] = {row0 + g, row0 + g + 8};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const long long row = rr[e >> 1];
      const int col = 2 * t + (e & 1);
      float d = 0.f;
      if (row < n && col < 6) {
        const float diff = o[0][e] - Y[row * 6 + col];
        lsum += diff * diff;
        d = 2.f * diff * inv_norm;
      }
      o[0][e] = d;
    }
    *reinterpret_cast<uint32_t*>(W.dO + g * 8 + 2 * t) = pack_bf16(o[0][0], o[0][1]);
    *reinterpret_cast<uint32_t*>(W.dO + (g + 8) * 8 + 2 * t) = pack_bf16(o[0][2], o[0][3]);
    __syncwarp();
    // layer 4 (W4: 64 x 6)
    grad_w<3>(W.h[2], W.dO, S.dW);
    grad_b<3, 1>(o, S.dW);
    uint32_t ad[16];
    ad[0] = pack_bf16(o[0][0], o[0][1]);
    ad[1] = pack_bf16(o[0][2], o[0][3]);
    ad[2] = ad[3] = 0u;
    back_dx<3>(S.net, ad, W.h[2], acc);  // dZ3
    // layer 3 (W3)
    store_tile(W.dz, acc);
    __syncwarp();
    grad_w<2>(W.h[1], W.dz, S.dW);
    grad_b<2, 8>(acc, S.dW);
    to_a<false>(acc, ad);
    __syncwarp();
    back_dx<2>(S.net, ad, W.h[1], acc);  // dZ2
    // layer 2 (W2)
    store_tile(W.dz, acc);
    __syncwarp();
    grad_w<1>(W.h[0], W.dz, S.dW);
    grad_b<1, 8>(acc, S.dW);
    to_a<false>(acc, ad);
    __syncwarp();
    back_dx<1>(S.net, ad, W.h[0], acc);  // dZ1
    // layer 1 (W1: 8 x 64, padded input tile)
    store_tile(W.dz, acc);
    __syncwarp();
    grad_w<0>(W.x, W.dz, S.dW);
    grad_b<0, 8>(acc, S.dW);
    __syncwarp();
  }
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o2);
  if (lane == 0) atomicAdd(&S.loss, (double)lsum);
  __syncthreads();
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x)
    if (S.dW[i] != 0.f) atomicAdd(&grad[i], S.dW[i]);
  if (threadIdx.x == 0) atomicAdd(loss, S.loss);
}

__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                            float* __restrict__ grad, float lr, float c1, float c2) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x) {
    const float gi = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    grad[i] = 0.f;
  }
}

// Stage 32 normalised input rows into a BF16 [32][XLD] tile (one row per
// lane; features 8..15 zero).
__device__ __forceinline__ void stage_x32(__nv_bfloat16* x, const float* __restrict__ X,
                                          long long row0, long long n) {
  const int lane = threadIdx.x & 31;
  const long long row = row0 + lane;
  float v[8];
  if (row < n) {
    const float4 p0 = *reinterpret_cast<const float4*>(X + row * 8);
    const float4 p1 = *reinterpret_cast<const float4*>(X + row * 8 + 4);
    v[0] = p0.x; v[1] = p0.y; v[2] = p0.z; v[3] = p0.w;
    v[4] = p1.x; v[5] = p1.y; v[6] = p1.z; v[7] = p1.w;
  } else {
#pragma unroll
    for (int f = 0; f < 8; ++f) v[f] = 0.f;
  }
  uint32_t* r = reinterpret_cast<uint32_t*>(x + lane * XLD);
#pragma unroll
  for (int f = 0; f < 4; ++f) r[f] = pack_bf16(v[2 * f], v[2 * f + 1]);
#pragma unroll
  for (int f = 4; f < 8; ++f) r[f] = 0u;
}

__global__ void __launch_bounds__(256, 2)
forward_kernel(Net net, const float* __restrict__ X, float* __restrict__ out, long long n) {
  __shared__ SmemFwd s;
  __shared__ __align__(16) __nv_bfloat16 xs[8][32 * XLD];
  load_fwd(s, net);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const long long tiles = (n + 31) / 32;
  for (long long tile = (long long)blockIdx.x * 8 + warp; tile < tiles;
       tile += (long long)gridDim.x * 8) {
    stage_x32(xs[warp], X, tile * 32, n);
    __syncwarp();
    float o[2][4];
    forward32(s, xs[warp], o[0], o[1]);
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const long long row = tile * 32 + 16 * h + g + (e >> 1) * 8;
        const int col = 2 * t + (e & 1);
        if (row < n && col < 6) out[row * 6 + col] = o[h][e];
      }
    __syncwarp();
  }
}

int grid_for(long long rows, int per_block) {
  long long b = (rows + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > 1184) b = 1184;
  return (int)b;
}

Net net_of(const pflb_mlp* m) { return Net{m->wf, m->wb, m->bias, m->theta}; }

}  // namespace

namespace pflb {
// Network pointers of a handle (used by the surrogate chemistry pre-pass).
Net mlp_net(const pflb_mlp* m) { return net_of(m); }
}  // namespace pflb

extern "C" {

int pflb_mlp_create(int device, void* stream, pflb_mlp** out) {
  if (!out) return PFLB_ERR_ARG;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return PFLB_ERR_CUDA;
  pflb_mlp* m = new (std::nothrow) pflb_mlp();
  if (!m) return PFLB_ERR_OOM;
  m->device = device;
  m->stream = static_cast<cudaStream_t>(stream);
  bool ok = cudaMalloc(&m->theta, NPARAM * 4) == cudaSuccess &&
            cudaMalloc(&m->m, NPARAM * 4) == cudaSuccess &&
            cudaMalloc(&m->v, NPARAM * 4) == cudaSuccess &&
            cudaMalloc(&m->grad, NPARAM * 4) == cudaSuccess &&
            cudaMalloc(&m->loss, sizeof(double)) == cudaSuccess &&
            cudaMalloc(&m->wf, NPAD * 2) == cudaSuccess &&
            cudaMalloc(&m->wb, NPAD * 2) == cudaSuccess &&
            cudaMalloc(&m->bias, NPB * 4) == cudaSuccess;
  if (!ok) {
    pflb_mlp_destroy(m);
    return PFLB_ERR_OOM;
  }
  cudaMemset(m->theta, 0, NPARAM * 4);
  cudaMemset(m->m, 0, NPARAM * 4);
  cudaMemset(m->v, 0, NPARAM * 4);
  cudaMemset(m->grad, 0, NPARAM * 4);
  cudaMemset(m->wf, 0, NPAD * 2);
  cudaMemset(m->wb, 0, NPAD * 2);
  cudaMemset(m->bias, 0, NPB * 4);
  if (cudaFuncSetAttribute(grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(TrainSmem)) != cudaSuccess) {
    pflb_mlp_destroy(m);
    return PFLB_ERR_CUDA;
  }
  *out = m;
  return PFLB_OK;
}

int pflb_mlp_set_params(pflb_mlp* m, const float* theta) {
  if (!m || !theta) return PFLB_ERR_ARG;
  cudaSetDevice(m->device);
  if (cudaMemcpyAsync(m->theta, theta, NPARAM * 4, cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
    return PFLB_ERR_CUDA;
  cudaMemsetAsync(m->m, 0, NPARAM * 4, m->stream);
  cudaMemsetAsync(m->v, 0, NPARAM * 4, m->stream);
  cudaMemsetAsync(m->grad, 0, NPARAM * 4, m->stream);
  m->t = 0;
  pack_kernel<<<(NPAD + NPB + 255) / 256, 256, 0, m->stream>>>(m->theta, m->wf, m->wb, m->bias);
  if (cudaGetLastError() != cudaSuccess) return PFLB_ERR_CUDA;
  return cudaStreamSynchronize(m->stream) == cudaSuccess ? PFLB_OK : PFLB_ERR_CUDA;
}

int pflb_mlp_get_params(pflb_mlp* m, float* theta) {
  if (!m || !theta) return PFLB_ERR_ARG;
  cudaSetDevice(m->device);
  if (cudaMemcpyAsync(theta, m->theta, NPARAM * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
    return PFLB_ERR_CUDA;
  return cudaStreamSynchronize(m->stream) == cudaSuccess ? PFLB_OK : PFLB_ERR_CUDA;
}

int pflb_mlp_forward(pflb_mlp* m, const float* X, float* out, long long n) {
  if (!m || !X || !out || n < 0 || (reinterpret_cast<uintptr_t>(X) & 15)) return PFLB_ERR_ARG;
  if (n == 0) return PFLB_OK;
  cudaSetDevice(m->device);
  forward_kernel<<<grid_for(n, 256), 256, 0, m->stream>>>(net_of(m), X, out, n);
  return cudaGetLastError() == cudaSuccess ? PFLB_OK : PFLB_ERR_CUDA;
}

int pflb_mlp_gradient(pflb_mlp* m, const float* X, const float* Y, long long n, float* grad,
                      double* loss) {
  if (!m || !X || !Y || n <= 0) return PFLB_ERR_ARG;
  cudaSetDevice(m->device);
  cudaMemsetAsync(m->grad, 0, NPARAM * 4, m->stream);
  cudaMemsetAsync(m->loss, 0, sizeof(double), m->stream);
  grad_kernel<<<grid_for(n, 16 * TW), TW * 32, sizeof(TrainSmem), m->stream>>>(
      net_of(m), X, Y, n, 1.f / (float)(n * 6), m->grad, m->loss);
  if (cudaGetLastError() != cudaSuccess) return PFLB_ERR_CUDA;
  double l = 0;
  if (grad && cudaMemcpyAsync(grad, m->grad, NPARAM * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
    return PFLB_ERR_CUDA;
  if (cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess)
    return PFLB_ERR_CUDA;
  cudaMemsetAsync(m->grad, 0, NPARAM * 4, m->stream);
  if (loss) *loss = l / (double)(n * 6);
  return PFLB_OK;
}

int pflb_mlp_train(pflb_mlp* m, const float* X, const float* Y, long long n, int batch, int steps,
                   float lr, double* last_loss) {
  if (!m || !X || !Y || n <= 0 || batch <= 0 || steps < 0) return PFLB_ERR_ARG;
  cudaSetDevice(m->device);
  const long long nb = (n + batch - 1) / batch;
  for (int s = 0; s < steps; ++s) {
    const long long b = s % nb;
    const long long r0 = b * batch;
    const long long rows = (r0 + batch <= n) ? batch : n - r0;
    const bool last = s == steps - 1;
    if (last) cudaMemsetAsync(m->loss, 0, sizeof(double), m->stream);
    grad_kernel<<<grid_for(rows, 16 * TW), TW * 32, sizeof(TrainSmem), m->stream>>>(
        net_of(m), X + r0 * 8, Y + r0 * 6, rows, 1.f / (float)(rows * 6), m->grad, m->loss);
    m->t += 1;
    const float c1 = 1.f / (1.f - powf(0.9f, (float)m->t));
    const float c2 = 1.f / (1.f - powf(0.999f, (float)m->t));
    adam_kernel<<<(NPARAM + 255) / 256, 256, 0, m->stream>>>(m->theta, m->m, m->v, m->grad, lr,
                                                             c1, c2);
    pack_kernel<<<(NPAD + NPB + 255) / 256, 256, 0, m->stream>>>(m->theta, m->wf, m->wb, m->bias);
    if (last && last_loss) {
      double l = 0;
      cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream);
      cudaStreamSynchronize(m->stream);
      *last_loss = l / (double)(rows * 6);
    }
  }
  return cudaGetLastError() == cudaSuccess ? PFLB_OK : PFLB_ERR_CUDA;
}

int pflb_mlp_destroy(pflb_mlp* m) {
  if (!m) return PFLB_OK;
  cudaSetDevice(m->device);
  cudaStreamSynchronize(m->stream);
  void* p[] = {m->theta, m->m, m->v, m->grad, m->loss, m->wf, m->wb, m->bias};
  for (void* q : p)
    if (q) cudaFree(q);
  delete m;
  return PFLB_OK;
}

}  // extern "C"
