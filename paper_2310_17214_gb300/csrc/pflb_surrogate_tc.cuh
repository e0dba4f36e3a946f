// pflb_surrogate_tc.cuh -- the surrogate's network on the fifth-generation
// tensor cores (tcgen05, accumulators in tensor memory).
//
// A block of 128 threads evaluates 128 cells at a time, one cell per thread
// and per TMEM lane.  The four dense layers 8 -> 64 -> 64 -> 64 -> 6 are four
// tcgen05.mma groups, M = 128, N = 64 (16 for the output layer, padded from
// 6), K = 16 per instruction (the input layer's 8 features padded to 16).
// Operands sit in shared memory in the canonical K-major layout without
// swizzle: 8-row x 16-byte core matrices, adjacent along K 128 bytes apart
// (leading byte offset) and along M or N K * 2 * 8 bytes apart (stride byte
// offset).  One elected thread issues the MMAs and commits them to an
// mbarrier; every warp then reads its 32 lanes of the accumulator with
// tcgen05.ld, adds the bias, applies tanh and writes the BF16 activations back
// as the next layer's A operand.  The weights are the network's FP32 master
// parameters rounded to BF16 (round to nearest), the same values as the
// warp-level kernel's; the accumulation is FP32.
#pragma once

#include "pflb_surrogate.cuh"
#include "pflb_tma.cuh"

namespace pflb {
namespace tc {

constexpr int M = 128;  // cells per tile (TMEM lanes)
constexpr int NCOL = 64;  // TMEM columns allocated (FP32 accumulator of 64 outputs)

// Shared memory of one block.  Every operand starts on a 128-byte boundary.
struct Smem {
  __align__(128) __nv_bfloat16 a[M * 64];     // activations, K-major core matrices
  __align__(128) __nv_bfloat16 w0[64 * 16];   // layer weights as B (N x K), K-major
  __align__(128) __nv_bfloat16 w1[64 * 64];
  __align__(128) __nv_bfloat16 w2[64 * 64];
  __align__(128) __nv_bfloat16 w3[16 * 64];
  float b0[64], b1[64], b2[64], b3[16];
  __align__(8) uint64_t bar;
  uint32_t tmem;
  int err;
  int layer_ok;  // the MMA group of the current layer reported in time
};

// Byte offset of element (row r, column k) in a K-major core-matrix layout
// of K columns.
__device__ __forceinline__ int kmajor_off(int r, int k, int K) {
  return (((r >> 3) * (K >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1);
}

// Shared-memory matrix descriptor (no swizzle): start address, leading byte
// offset (along K), stride byte offset (along M / N), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(const void* p, uint32_t lbo, uint32_t sbo) {
  const uint32_t a = smem_u32(p);
  uint64_t d = 0;
  d |= (uint64_t)((a & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N and M.
__host__ __device__ constexpr uint32_t idesc(int n, int m) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(id), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane, without waiting:
// the registers are valid after tmem_wait_ld().
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Weight W_l (input-major [in][out], FP32, inside the flat parameter vector)
// as the B operand (N = out padded to NP, K = in padded to KP), BF16, by the
// block's M threads: every load is issued before the first store (read along
// the output index, so that neighbouring threads read neighbouring weights).
template <int L, int NP, int KP>
__device__ __forceinline__ void load_b(__nv_bfloat16* dst, const float* __restrict__ theta) {
  constexpr int IN = mlp::dim(L), OUT = mlp::dim(L + 1), R = NP * KP / M;
  static_assert(NP * KP % M == 0, "whole rounds of the block");
  constexpr int C = R < 16 ? R : 16;  // loads in flight per thread
  static_assert(R % C == 0, "whole chunks");
  const float* W = theta + mlp::woff(L);
  char* base = reinterpret_cast<char*>(dst);
#pragma unroll 1
  for (int r0 = 0; r0 < R; r0 += C) {
    float v[C];
#pragma unroll
    for (int r = 0; r < C; ++r) {
      const int i = threadIdx.x + (r0 + r) * M, n = i % NP, k = i / NP;
      v[r] = (n < OUT && k < IN) ? __ldg(W + k * OUT + n) : 0.f;
    }
#pragma unroll
    for (int r = 0; r < C; ++r) {
      const int i = threadIdx.x + (r0 + r) * M, n = i % NP, k = i / NP;
      *reinterpret_cast<__nv_bfloat16*>(base + kmajor_off(n, k, KP)) = __float2bfloat16_rn(v[r]);
    }
  }
}

}  // namespace tc

// The surrogate pre-pass of chem_surrogate_kernel with the network on
// tcgen05.  Grid-strides over tiles of 128 cells; per cell the same
// acceptance test, projection and fallback list as the warp-level kernel.
template <int K, class Real, class Store>
__global__ void __launch_bounds__(tc::M, 5)
chem_surrogate_tc_kernel(const Params<Real, K> P, const State<Real, Store> S,
                         Real* __restrict__ src, const SurrArgs A, long long wait_limit) {
  static_assert(K == 6, "the surrogate is built for the six-species mechanism");
  using namespace tc;
  extern __shared__ __align__(16) unsigned char tc_raw[];
  // the operands want 128-byte alignment: the launch adds 128 bytes of slack
  Smem& s = *reinterpret_cast<Smem*>((reinterpret_cast<uintptr_t>(tc_raw) + 127) & ~uintptr_t(127));
  __shared__ unsigned blk_eval, blk_fb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // weights, biases, barrier, tensor memory
  load_b<0, 64, 16>(s.w0, A.net.theta);
  load_b<1, 64, 64>(s.w1, A.net.theta);
  load_b<2, 64, 64>(s.w2, A.net.theta);
  load_b<3, 16, 64>(s.w3, A.net.theta);
  for (int i = threadIdx.x; i < 64; i += blockDim.x) {
    s.b0[i] = A.net.theta[mlp::boff(0) + i];
    s.b1[i] = A.net.theta[mlp::boff(1) + i];
    s.b2[i] = A.net.theta[mlp::boff(2) + i];
    if (i < 16) s.b3[i] = i < 6 ? A.net.theta[mlp::boff(3) + i] : 0.f;
  }
  if (threadIdx.x == 0) {
    blk_eval = blk_fb = 0;
    s.err = 0;
    mbar_init(&s.bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&s.tmem, NCOL);
  fence_proxy_async();  // weights written by threads, read by the tensor cores
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s.tmem;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's lanes

  // operand descriptors (LBO 128 bytes; SBO = K * 16 bytes)
  const uint64_t dw0 = sdesc(s.w0, 128, 16 * 16), dw1 = sdesc(s.w1, 128, 64 * 16);
  const uint64_t dw2 = sdesc(s.w2, 128, 64 * 16), dw3 = sdesc(s.w3, 128, 64 * 16);
  const uint64_t da16 = sdesc(s.a, 128, 16 * 16), da64 = sdesc(s.a, 128, 64 * 16);
  constexpr uint32_t ID64 = idesc(64, M), ID16 = idesc(16, M);

  const Real P0 = scal_P0<Real>(S.scal);
  const long long tiles = ((long long)P.N + M - 1) / M;
  unsigned evaluated = 0, fallbacks = 0, phase = 0;
  char* abase = reinterpret_cast<char*>(s.a);
  const int m = threadIdx.x;
  bool failed = false;

  // one layer: MMA group of ksteps K = 16 steps, wait, bias + tanh into the
  // next A operand (or the outputs)
  auto run_layer = [&](uint64_t da, uint64_t db, uint32_t id, int ksteps) -> bool {
    fence_proxy_async();
    fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
      fence_after();
      for (int ks = 0; ks < ksteps; ++ks)  // K = 16 per step: two core matrices (256 bytes)
        tc::mma_bf16(tmem, da + (uint64_t)((ks * 256) >> 4), db + (uint64_t)((ks * 256) >> 4),
                     id, ks > 0 ? 1u : 0u);
      tc::mma_commit(&s.bar);
      // one thread waits for the group; the barrier then releases the block
      // (and makes the outcome the same for every thread)
      s.layer_ok = mbar_wait_bounded(&s.bar, phase & 1u, wait_limit) ? 1 : 0;
    }
    phase ^= 1u;
    __syncthreads();
    fence_after();
    return s.layer_ok != 0;
  };

  // the inputs of the block's next tile are loaded while the current one
  // runs through the network
  Real nT = 1, nphi = 0, nY[6];
  auto fetch = [&](long long t) {
    const long long cn = t * M + m;
    nT = 1;
    nphi = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) nY[k] = 0;
    if (t < tiles && cn < P.N) {
      nT = S.T_in[cn];
      nphi = S.phi[cn];
#pragma unroll
      for (int k = 0; k < 6; ++k) nY[k] = S.Y_in[(size_t)k * P.N + cn];
    }
  };
  fetch(blockIdx.x);
  for (long long tile = blockIdx.x; tile < tiles && !failed; tile += gridDim.x) {
    const long long c = tile * M + m;
    const bool live = c < P.N;
    float raw[8];
    Real Y[6];
    const Real T = nT, phif = Real(1) - nphi;
#pragma unroll
    for (int k = 0; k < 6; ++k) Y[k] = nY[k];
    fetch(tile + gridDim.x);
    raw[0] = float(T);
#pragma unroll
    for (int k = 0; k < 6; ++k) raw[1 + k] = float(Y[k]);
    raw[7] = float(P0);
    if (!__syncthreads_or(live && surrogate_needs_net<K, Real>(P, A, raw, T, phif))) {
      // no cell of the tile needs the network
      const bool reject =
          live && surrogate_skip_cell<K, Real>(P, A, src, c, raw, phif, evaluated, fallbacks);
      surrogate_append_fallback(A, reject, c);
      continue;
    }
    // layer-0 input row: 8 normalised features and 8 zeros (K = 16)
    {
      uint32_t w[8];
#pragma unroll
      for (int f = 0; f < 4; ++f)
        w[f] = mlp::pack_bf16((raw[2 * f] - A.x_mean[2 * f]) * A.x_istd[2 * f],
                              (raw[2 * f + 1] - A.x_mean[2 * f + 1]) * A.x_istd[2 * f + 1]);
#pragma unroll
      for (int f = 4; f < 8; ++f) w[f] = 0u;
      *reinterpret_cast<uint4*>(abase + tc::kmajor_off(m, 0, 16)) = make_uint4(w[0], w[1], w[2], w[3]);
      *reinterpret_cast<uint4*>(abase + tc::kmajor_off(m, 8, 16)) = make_uint4(w[4], w[5], w[6], w[7]);
    }
    float o[16];
    const float* bias[3] = {s.b0, s.b1, s.b2};
    const uint64_t dws[3] = {dw0, dw1, dw2};
    for (int l = 0; l < 3 && !failed; ++l) {
      if (!run_layer(l == 0 ? da16 : da64, dws[l], ID64, l == 0 ? 1 : 4)) { failed = true; break; }
      // bias + tanh -> BF16 A operand of the next layer (K = 64)
      // two 16-column groups in flight per wait
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t acc[2][16];
        tc::tmem_ld16_async(trow + 32 * h, acc[0]);
        tc::tmem_ld16_async(trow + 32 * h + 16, acc[1]);
        tc::tmem_wait_ld();
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          const int q = 2 * h + g;
          uint32_t w[8];
#pragma unroll
          for (int e = 0; e < 8; ++e)
            w[e] = mlp::pack_bf16(
                mlp::fast_tanh(__uint_as_float(acc[g][2 * e]) + bias[l][16 * q + 2 * e]),
                mlp::fast_tanh(__uint_as_float(acc[g][2 * e + 1]) + bias[l][16 * q + 2 * e + 1]));
          *reinterpret_cast<uint4*>(abase + tc::kmajor_off(m, 16 * q, 64)) =
              make_uint4(w[0], w[1], w[2], w[3]);
          *reinterpret_cast<uint4*>(abase + tc::kmajor_off(m, 16 * q + 8, 64)) =
              make_uint4(w[4], w[5], w[6], w[7]);
        }
      }
    }
    if (failed || !run_layer(da64, dw3, ID16, 4)) { failed = true; break; }
    tc::tmem_ld16(trow, o);
#pragma unroll
    for (int k = 0; k < 6; ++k) o[k] += s.b3[k];

    bool reject = false;
    if (live)
      reject = surrogate_post_cell<K, Real, Store>(P, S, A, src, c, raw, Y, T, phif, P0, o,
                                                   evaluated, fallbacks);
    surrogate_append_fallback(A, reject, c);
  }
  if (failed) {
    // an MMA group that did not report: wait once more (bounded) for it
    // before the tensor memory is released
    if (threadIdx.x == 0) {
      mbar_wait_bounded(&s.bar, (phase ^ 1u) & 1u, wait_limit);
      s.err = 1;
    }
  }
  // counts of this warp
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) {
    evaluated += __shfl_xor_sync(0xffffffffu, evaluated, o2);
    fallbacks += __shfl_xor_sync(0xffffffffu, fallbacks, o2);
  }
  if (lane == 0 && (evaluated || fallbacks)) {
    atomicAdd(&blk_fb, fallbacks);
    atomicAdd(&blk_eval, evaluated);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, NCOL);
  if (threadIdx.x == 0) {
    if (blk_eval || blk_fb) {
      atomicAdd(&A.stats[0], (double)blk_fb);
      atomicAdd(&A.stats[1], (double)blk_eval);
    }
    if (s.err) atomicCAS(&S.scal->status, 0, -6);  // PFLB_ERR_TIMEOUT
  }
}

constexpr size_t tc_smem_bytes() { return sizeof(tc::Smem) + 128; }
constexpr int kTcBlocksPerSm = 5;  // shared memory: 5 x 38 KB

}  // namespace pflb
