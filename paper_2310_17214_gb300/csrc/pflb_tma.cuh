// pflb_tma.cuh -- persistent, TMA-pipelined fused step for 2-D lattices with
// FP32 compute (FP32 or FP16-stored populations).
//
// Each block walks a strided list of 32 x 8 tiles.  One elected thread issues
// the tensor-memory-accelerator loads of the NEXT tile into the other half of
// a double-buffered stage while the block works on the current one:
//   - T, phi_s, Ts: 2-D boxes of (32 + 2 XL) x 10 cells (tile + halo; the x
//     start is rounded down to a 16-byte boundary, XL = 16 / sizeof(Real));
//   - Y_k: one 3-D box (32 + 2 XL) x 10 x K;
//   - populations: for each direction i the 32 + 2 XLp by 8 window of g_i
//     shifted by -c_iy rows (the -c_ix column shift is an offset into the
//     box), so the pull of every interior cell reads shared memory.
// Loads complete on an mbarrier per stage (expect_tx = box bytes, a box that
// crosses the domain edge is zero-filled and still counts in full).  Cells on
// the domain edge use the boundary rules of the global-memory pull, and the
// staged halo of edge tiles is overwritten with the ghost / periodic values.
// Waits are bounded (pflb_set_wait_limit): a wait that runs out latches
// PFLB_ERR_TIMEOUT in the status word, waits (with the default bound) for the
// copies the block has in flight, and stops working on tiles; the block still
// publishes its partial sums so that the step's reduction completes.
#pragma once

#include <cuda.h>

#include "pflb_kernels.cuh"

namespace pflb {

// --------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait of at most `limit` SM clock cycles (a limit of 0 is one
// non-blocking probe): false when it ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity,
                                                  long long limit = kDefaultWaitCycles) {
  if (limit <= 0) return mbar_test_wait(bar, parity);
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y,
                                            int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Tensor maps of one step (input side of the current parity), kept on the
// host; the kernel receives each as its own __grid_constant__ parameter.
struct TmaMaps {
  CUtensorMap T, phi, Ts, Y, g;
};
struct TmaMapRefs {
  const CUtensorMap* T;
  const CUtensorMap* phi;
  const CUtensorMap* Ts;
  const CUtensorMap* Y;
  const CUtensorMap* g;
};

// ------------------------------------------------------------ stage layout
template <int K, class Store>
struct TmaLayout {
  static constexpr int TX = 32, TY = 8;
  static constexpr int XL = 4;                        // 16 B of floats
  static constexpr int FW = TX + 2 * XL, FH = TY + 2;  // field box
  static constexpr int XLP = 16 / (int)sizeof(Store);
  static constexpr int PW = TX + 2 * XLP, PH = TY;    // population box
  static constexpr int Q = 9;
  static constexpr int NRAW = 3 + K;                  // T, phi, Ts, Y_k
  static constexpr int FBOX = FW * FH;                // floats per field box
  static constexpr int FBP = (FBOX * 4 + 127) / 128 * 32;  // 128-byte aligned box slot
  static constexpr int OFF_T = 0, OFF_PHI = FBP, OFF_TS = 2 * FBP, OFF_Y = 3 * FBP;
  static constexpr int PBOX = PW * PH;                // Stores per population box
  static constexpr int HX = TX + 2, HP = HX * (TY + 2);
  static constexpr int NDER = 5;                      // rho, kT, mu, fD, RF
  static constexpr size_t raw_bytes = ((size_t)(3 * FBP + K * FBOX) * 4 + 127) / 128 * 128;
  static constexpr size_t pop_bytes = (size_t)Q * PBOX * sizeof(Store);
  static constexpr size_t stage_bytes = (raw_bytes + pop_bytes + 127) / 128 * 128;
  static constexpr size_t der_bytes = (size_t)NDER * HP * 4;
  // [stage 0][stage 1][derived plane][2 mbarriers][block-sum scratch][flag];
  // +128 so the base can be rounded up to a 128-byte boundary in the kernel
  static constexpr size_t bar_off = 2 * stage_bytes + der_bytes;
  static constexpr size_t red_off = bar_off + 64;
  static constexpr size_t flag_off = red_off + 32 * sizeof(double);
  static constexpr size_t smem_bytes = flag_off + 16 + 128;
};

// Accessor over a TMA stage (raw fields, populations) plus the derived plane.
template <int K, class Store>
struct TmaAcc {
  using LY = TmaLayout<K, Store>;
  static constexpr bool has_pops = true;
  static constexpr bool kStash = false;
  const float* __restrict__ raw;
  const Store* __restrict__ pops;
  const float* __restrict__ der;
  int lx, ly;
  bool pv;  // the stage's population windows are valid for this cell (off every face)
  __device__ __forceinline__ int ridx(int dx, int dy) const {
    return (ly + 1 + dy) * LY::FW + lx + LY::XL + dx;
  }
  __device__ __forceinline__ int didx(int dx, int dy) const {
    return (ly + 1 + dy) * LY::HX + lx + 1 + dx;
  }
  __device__ __forceinline__ float get(int f, int dx, int dy) const {
    switch (f) {
      case F_T: return raw[LY::OFF_T + ridx(dx, dy)];
      case F_PHI: return raw[LY::OFF_PHI + ridx(dx, dy)];
      case F_TS: return raw[LY::OFF_TS + ridx(dx, dy)];
      case F_RHO: return der[0 * LY::HP + didx(dx, dy)];
      case F_KT: return der[1 * LY::HP + didx(dx, dy)];
      case F_MU: return der[2 * LY::HP + didx(dx, dy)];
      case F_FD: return der[3 * LY::HP + didx(dx, dy)];
      case F_RF: return der[4 * LY::HP + didx(dx, dy)];
      default: return raw[LY::OFF_Y + (f - F_Y0) * LY::FBOX + ridx(dx, dy)];
    }
  }
  __device__ __forceinline__ float c(int f) const { return get(f, 0, 0); }
  __device__ __forceinline__ float n(int f, int a, int s) const {
    return a == 0 ? get(f, s, 0) : get(f, 0, s);
  }
  template <class S>
  __device__ __forceinline__ float pop(int i, float w_over_scale) const {
    const int cx = Lattice<2>::c(i, 0);
    return Codec<Store, float>::get(pops + i * LY::PBOX + ly * LY::PW + lx - cx + LY::XLP,
                                    w_over_scale);
  }
};

// Ghost / periodic values for the out-of-domain cells of an edge tile's
// staged halo (same rules as the staged-plane path).
template <int K, class Store>
__device__ __forceinline__ void fix_halo(const Params<float, K>& P,
                                         const State<float, Store>& S, float* raw, int x0,
                                         int y0) {
  using LY = TmaLayout<K, Store>;
  for (int h = threadIdx.x; h < LY::HP; h += blockDim.x) {
    const int hx = h % LY::HX, hy = h / LY::HX;
    int q[2] = {x0 - 1 + hx, y0 - 1 + hy};
    if ((q[0] >= 0 && q[0] < P.nx) && (q[1] >= 0 && q[1] < P.ny)) continue;
    int ghost_face = -1, nout = 0;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int n = a == 0 ? P.nx : P.ny;
      if (q[a] < 0 || q[a] >= n) {
        const int face = 2 * a + (q[a] >= n ? 1 : 0);
        if (P.bc[face] == BC_PERIODIC) {
          q[a] = q[a] < 0 ? q[a] + n : q[a] - n;
          if (q[a] < 0 || q[a] >= n) q[a] = q[a] < 0 ? 0 : n - 1;
        } else {
          q[a] = q[a] < 0 ? 0 : n - 1;
          ghost_face = face;
          ++nout;
        }
      }
    }
    const int c = q[0] + P.nx * q[1];
    float T = __ldg(S.T_in + c);
    const float phis = __ldg(S.phi + c);
    const float Ts = P.Ts_field ? __ldg(S.Ts_in + c) : P.Ts_uniform;
    float Y[Params<float, K>::KK];
#pragma unroll
    for (int k = 0; k < K; ++k) Y[k] = __ldg(S.Y_in + (size_t)k * P.N + c);
    if (nout == 1) {
      const int bc = P.bc[ghost_face];
      if (bc == BC_INLET) {
        T = P.T_in;
#pragma unroll
        for (int k = 0; k < K; ++k) Y[k] = P.Y_in[k];
      } else if (bc == BC_WALL && P.wall_T[ghost_face] > 0.f) {
        T = P.wall_T[ghost_face];
      }
    }
    const int r = hy * LY::FW + hx - 1 + LY::XL;
    raw[LY::OFF_T + r] = T;
    raw[LY::OFF_PHI + r] = phis;
    raw[LY::OFF_TS + r] = Ts;
#pragma unroll
    for (int k = 0; k < K; ++k) raw[LY::OFF_Y + k * LY::FBOX + r] = Y[k];
  }
}

// Properties of every staged cell (tile + halo) from the staged raw fields.
template <int K, class Store>
__device__ __forceinline__ void derive_plane(const Params<float, K>& P, float* raw,
                                             float* der, float P0) {
  using LY = TmaLayout<K, Store>;
  for (int h = threadIdx.x; h < LY::HP; h += blockDim.x) {
    const int hx = h % LY::HX, hy = h / LY::HX;
    if ((hx == 0 || hx == LY::HX - 1) && (hy == 0 || hy == LY::TY + 1)) continue;  // corners
    const int r = hy * LY::FW + hx - 1 + LY::XL;
    const float T = raw[LY::OFF_T + r];
    const float phis = raw[LY::OFF_PHI + r];
    if (!P.Ts_field) raw[LY::OFF_TS + r] = P.Ts_uniform;
    float Y[Params<float, K>::KK];
#pragma unroll
    for (int k = 0; k < K; ++k) Y[k] = raw[LY::OFF_Y + k * LY::FBOX + r];
    const float phif = 1.f - phis;
    const float invMw = mixture_invMw(P, Y);
    const float rho = fdiv(P0 * P.eos_cr, T * invMw);
    const float cp = mixture_cp(P, Y);
    float mu, lam;
    transport(P, T, Y, invMw, cp, mu, lam);
    float fD = 1.f;
    if constexpr (K > 0) {
      if (P.D_Tdep) fD = fpow(T * P.inv_DTref, P.D_exp);
    }
    der[0 * LY::HP + h] = rho;
    der[1 * LY::HP + h] = phif * lam;
    der[2 * LY::HP + h] = mu;
    der[3 * LY::HP + h] = fD;
    der[4 * LY::HP + h] = phif * rho * fD;
  }
}

template <int K, class Store>
__device__ __forceinline__ void issue_tile(const TmaMapRefs& M, const Params<float, K>& P,
                                           unsigned char* stage, uint64_t* bar, int x0, int y0) {
  using LY = TmaLayout<K, Store>;
  constexpr unsigned field_bytes = LY::FBOX * 4;
  const unsigned bytes = (unsigned)((P.Ts_field ? 3 : 2) * field_bytes + K * field_bytes +
                                    LY::pop_bytes);
  float* raw = reinterpret_cast<float*>(stage);
  Store* pops = reinterpret_cast<Store*>(stage + LY::raw_bytes);
  mbar_expect_tx(bar, bytes);
  tma_load_2d(raw + LY::OFF_T, M.T, x0 - LY::XL, y0 - 1, bar);
  tma_load_2d(raw + LY::OFF_PHI, M.phi, x0 - LY::XL, y0 - 1, bar);
  if (P.Ts_field) tma_load_2d(raw + LY::OFF_TS, M.Ts, x0 - LY::XL, y0 - 1, bar);
  if constexpr (K > 0) tma_load_3d(raw + LY::OFF_Y, M.Y, x0 - LY::XL, y0 - 1, 0, bar);
#pragma unroll
  for (int i = 0; i < LY::Q; ++i)
    tma_load_3d(pops + i * LY::PBOX, M.g, x0 - LY::XLP, y0 - Lattice<2>::c(i, 1), i, bar);
}

template <int K, class Store>
__global__ void __launch_bounds__(BLOCK, 2)
step_tma_kernel(const Params<float, K> P, const State<float, Store> S, int p0_closed,
                const double* __restrict__ prev_partials, unsigned prev_nb,
                const __grid_constant__ CUtensorMap mT, const __grid_constant__ CUtensorMap mPhi,
                const __grid_constant__ CUtensorMap mTs, const __grid_constant__ CUtensorMap mY,
                const __grid_constant__ CUtensorMap mG, int tiles_x, int n_tiles,
                long long wait_limit) {
  const TmaMapRefs M{&mT, &mPhi, &mTs, &mY, &mG};
  using LY = TmaLayout<K, Store>;
  // All shared memory of this kernel is the dynamic buffer, its base rounded up
  // to 128 bytes: TMA destinations are 128-byte aligned, mbarriers 8-byte.
  extern __shared__ unsigned char smem_dyn[];
  unsigned char* smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
  unsigned char* stage[2] = {smem_raw, smem_raw + LY::stage_bytes};
  float* der = reinterpret_cast<float*>(smem_raw + 2 * LY::stage_bytes);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + LY::bar_off);
  double* red_sh = reinterpret_cast<double*>(smem_raw + LY::red_off);
  int& s_ok = *reinterpret_cast<int*>(smem_raw + LY::flag_off);

  const float P0 = scal_P0<float>(S.scal);
  const float dlnP0 = scal_dlnP0<float>(S.scal);
  const float dP0r = scal_dP0r<float>(S.scal);

  if (prev_partials && blockIdx.x == 0 && threadIdx.x < 32)
    combine_partials(prev_partials, prev_nb, S.scal, 0, false, 0.0, P.eos_c, P.inv_rho_ref);

  // self-check of the alignment every TMA issue relies on (the same answer
  // in every thread): record it and skip all copies rather than fault
  const bool aligned = (smem_u32(stage[0]) & 127u) == 0 && (smem_u32(stage[1]) & 127u) == 0 &&
                       (smem_u32(bar) & 7u) == 0 &&
                       ((reinterpret_cast<uintptr_t>(&mT) | reinterpret_cast<uintptr_t>(&mPhi) |
                         reinterpret_cast<uintptr_t>(&mTs) | reinterpret_cast<uintptr_t>(&mY) |
                         reinterpret_cast<uintptr_t>(&mG)) & 63u) == 0;
  if (!aligned) {
    if (threadIdx.x == 0) atomicExch(&S.scal->status, -7);
    return;
  }

  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();

  const int lx = threadIdx.x % LY::TX, ly = threadIdx.x / LY::TX;
  float accI = 0.f, accIn = 0.f, accOut = 0.f;
  bool any_flux = false;
  int first = blockIdx.x;
  if (threadIdx.x == 0 && first < n_tiles)
    issue_tile<K, Store>(M, P, stage[0], &bar[0], (first % tiles_x) * LY::TX,
                         (first / tiles_x) * LY::TY);
  int it = 0;
  for (int t = first; t < n_tiles; t += gridDim.x, ++it) {
    const int s = it & 1;
    const int x0 = (t % tiles_x) * LY::TX, y0 = (t / tiles_x) * LY::TY;
    const int tn = t + gridDim.x;
    if (threadIdx.x == 0) {
      if (tn < n_tiles) {
        fence_proxy_async();
        issue_tile<K, Store>(M, P, stage[s ^ 1], &bar[s ^ 1], (tn % tiles_x) * LY::TX,
                             (tn / tiles_x) * LY::TY);
      }
      s_ok = mbar_wait_bounded(&bar[s], (it >> 1) & 1, wait_limit) ? 1 : 0;
      if (!s_ok) {
        // latch the timeout; then drain: every copy this block issued (the
        // current tile's and the next one's) completes before the block
        // leaves the loop, so none lands in a finished block's shared memory
        atomicExch(&S.scal->status, -6);
        mbar_wait_bounded(&bar[s], (it >> 1) & 1);
        if (tn < n_tiles) mbar_wait_bounded(&bar[s ^ 1], ((it + 1) >> 1) & 1);
      }
    }
    __syncthreads();
    if (!s_ok) break;  // uniform: the block still publishes its (partial) sums
    float* raw = reinterpret_cast<float*>(stage[s]);
    const bool edge_tile = x0 == 0 || y0 == 0 || x0 + LY::TX >= P.nx || y0 + LY::TY >= P.ny;
    if (edge_tile) {
      fix_halo<K, Store>(P, S, raw, x0, y0);
      __syncthreads();
    }
    derive_plane<K, Store>(P, raw, der, P0);
    __syncthreads();
    const int x = x0 + lx, y = y0 + ly;
    if (x < P.nx && y < P.ny) {
      const TmaAcc<K, Store> A{raw, reinterpret_cast<const Store*>(stage[s] + LY::raw_bytes), der,
                               lx, ly, x > 0 && x < P.nx - 1 && y > 0 && y < P.ny - 1};
      const int c = x + P.nx * y;
      const int xyz[3] = {x, y, 0};
      float fi, fo;
      accI += cell_update<2, K, float, Store>(P, S, A, c, xyz, P0, dlnP0, dP0r, fi, fo);
      accIn += fi;
      accOut += fo;
    }
    any_flux = any_flux || (x0 == 0 && P.bc[0] == BC_INLET) ||
               (x0 + LY::TX >= P.nx && P.bc[1] == BC_OUTLET);
    __syncthreads();
  }

  const double sI = block_sum<float>(accI, red_sh);
  double sIn = 0, sOut = 0;
  if (any_flux) {
    sIn = block_sum<float>(accIn, red_sh);
    sOut = block_sum<float>(accOut, red_sh);
  }
  publish_partials(sI, sIn, sOut, S.partials, S.counter, S.scal, p0_closed, false, 0.0, P.eos_c,
                   P.inv_rho_ref);
}

}  // namespace pflb
