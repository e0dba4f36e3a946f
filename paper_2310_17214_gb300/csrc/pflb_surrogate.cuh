// pflb_surrogate.cuh -- chemistry pre-pass with the learned surrogate.
//
// Per cell the MLP maps the normalised (T, Y_1..Y_6, P0) to the normalised
// species change over one step, dY_k = exp(-theta_s / T) (y_mean_k + y_std_k
// out_k): the Arrhenius factor takes out most of the temperature dependence,
// and cold gas gets a change that vanishes with the true one.  A cell keeps the network's answer when its
// inputs lie inside the training bounding box and the raw output conserves
// every element to within `tol` (|sum_k a_ek M_e / M_k dY_k| <= tol); the
// accepted change is projected onto the element-conserving subspace and the
// temperature change follows from the formation enthalpies at fixed density
// (dT = -sum hf_k dY_k / cp(Y + dY), as the backward-Euler step satisfies).
// Other fluid cells are appended to a fallback list that the backward-Euler
// Newton integrator then processes.
#pragma once

#include "pflb_kernels.cuh"
#include "pflb_mlp.cuh"

namespace pflb {

struct SurrArgs {
  mlp::Net net;
  float x_mean[8], x_istd[8], y_mean[6], y_std[6];
  float lo[8], hi[8];       // training bounding box of the raw inputs
  double theta_s;           // output scale temperature
  int n_elem;
  double E[4][6];           // residual weights a_ek M_e / M_k
  double Pj[6][6];          // projection onto element-conserving increments
  double tol;
  float E_f[4][6], Pj_f[6][6], tol_f, theta_f;  // the same in FP32
  double T_skip;            // cells at T <= T_skip need no network (0: none)
  float T_skip_f;
  int engine;               // 0: warp-level mma.sync network kernel, 1: tcgen05 kernel
  int* fb_idx;              // fallback cell list
  unsigned* fb_count;
  double* stats;            // [0] fallback cells, [1] cells evaluated by the network
};

// Raw inputs (T, Y_1..Y_6, P0) inside the training bounding box.
__device__ __forceinline__ bool surrogate_in_box(const SurrArgs& A, const float* raw) {
  bool ok = true;
#pragma unroll
  for (int f = 0; f < 8; ++f) ok = ok && raw[f] >= A.lo[f] && raw[f] <= A.hi[f];
  return ok;
}

// Whether live cell c needs the network: a fluid cell inside the box above
// T_skip (a solid cell takes no source, a cell outside the box goes to the
// fallback whatever the network says, and below T_skip the network's
// projected increment is bounded by the record's skip_eps).
template <int K, class Real>
__device__ __forceinline__ bool surrogate_needs_net(const Params<Real, K>& P, const SurrArgs& A,
                                                    const float* raw, Real T, Real phif) {
  const Real Ts = sizeof(Real) == 8 ? Real(A.T_skip) : Real(A.T_skip_f);
  return phif >= P.phi_min && T > Ts && surrogate_in_box(A, raw);
}

// Live cell c of a tile that skips the network (no cell of it needs the
// network): zero source, and the bookkeeping of surrogate_post_cell (a fluid
// cell is evaluated; outside the box it is reported for the fallback: true).
template <int K, class Real>
__device__ __forceinline__ bool surrogate_skip_cell(const Params<Real, K>& P, const SurrArgs& A,
                                                    Real* __restrict__ src, long long c,
                                                    const float* raw, Real phif,
                                                    unsigned& evaluated, unsigned& fallbacks) {
  bool reject = false;
  if (phif >= P.phi_min) {
    ++evaluated;
    if (!surrogate_in_box(A, raw)) {
      ++fallbacks;
      reject = true;
    }
  }
#pragma unroll
  for (int k = 0; k <= 6; ++k) src[(size_t)k * P.N + c] = Real(0);
  return reject;
}

// Ordered, warp-aggregated append of the warp's rejected cells to the
// fallback list: neighbouring cells stay together in the list, so the
// integrator's warps see similar states.  Every lane of the warp calls it.
__device__ __forceinline__ void surrogate_append_fallback(const SurrArgs& A, bool reject,
                                                          long long c) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned mask = __ballot_sync(0xffffffffu, reject);
  if (mask) {
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(A.fb_count, (unsigned)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (reject) A.fb_idx[base + __popc(mask & ((1u << lane) - 1u))] = (int)c;
  }
}

// Per-cell use of the network's raw outputs o[0..5] for live cell c:
// de-normalise, test the bounding box and the element residuals, project and
// write the source, or leave the source zero and report the cell for the
// fallback (returns true).  Cells below phi_min get a zero source.
template <int K, class Real, class Store>
__device__ __forceinline__ bool surrogate_post_cell(const Params<Real, K>& P,
                                                    const State<Real, Store>& S,
                                                    const SurrArgs& A, Real* __restrict__ src,
                                                    long long c, const float* raw, const Real* Y,
                                                    Real T, Real phif, Real P0, const float* o,
                                                    unsigned& evaluated, unsigned& fallbacks) {
  bool reject = false;
  Real om[6], omT = 0;
#pragma unroll
  for (int k = 0; k < 6; ++k) om[k] = 0;
  if (phif >= P.phi_min) {
    ++evaluated;
    bool ok = surrogate_in_box(A, raw);
    // post-processing in the compute precision (FP64 domains keep FP64)
    constexpr bool D64 = sizeof(Real) == 8;
    Real dY[6];
    const Real th = D64 ? Real(A.theta_s) : Real(A.theta_f);
    const Real sc = th > Real(0) ? fexp(-fdiv(th, T)) : Real(1);
#pragma unroll
    for (int k = 0; k < 6; ++k) dY[k] = sc * (Real(o[k]) * Real(A.y_std[k]) + Real(A.y_mean[k]));
    const Real tol = D64 ? Real(A.tol) : Real(A.tol_f);
    for (int e = 0; e < A.n_elem; ++e) {
      Real r = 0;
#pragma unroll
      for (int k = 0; k < 6; ++k) r += (D64 ? Real(A.E[e][k]) : Real(A.E_f[e][k])) * dY[k];
      ok = ok && fabs(r) <= tol;
    }
    if (ok) {
      Real pY[6], cpn = 0, hsum = 0;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        Real sum = 0;
#pragma unroll
        for (int q = 0; q < 6; ++q) sum += (D64 ? Real(A.Pj[k][q]) : Real(A.Pj_f[k][q])) * dY[q];
        pY[k] = sum;
        cpn += (Y[k] + sum) * P.cp[k];
        hsum += P.hf[k] * sum;
      }
      const Real rho = fdiv(P0 * P.eos_cr, T * mixture_invMw(P, Y));
#pragma unroll
      for (int k = 0; k < 6; ++k) om[k] = rho * pY[k];
      omT = rho * mixture_cp(P, Y) * fdiv(-hsum, cpn);
    } else {
      ++fallbacks;
      reject = true;
    }
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) src[(size_t)k * P.N + c] = om[k];
  src[(size_t)6 * P.N + c] = omT;
  return reject;
}

template <int K, class Real, class Store>
__global__ void __launch_bounds__(256, 2)
chem_surrogate_kernel(const Params<Real, K> P, const State<Real, Store> S, Real* __restrict__ src,
                      const SurrArgs A) {
  static_assert(K == 6, "the surrogate is built for the six-species mechanism");
  __shared__ mlp::SmemFwd net;
  __shared__ __align__(16) __nv_bfloat16 xs[8][32 * mlp::XLD];
  __shared__ float ys[8][32 * 8];
  __shared__ unsigned blk_eval, blk_fb;
  mlp::load_fwd(net, A.net);
  if (threadIdx.x == 0) blk_eval = blk_fb = 0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const Real P0 = scal_P0<Real>(S.scal);
  const long long tiles = ((long long)P.N + 31) / 32;
  unsigned evaluated = 0, fallbacks = 0;
  for (long long tile = (long long)blockIdx.x * 8 + warp; tile < tiles;
       tile += (long long)gridDim.x * 8) {
    // one cell per lane: 32 consecutive cells per warp
    const long long c = tile * 32 + lane;
    const bool live = c < P.N;
    float raw[8];
    Real Y[6];
    Real T = 1, phif = 0;
    if (live) {
      T = S.T_in[c];
      phif = Real(1) - S.phi[c];
#pragma unroll
      for (int k = 0; k < 6; ++k) Y[k] = S.Y_in[(size_t)k * P.N + c];
    } else {
#pragma unroll
      for (int k = 0; k < 6; ++k) Y[k] = 0;
    }
    raw[0] = float(T);
#pragma unroll
    for (int k = 0; k < 6; ++k) raw[1 + k] = float(Y[k]);
    raw[7] = float(P0);
    if (!__any_sync(0xffffffffu, live && surrogate_needs_net<K, Real>(P, A, raw, T, phif))) {
      // no cell of the tile needs the network
      const bool reject =
          live && surrogate_skip_cell<K, Real>(P, A, src, c, raw, phif, evaluated, fallbacks);
      surrogate_append_fallback(A, reject, c);
      continue;
    }
    {
      uint32_t* xr = reinterpret_cast<uint32_t*>(xs[warp] + lane * mlp::XLD);
#pragma unroll
      for (int f = 0; f < 4; ++f)
        xr[f] = mlp::pack_bf16((raw[2 * f] - A.x_mean[2 * f]) * A.x_istd[2 * f],
                               (raw[2 * f + 1] - A.x_mean[2 * f + 1]) * A.x_istd[2 * f + 1]);
#pragma unroll
      for (int f = 4; f < 8; ++f) xr[f] = 0u;
    }
    __syncwarp();
    float o[2][4];
    mlp::forward32(net, xs[warp], o[0], o[1]);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      *reinterpret_cast<float2*>(&ys[warp][(16 * h + g) * 8 + 2 * t]) = make_float2(o[h][0], o[h][1]);
      *reinterpret_cast<float2*>(&ys[warp][(16 * h + g + 8) * 8 + 2 * t]) =
          make_float2(o[h][2], o[h][3]);
    }
    __syncwarp();
    bool reject = false;
    if (live) {
      float o[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) o[k] = ys[warp][lane * 8 + k];
      reject = surrogate_post_cell<K, Real, Store>(P, S, A, src, c, raw, Y, T, phif, P0, o,
                                                   evaluated, fallbacks);
    }
    surrogate_append_fallback(A, reject, c);
    __syncwarp();
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
  __syncthreads();
  if (threadIdx.x == 0 && (blk_eval || blk_fb)) {
    atomicAdd(&A.stats[0], (double)blk_fb);
    atomicAdd(&A.stats[1], (double)blk_eval);
  }
}

template <int K, class Real, class Store>
__device__ __forceinline__ void fallback_cell(const Params<Real, K>& P, const State<Real, Store>& S,
                                              Real* __restrict__ src, const int c) {
  constexpr int KK = K > 0 ? K : 1;
  const Real T = S.T_in[c];
  Real Y[KK];
#pragma unroll
  for (int k = 0; k < K; ++k) Y[k] = S.Y_in[(size_t)k * P.N + c];
  const Real P0 = scal_P0<Real>(S.scal);
  const Real rho = fdiv(P0 * P.eos_cr, T * mixture_invMw(P, Y));
  if constexpr (sizeof(Real) == 4) {
    // FP32 domains: the FP32 integrator (the fields it feeds are FP32)
    float dY[KK], dT;
    chem_be_newton32<K>(P.c32, T, Y, rho * float(P.c64.rho_ref), dY, &dT);
#pragma unroll
    for (int k = 0; k < K; ++k) src[(size_t)k * P.N + c] = rho * dY[k];
    src[(size_t)K * P.N + c] = rho * mixture_cp(P, Y) * dT;
  } else {
    double Yd[KK], dY[KK], dT;
#pragma unroll
    for (int k = 0; k < K; ++k) Yd[k] = double(Y[k]);
    chem_be_newton<K, Real>(&P.c64, double(T), Yd, double(rho) * P.c64.rho_ref, dY, &dT);
#pragma unroll
    for (int k = 0; k < K; ++k) src[(size_t)k * P.N + c] = rho * Real(dY[k]);
    src[(size_t)K * P.N + c] = rho * mixture_cp(P, Y) * Real(dT);
  }
}

// Backward-Euler Newton for the cells the surrogate rejected.  The list is
// short and the integrator is bound by the latency of its chain,
// so the kernel runs one warp per block, grid-striding: a list of a few
// hundred cells spreads over as many SMs as it has warps.
constexpr int FALLBACK_BLOCK = 32;

template <int K, class Real, class Store>
__global__ void __launch_bounds__(FALLBACK_BLOCK)
chem_fallback_kernel(const __grid_constant__ Params<Real, K> P, const State<Real, Store> S,
                     Real* __restrict__ src,
                     const int* __restrict__ fb_idx, const unsigned* __restrict__ fb_count) {
  const unsigned n = *fb_count;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    fallback_cell<K>(P, S, src, fb_idx[i]);
}

// src (rho* dY_k, rho* cp dT) -> increments (dY_k, dT) of the current state.
template <int K, class Real, class Store>
__global__ void __launch_bounds__(BLOCK)
src_to_increments_kernel(const Params<Real, K> P, const State<Real, Store> S,
                         const Real* __restrict__ src, double* __restrict__ out) {
  constexpr int KK = K > 0 ? K : 1;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P.N) return;
  const Real T = S.T_in[c];
  Real Y[KK];
#pragma unroll
  for (int k = 0; k < K; ++k) Y[k] = S.Y_in[(size_t)k * P.N + c];
  const Real P0 = scal_P0<Real>(S.scal);
  const Real rho = fdiv(P0 * P.eos_cr, T * mixture_invMw(P, Y));
#pragma unroll
  for (int k = 0; k < K; ++k) out[(size_t)k * P.N + c] = double(src[(size_t)k * P.N + c]) / double(rho);
  out[(size_t)K * P.N + c] = double(src[(size_t)K * P.N + c]) / (double(rho) * double(mixture_cp(P, Y)));
}

}  // namespace pflb
