// pflb_launch.cuh -- host-side launcher of the PF-LB-FD kernels for one
// (lattice, species count, precision) combination: converts the physical
// description to lattice units once and queues the kernels on a stream.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include <type_traits>

#include "../../include/pflb.h"
#include "pflb_batch.cuh"
#include "pflb_chem.cuh"
#include "pflb_step3d.cuh"
#include "pflb_kernels.cuh"
#include "pflb_surrogate.cuh"
#include "pflb_tma.cuh"

namespace pflb {

struct Buffers {
  void* g[2];
  void* M[2];              // FP16 storage: FP32 moments [DIM+1][N] of g[b] (else null)
  void* T[2];
  void* Y[2];
  void* Ts[2];
  void* phi;
  void* src;               // chemistry increments [K+1][N] (implicit / surrogate modes)
  int* fb_idx;             // surrogate fallback list [N]
  unsigned* fb_count;
  double* chem_stats;      // [0] fallback cells, [1] cells evaluated by the network
  DevScalars* scal;
  double* partials;        // two buffers of `slots` x 4 doubles (step parity)
  unsigned* counter;
  unsigned* tile_ctr;      // tile counters of the persistent step, one per parity
  double* feed_part;       // inlet feedback block partials [kFeedBlocks]
  void* ob;                // characteristic outlet columns [5][ny nz] (compute type)
  void* phi0;              // moving solid: the phase field of step 0 (phi is the current one)
  long long nstep;         // steps taken (host copy; the phase field of a moving solid)
  int N;
  long long slots;         // partial slots per buffer (>= blocks of any launch)
  int pending;             // the last step's partials are not combined yet
  int last_parity;         // buffer holding them
  long long last_nb;       // blocks of the launch that wrote them
};

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
inline EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// Tiled tensor map of a row-major array with `rank` dims (x fastest).
inline bool encode_map(CUtensorMap* m, const void* base, CUtensorMapDataType dt, int esz,
                       int rank, const unsigned long long* dims, const unsigned* box) {
  EncodeTiledFn f = encode_tiled();
  if (!f) return false;
  cuuint64_t gd[3], gs[2];
  cuuint32_t bd[3], es[3] = {1, 1, 1};
  unsigned long long stride = (unsigned long long)esz;
  for (int r = 0; r < rank; ++r) {
    gd[r] = dims[r];
    bd[r] = box[r];
    if (r > 0) gs[r - 1] = stride;
    stride *= dims[r];
  }
  return f(m, dt, rank, const_cast<void*>(base), gd, gs, bd, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct Launcher {
  virtual ~Launcher() {}
  // g = g_eq from the current T, Y (and optional u, dim*N in the compute type)
  virtual cudaError_t init(const Buffers& B, int cur, const void* u_init, double P0,
                           cudaStream_t st) = 0;
  // nsteps fused steps; `cur` flips once per step
  virtual cudaError_t step(Buffers& B, int& cur, int nsteps, cudaStream_t st) = 0;
  virtual cudaError_t moments(const Buffers& B, int cur, double* u, double* rho, double* ph,
                              cudaStream_t st) = 0;
  // combine deferred partials of the last step into the scalar state
  virtual cudaError_t finalize(Buffers& B, cudaStream_t st) = 0;
  // step kernel: 0 = staged tiles, 1 = TMA-pipelined persistent tiles (2-D
  // FP32 compute with 16-byte rows), 2 / 3 = persistent staged tiles 32 x 8 /
  // 32 x 16 (2-D); returns false if not available here
  virtual bool select_kernel(int k, const Buffers& B, int cur) = 0;
  virtual int kernel() const = 0;
  // learned chemistry (six-species mechanism only)
  virtual bool set_surrogate(const SurrArgs& a) = 0;
  // chemistry pre-pass of the current state into B.src; increments (dY, dT)
  // into `out` ([K+1][N] doubles) when non-null
  virtual cudaError_t chem_pass(Buffers& B, int cur, double* out, cudaStream_t st) = 0;
  virtual float g_scale() const = 0;
  // ---- batched stepping (2-D lattices without species) ----
  // bytes of this domain's batch work-list entry (0: cannot be batched)
  virtual size_t batch_entry_bytes() const = 0;
  // the entry: parameters, both ping-pong states, P0 mode, current buffer
  virtual void batch_entry(void* dst, const Buffers& B, int cur) const = 0;
  // resident blocks per SM of the batch kernel for tile shape cfg
  virtual int batch_occupancy(int cfg) const = 0;
  virtual cudaError_t batch_launch(const void* entries, const int* tile_begin, int ndom, int cfg,
                                   int grid, int flip, unsigned* tile_ctr,
                                   cudaStream_t st) const = 0;
  // domains can share a batch when their keys are equal (same kernel)
  virtual int batch_key() const = 0;
  // bound of the kernels' device waits (SM clock cycles)
  virtual void set_wait_limit(long long cycles) = 0;
  // NDIAG diagnostic sums of the current state into out (device); part holds
  // blocks() * NDIAG doubles
  virtual cudaError_t diagnostics(const Buffers& B, int cur, double* part, double* out,
                                  cudaStream_t st) = 0;
  virtual int diag_blocks() const = 0;
  // steps taken is n (after init or a restored state): a moving solid's phase
  // field becomes the one of step n
  virtual cudaError_t set_step(Buffers& B, long long n, cudaStream_t st) = 0;
};

constexpr double R_GAS = 8.314;  // J/(mol K), value printed in Sec. 3.1

template <class Real, int K>
Params<Real, K> make_params(const pflb_domain_desc& d, const pflb_mechanism& m, int mode) {
  Params<Real, K> P;
  std::memset(&P, 0, sizeof(P));
  P.nx = d.nx;
  P.ny = d.ny;
  P.nz = d.dim == 3 ? d.nz : 1;
  P.N = P.nx * P.ny * P.nz;
  for (int f = 0; f < 6; ++f) {
    P.bc[f] = d.bc[f];
    for (int a = 0; a < 3; ++a) P.wall_u[f][a] = Real(d.wall_u[f][a]);
    P.wall_T[f] = Real(d.wall_T[f]);
  }
  const double h2 = d.dt / (d.dx * d.dx);
  P.eos_c = 1.0 / (R_GAS * d.rho_ref);
  P.eos_cr = Real(P.eos_c);
  P.inv_rho_ref = 1.0 / d.rho_ref;
  P.mu_lat = Real(d.mu_ref * h2 / d.rho_ref);
  P.sutherland = d.sutherland;
  P.inv_suth_T = Real(d.sutherland ? 1.0 / d.suth_T : 1.0);
  P.suth_S = Real(d.suth_S);
  P.suth_TS = Real(d.suth_T + d.suth_S);
  P.inv_Pr = Real(1.0 / d.Pr);
  P.Au_eta2 = Real(d.A_u / (d.eta * d.eta));
  P.AT_eta2 = Real(d.A_T / (d.eta * d.eta));
  for (int a = 0; a < 3; ++a) P.Fb[a] = Real(d.Fb[a]);
  P.inlet_parabolic = d.inlet_parabolic;
  P.u_in = Real(d.u_in);
  P.T_in = Real(d.T_in);
  P.M0 = Real(d.M0);
  P.cp0 = Real(d.cp0);
  for (int k = 0; k < K; ++k) {
    P.Y_in[k] = Real(m.Y_in[k]);
    P.invM[k] = Real(1.0 / m.M[k]);
    P.cp[k] = Real(m.cp[k]);
    P.hf[k] = Real(m.hf[k]);
    P.Dlat[k] = Real(m.Dref[k] * h2);
    P.cpD[k] = Real(m.cp[k] * m.Dref[k] * h2);
    P.rho_ref_M[k] = Real(d.rho_ref / m.M[k]);
  }
  P.D_Tdep = (K > 0 && m.D_exp != 0.0) ? 1 : 0;
  P.inv_DTref = Real(K > 0 && m.D_Tref > 0 ? 1.0 / m.D_Tref : 1.0);
  P.D_exp = Real(K > 0 ? m.D_exp : 0.0);
  P.Ts_field = d.Ts_field;
  P.Ts_uniform = Real(d.Ts_uniform);
  P.Cs = Real(d.rhocp_s / d.rho_ref);
  P.Lams = Real(d.lambda_s * h2 / d.rho_ref);
  P.phi_min = Real(d.phi_min);
  P.chem = K > 0 ? m.chem_mode : 0;
  P.J = K > 0 ? m.J : 0;
  for (int j = 0; j < P.J; ++j) {
    P.A_lat[j] = Real(m.A[j] * d.dt / d.rho_ref);
    P.b[j] = Real(m.b[j]);
    P.EaR[j] = Real(m.EaR[j]);
    for (int k = 0; k < K; ++k) {
      P.order[j][k] = Real(m.order[j][k]);
      P.stoichM[j][k] = Real(m.stoich[j][k] * m.M[k]);
    }
  }
  for (int j = 0; j < P.J; ++j) {
    P.rev[j] = m.rev[j];
    double dn = 0;
    for (int k = 0; k < K; ++k) {
      P.rorder[j][k] = Real(m.rorder[j][k]);
      dn += m.stoich[j][k];
    }
    P.dS_R[j] = Real(m.dS[j] / R_GAS);
    P.dH_R[j] = Real(m.dH[j] / R_GAS);
    P.dn[j] = Real(dn);
    auto& c = P.c64;
    c.A[j] = m.A[j];
    c.b[j] = m.b[j];
    c.EaR[j] = m.EaR[j];
    c.dH[j] = m.dH[j];
    c.dS[j] = m.dS[j];
    c.dn[j] = dn;
    c.rev[j] = m.rev[j];
    for (int k = 0; k < K; ++k) {
      c.order[j][k] = m.order[j][k];
      c.rorder[j][k] = m.rorder[j][k];
      c.stoich[j][k] = m.stoich[j][k];
      c.Ms[j][k] = m.M[k] * m.stoich[j][k];
    }
    c.dS_R[j] = m.dS[j] / R_GAS;
    c.dH_R[j] = m.dH[j] / R_GAS;
  }
  P.p_ref_R = Real(K > 0 && m.p_ref > 0 ? m.p_ref / R_GAS : 101325.0 / R_GAS);
  for (int k = 0; k < K; ++k) {
    P.c64.M[k] = m.M[k];
    P.c64.invM[k] = 1.0 / m.M[k];
    P.c64.cp[k] = m.cp[k];
    P.c64.hf[k] = m.hf[k];
  }
  P.c64.p_ref = m.p_ref > 0 ? m.p_ref : 101325.0;
  P.c64.ln_pref_R = std::log(P.c64.p_ref / R_GAS);
  P.c64.rho_ref = d.rho_ref;
  P.c64.dt = d.dt;
  {
    auto& f = P.c32;
    const auto& c = P.c64;
    for (int j = 0; j < P.J; ++j) {
      f.on[j] = c.A[j] > 0.0 ? 1 : 0;
      f.lnA[j] = float(c.A[j] > 0.0 ? std::log(c.A[j]) : 0.0);
      f.b[j] = float(c.b[j]);
      f.EaR[j] = float(c.EaR[j]);
      f.dn[j] = float(c.dn[j]);
      f.dS_R[j] = float(c.dS_R[j]);
      f.dH_R[j] = float(c.dH_R[j]);
      f.rev[j] = c.rev[j];
      for (int k = 0; k < K; ++k) {
        f.order[j][k] = float(c.order[j][k]);
        f.rorder[j][k] = float(c.rorder[j][k]);
        f.Ms[j][k] = float(c.Ms[j][k]);
      }
    }
    for (int k = 0; k < K; ++k) {
      f.invM[k] = float(c.invM[k]);
      f.cp[k] = float(c.cp[k]);
      f.hf[k] = float(c.hf[k]);
    }
    f.ln_pref_R = float(c.ln_pref_R);
    f.dt = float(c.dt);
  }
  // inlet feedback: rho_in / P0 (lattice) and the inlet area A, the inlet
  // profile at unit peak speed summed over the x = 0 face
  P.feed = (K > 0 && m.inlet_feedback > 0) ? 1 : 0;
  P.feed_k = P.feed ? m.inlet_feedback - 1 : 0;
  P.feed_c = 0.0;
  if (P.feed) {
    double invMw = 0;
    for (int k = 0; k < K; ++k) invMw += m.Y_in[k] / m.M[k];
    const double rin = 1.0 / (invMw * R_GAS * d.T_in * d.rho_ref);
    const int nz = d.dim == 3 ? d.nz : 1;
    double area = 0;
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < d.ny; ++y) {
        double u = 1.0;
        for (int a = 1; a < d.dim && d.inlet_parabolic; ++a) {
          if (d.bc[2 * a] != PFLB_BC_WALL) continue;
          const double n = a == 1 ? d.ny : d.nz, sa = (a == 1 ? y : z) + 0.5;
          u *= 4.0 * sa * (n - sa) / (n * n);
        }
        area += u;
      }
    P.feed_c = 1.0 / (rin * m.Y_in[P.feed_k] * area);
  }
  P.moving = (d.u_s[0] != 0.0 || d.u_s[1] != 0.0 || (d.dim == 3 && d.u_s[2] != 0.0)) ? 1 : 0;
  for (int a = 0; a < 3; ++a) P.u_s[a] = Real(a < d.dim ? d.u_s[a] : 0.0);
  P.nscbc = (d.outlet_nscbc && d.bc[1] == PFLB_BC_OUTLET) ? 1 : 0;
  P.nscbc_K = P.nscbc ? d.nscbc_sigma * std::sqrt(1.0 / 3.0) / d.nx : 0.0;
  // FP16 residual scale: residuals |r / w| from 4 down to 3.7e-9 (lattice
  // units) stay in the normal FP16 range; smaller ones keep an absolute
  // resolution of 3.6e-12 as subnormals
  P.mix = (K > 0 && m.transport == PFLB_TRANSPORT_MIXTURE) ? 1 : 0;
  for (int k = 0; k < K; ++k) {
    const double sT = m.suth_Tk[k] > 0 ? m.suth_Tk[k] : 1.0;
    P.mu_lat_k[k] = Real(m.mu_k[k] * h2 / d.rho_ref);
    P.inv_suth_Tk[k] = Real(1.0 / sT);
    P.suth_Sk[k] = Real(m.suth_Sk[k]);
    P.suth_TSk[k] = Real(sT + m.suth_Sk[k]);
    const double RM = R_GAS / m.M[k];
    P.eucken_k[k] = Real(1.32 * (m.cp[k] - RM) + 1.77 * RM);
    for (int j = 0; j < K; ++j) {
      P.wA[k][j] = Real(std::pow(m.M[j] / m.M[k], 0.25));
      P.wB[k][j] = Real(1.0 / (std::sqrt(8.0) * std::sqrt(1.0 + m.M[k] / m.M[j])));
    }
  }
  const float s = mode == MODE_FP16 ? 16384.0f : 1.0f;
  P.g_scale = Real(s);
  P.g_inv_scale = Real(1.0f / s);
  return P;
}

template <int MODE> struct ModeTypes;
template <> struct ModeTypes<MODE_FP64> { using Real = double; using Store = double; };
template <> struct ModeTypes<MODE_FP32> { using Real = float; using Store = float; };
template <> struct ModeTypes<MODE_FP16> { using Real = float; using Store = __half; };

template <int DIM, int K, int MODE>
struct LauncherImpl final : Launcher {
  using Real = typename ModeTypes<MODE>::Real;
  using Store = typename ModeTypes<MODE>::Store;
  Params<Real, K> P;
  int p0_closed;
  double u_in0;  // inlet peak speed of the first step

  LauncherImpl(const pflb_domain_desc& d, const pflb_mechanism& m)
      : P(make_params<Real, K>(d, m, MODE)), p0_closed(d.p0_mode == PFLB_P0_CLOSED),
        u_in0(d.u_in) {}

  State<Real, Store> state(const Buffers& B, int cur) const {
    State<Real, Store> S;
    const int nxt = 1 - cur;
    S.g_in = static_cast<const Store*>(B.g[cur]);
    S.g_out = static_cast<Store*>(B.g[nxt]);
    S.M_in = static_cast<const Real*>(B.M[cur]);
    S.M_out = static_cast<Real*>(B.M[nxt]);
    S.T_in = static_cast<const Real*>(B.T[cur]);
    S.T_out = static_cast<Real*>(B.T[nxt]);
    S.Y_in = static_cast<const Real*>(B.Y[cur]);
    S.Y_out = static_cast<Real*>(B.Y[nxt]);
    S.Ts_in = static_cast<const Real*>(B.Ts[cur]);
    S.Ts_out = static_cast<Real*>(B.Ts[nxt]);
    S.phi = static_cast<const Real*>(B.phi);
    S.src = static_cast<const Real*>(B.src);
    S.scal = B.scal;
    S.partials = B.partials + (size_t)4 * B.slots * cur;
    S.counter = B.counter;
    S.ob = static_cast<Real*>(B.ob);
    return S;
  }
  int blocks() const { return (P.N + BLOCK - 1) / BLOCK; }
  // tile grid of the fused step (32 x 8 tiles; 3-D blocks march 16 planes)
  dim3 step_grid() const {
    using T_ = Tile<DIM>;
    return dim3((P.nx + T_::TX - 1) / T_::TX, (P.ny + T_::TY - 1) / T_::TY,
                DIM == 3 ? (P.nz + T_::ZC - 1) / T_::ZC : 1);
  }
  long long step_blocks() const {
    dim3 g = step_grid();
    return (long long)g.x * g.y * g.z;
  }

  cudaError_t init(const Buffers& B, int cur, const void* u_init, double P0,
                   cudaStream_t st) override {
    State<Real, Store> S = state(B, cur);
    // the equilibrium is written into the current buffer
    S.g_out = static_cast<Store*>(B.g[cur]);
    S.M_out = static_cast<Real*>(B.M[cur]);
    init_kernel<DIM, K, Real, Store><<<blocks(), BLOCK, 0, st>>>(
        P, S, static_cast<const Real*>(u_init), P0);
    set_inlet_kernel<<<1, 1, 0, st>>>(B.scal, u_in0);
    return cudaGetLastError();
  }
  // phase field of step n of a moving solid from the step-0 field
  cudaError_t phase(const Buffers& B, long long n, cudaStream_t st) const {
    int per = 0;
    for (int a = 0; a < DIM; ++a)
      if (P.bc[2 * a] == BC_PERIODIC) per |= 1 << a;
    int sh[3] = {0, 0, 0};
    double fr[3] = {0, 0, 0};
    for (int a = 0; a < DIM; ++a) {
      const double sa = double(n) * double(P.u_s[a]);
      sh[a] = (int)std::floor(sa);
      fr[a] = sa - sh[a];
    }
    phase_shift_kernel<DIM, Real><<<blocks(), BLOCK, 0, st>>>(
        static_cast<const Real*>(B.phi0), static_cast<Real*>(B.phi), P.nx, P.ny, P.nz, per,
        make_int3(sh[0], sh[1], sh[2]), Real(fr[0]), Real(fr[1]), Real(fr[2]));
    return cudaGetLastError();
  }
  cudaError_t set_step(Buffers& B, long long n, cudaStream_t st) override {
    B.nstep = n;
    return P.moving ? phase(B, n, st) : cudaSuccess;
  }
  // inlet feedback after the step whose input state is buffer `cur`
  cudaError_t feed(const Buffers& B, int cur, cudaStream_t st) const {
    const int grid = blocks() < kFeedBlocks ? blocks() : kFeedBlocks;
    feed_kernel<K, Real, Store><<<grid, BLOCK, 0, st>>>(P, state(B, cur), B.feed_part);
    feed_combine_kernel<<<1, 32, 0, st>>>(B.feed_part, (unsigned)grid, B.scal, P.feed_c);
    return cudaGetLastError();
  }
  // The partials of a step go to buffer `cur` (the parity of its input
  // state); with a fixed P0 the next launch combines them in block 0.
  // ---- TMA path (2-D, FP32 compute): maps per input parity, persistent grid
  static constexpr bool kTmaType =
      DIM == 2 && std::is_same<Real, float>::value && !IsHalf<Store>::value;
  TmaMaps maps[2];
  const void* map_key[2][5] = {};
  int tma_state = 0;  // 0 unknown, 1 usable, -1 not usable
  int tma_grid = 0;
  // default step kernel: the z-march for 3-D FP32 storage (fastest measured on
  // the 3-D bed), the staged-tile kernel otherwise
  int kernel_sel = (DIM == 3 && MODE == MODE_FP32) ? 4 : 0;
  long long wait_limit = kDefaultWaitCycles;
  void set_wait_limit(long long cycles) override { wait_limit = cycles; }
  SurrArgs surr;
  bool has_surr = false;

  bool set_surrogate(const SurrArgs& a) override {
    if constexpr (K != 6) {
      return false;
    } else {
      surr = a;
      has_surr = true;
      return true;
    }
  }

  cudaError_t chem_pass(Buffers& B, int cur, double* out, cudaStream_t st) override {
    if constexpr (K == 0) {
      return cudaErrorNotSupported;
    } else {
      if (!B.src) return cudaErrorInvalidValue;
      // the chemistry reads T, Y, phi and P0 only: one instantiation per
      // (K, compute type), shared by 2-D and 3-D and by both storage types
      const State<Real, Store> S = state(B, cur);
      State<Real, Real> C;
      std::memset(&C, 0, sizeof(C));
      C.T_in = S.T_in;
      C.Y_in = S.Y_in;
      C.phi = S.phi;
      C.scal = S.scal;
      return chem_pass_launch<K, Real>(P, C, static_cast<Real*>(B.src), has_surr ? &surr : nullptr,
                                       B.fb_idx, B.fb_count, B.chem_stats, out, st);
    }
  }

  bool select_kernel(int k, const Buffers& B, int cur) override {
    if (k == 0) { kernel_sel = 0; return true; }
    if (k == 1 && tma_usable(B, cur) && tma_usable(B, 1 - cur)) { kernel_sel = 1; return true; }
    if ((k == 2 || k == 3) && DIM == 2 && B.tile_ctr) { kernel_sel = k; return true; }
    if ((k == 4 || k == 5) && DIM == 3) { kernel_sel = k; return true; }
    return false;
  }

  // persistent z-march (3-D): grid = resident blocks per SM x SMs
  int mgrid[2] = {0, 0};
  template <bool PRE>
  cudaError_t step_march(Buffers& B, int cur, cudaStream_t st, const double* prev) {
    if constexpr (DIM == 3) {
      constexpr size_t smem = march_smem_bytes<K, Real, Store>();
      auto kern = step3d_march_kernel<K, Real, Store, PRE>;
      int& grid = mgrid[PRE ? 1 : 0];
      if (grid == 0) {
        int dev = 0, sms = 0, occ = 0;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
          e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, BLOCK, smem);
        if (e != cudaSuccess) return e;
        grid = std::max(1, occ) * sms;
        if (grid > B.slots) grid = (int)B.slots;
      }
      kern<<<grid, BLOCK, smem, st>>>(P, state(B, cur), p0_closed, prev, (unsigned)B.last_nb);
      B.last_nb = grid;
      return cudaGetLastError();
    } else {
      return cudaErrorNotSupported;
    }
  }

  // persistent 2-D step with tile shape T_ (kernels 2: 32 x 8, 3: 32 x 16)
  int pgrid[2] = {0, 0};
  template <class T_>
  cudaError_t step_persistent(Buffers& B, int cur, cudaStream_t st, const double* prev,
                              int& grid_cache) {
    if constexpr (DIM == 2) {
      constexpr size_t smem = step_smem_bytes<DIM, K, Real, Store, T_>();
      auto kern = step_persistent_kernel<DIM, K, Real, Store, T_>;
      if (grid_cache == 0) {
        int dev = 0, sms = 0, occ = 0;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
          e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, BLOCK, smem);
        if (e != cudaSuccess) return e;
        grid_cache = std::max(1, occ) * sms;
      }
      const int tiles = ((P.nx + T_::TX - 1) / T_::TX) * ((P.ny + T_::TY - 1) / T_::TY);
      if (tiles > B.slots) return cudaErrorInvalidValue;
      kern<<<std::min(grid_cache, tiles), BLOCK, smem, st>>>(
          P, state(B, cur), p0_closed, prev, (unsigned)B.last_nb, B.tile_ctr, cur);
      B.last_nb = tiles;
      return cudaGetLastError();
    } else {
      return cudaErrorNotSupported;
    }
  }
  int kernel() const override { return kernel_sel; }

  static constexpr bool kBatchable = DIM == 2 && K == 0;
  size_t batch_entry_bytes() const override {
    return kBatchable ? sizeof(BatchDom<K, Real, Store>) : 0;
  }
  void batch_entry(void* dst, const Buffers& B, int cur) const override {
    if constexpr (kBatchable) {
      BatchDom<K, Real, Store> e;
      std::memset(&e, 0, sizeof(e));
      e.P = P;
      e.S[0] = state(B, 0);
      e.S[1] = state(B, 1);
      e.p0_closed = p0_closed;
      e.cur0 = cur;
      std::memcpy(dst, &e, sizeof(e));
    }
  }
  template <int CFG>
  static int batch_occ_of() {
    using T_ = typename BatchShape<CFG>::T;
    int nb = 0;
    auto kern = batch_step_kernel<K, Real, Store, T_>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)batch_smem_bytes<K, Real, Store, T_>()) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, BLOCK,
                                                      batch_smem_bytes<K, Real, Store, T_>()) !=
            cudaSuccess)
      return 0;
    return nb;
  }
  int batch_occupancy(int cfg) const override {
    if constexpr (kBatchable) {
      return cfg == 0 ? batch_occ_of<0>() : cfg == 1 ? batch_occ_of<1>()
                                                      : cfg == 2 ? batch_occ_of<2>() : 0;
    } else {
      return 0;
    }
  }
  template <int CFG>
  static cudaError_t batch_launch_cfg(const void* entries, const int* tile_begin, int ndom,
                                      int grid, int flip, unsigned* ctr, cudaStream_t st) {
    using T_ = typename BatchShape<CFG>::T;
    batch_step_kernel<K, Real, Store, T_><<<grid, BLOCK, batch_smem_bytes<K, Real, Store, T_>(), st>>>(
        static_cast<const BatchDom<K, Real, Store>*>(entries), tile_begin, ndom, flip, ctr);
    return cudaGetLastError();
  }
  cudaError_t batch_launch(const void* entries, const int* tile_begin, int ndom, int cfg, int grid,
                           int flip, unsigned* ctr, cudaStream_t st) const override {
    if constexpr (kBatchable) {
      switch (cfg) {
        case 0: return batch_launch_cfg<0>(entries, tile_begin, ndom, grid, flip, ctr, st);
        case 1: return batch_launch_cfg<1>(entries, tile_begin, ndom, grid, flip, ctr, st);
        case 2: return batch_launch_cfg<2>(entries, tile_begin, ndom, grid, flip, ctr, st);
        default: return cudaErrorInvalidValue;
      }
    } else {
      return cudaErrorNotSupported;
    }
  }
  int batch_key() const override { return kBatchable ? 100 + MODE : -1; }

  bool tma_usable(const Buffers& B, int cur) {
    if constexpr (!kTmaType) {
      return false;
    } else {
      using LY = TmaLayout<K, Store>;
      if (tma_state < 0) return false;
      if (tma_state == 0) {
        // rows must be whole 16-byte units for every array the boxes read
        if (P.nx % (16 / (int)sizeof(Store)) != 0 || P.nx % 4 != 0 || !encode_tiled()) {
          tma_state = -1;
          return false;
        }
        auto kern = step_tma_kernel<K, Store>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)LY::smem_bytes) != cudaSuccess) {
          tma_state = -1;
          return false;
        }
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, BLOCK, LY::smem_bytes);
        const long long tiles = (long long)((P.nx + LY::TX - 1) / LY::TX) *
                                ((P.ny + LY::TY - 1) / LY::TY);
        if (per < 1 || sms < 1) {
          tma_state = -1;
          return false;
        }
        tma_grid = (int)std::min<long long>(tiles, (long long)sms * per);
        if (tma_grid > B.slots) tma_grid = (int)B.slots;
        tma_state = 1;
      }
      const void* key[5] = {B.g[cur], B.T[cur], B.Y[cur], B.Ts[cur], B.phi};
      bool same = true;
      for (int j = 0; j < 5; ++j) same = same && map_key[cur][j] == key[j];
      if (!same) {
        const unsigned long long nx = P.nx, ny = P.ny;
        const unsigned fb[3] = {(unsigned)LY::FW, (unsigned)LY::FH, (unsigned)(K > 0 ? K : 1)};
        const unsigned long long d2[2] = {nx, ny};
        const unsigned long long dY[3] = {nx, ny, (unsigned long long)(K > 0 ? K : 1)};
        const unsigned long long dg[3] = {nx, ny, 9ull};
        const unsigned pb[3] = {(unsigned)LY::PW, (unsigned)LY::PH, 1u};
        const CUtensorMapDataType gdt = sizeof(Store) == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                                           : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
        TmaMaps& m = maps[cur];
        const void* Ts = B.Ts[cur] ? B.Ts[cur] : B.T[cur];
        const void* Y = K > 0 ? B.Y[cur] : B.T[cur];
        bool ok = encode_map(&m.T, B.T[cur], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, 2, d2, fb) &&
                  encode_map(&m.phi, B.phi, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, 2, d2, fb) &&
                  encode_map(&m.Ts, Ts, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, 2, d2, fb) &&
                  (K > 0 ? encode_map(&m.Y, Y, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, 3, dY, fb)
                         : encode_map(&m.Y, Y, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, 2, d2, fb)) &&
                  encode_map(&m.g, B.g[cur], gdt, (int)sizeof(Store), 3, dg, pb);
        if (!ok) {
          tma_state = -1;
          return false;
        }
        for (int j = 0; j < 5; ++j) map_key[cur][j] = key[j];
      }
      return true;
    }
  }

  cudaError_t step_tma(Buffers& B, int cur, cudaStream_t st, const double* prev) {
    if constexpr (kTmaType) {
      using LY = TmaLayout<K, Store>;
      const int tiles_x = (P.nx + LY::TX - 1) / LY::TX;
      const int n_tiles = tiles_x * ((P.ny + LY::TY - 1) / LY::TY);
      const TmaMaps& m = maps[cur];
      step_tma_kernel<K, Store><<<tma_grid, BLOCK, LY::smem_bytes, st>>>(
          P, state(B, cur), p0_closed, prev, (unsigned)B.last_nb, m.T, m.phi, m.Ts, m.Y, m.g,
          tiles_x, n_tiles, wait_limit);
      B.last_nb = tma_grid;
      return cudaGetLastError();
    } else {
      return cudaErrorNotSupported;
    }
  }

  // One step's launches on stream st, with its host bookkeeping.
  cudaError_t one_step(Buffers& B, int& cur, cudaStream_t st, dim3 grid, size_t smem) {
    cudaError_t e = cudaSuccess;
    if constexpr (K > 0) {
      if (P.chem >= 2) {
        e = chem_pass(B, cur, nullptr, st);
        if (e != cudaSuccess) return e;
      }
    }
    const double* prev = (!p0_closed && B.pending)
                             ? B.partials + (size_t)4 * B.slots * B.last_parity : nullptr;
    if (kernel_sel == 1 && tma_usable(B, cur)) {
      e = step_tma(B, cur, st, prev);
      if (e != cudaSuccess) return e;
    } else if (kernel_sel == 2) {
      e = step_persistent<Tile<DIM, 32, 1>>(B, cur, st, prev, pgrid[0]);
      if (e != cudaSuccess) return e;
    } else if (kernel_sel == 3) {
      e = step_persistent<Tile<DIM, 32, 2>>(B, cur, st, prev, pgrid[1]);
      if (e != cudaSuccess) return e;
    } else if (kernel_sel == 4 || kernel_sel == 5) {
      e = kernel_sel == 5 ? step_march<true>(B, cur, st, prev) : step_march<false>(B, cur, st, prev);
      if (e != cudaSuccess) return e;
    } else {
      step_kernel<DIM, K, Real, Store><<<grid, BLOCK, smem, st>>>(P, state(B, cur), p0_closed,
                                                                   prev, (unsigned)B.last_nb);
      B.last_nb = step_blocks();
    }
    if (P.feed) {
      e = feed(B, cur, st);
      if (e != cudaSuccess) return e;
    }
    if (P.nscbc)
      outlet_kernel<Real><<<1, BLOCK, 0, st>>>(static_cast<const Real*>(B.ob), P.ny * P.nz,
                                               B.scal, P.nscbc_K);
    ++B.nstep;
    if (P.moving) {
      e = phase(B, B.nstep, st);
      if (e != cudaSuccess) return e;
    }
    B.pending = p0_closed ? 0 : 1;
    B.last_parity = cur;
    cur = 1 - cur;
    return cudaGetLastError();
  }

  // Steps are replayed in pairs from a CUDA graph when a call asks for many:
  // after two plain steps every launch argument repeats every second step
  // (the ping-pong buffers, the reduction's parity and block count), and a
  // graph launch of the pair costs one launch instead of one per kernel
  // (the small domains are launch-bound).  Not for moving solids, whose
  // phase kernel takes the step number as an argument.
  static constexpr int kGraphMinSteps = 32;
  cudaStream_t cap_st = nullptr;  // capture stream, created on first use
  ~LauncherImpl() override {
    if (cap_st) cudaStreamDestroy(cap_st);
  }

  cudaError_t step(Buffers& B, int& cur, int nsteps, cudaStream_t st) override {
    constexpr size_t smem = step_smem_bytes<DIM, K, Real, Store>();
    cudaError_t e = cudaFuncSetAttribute(step_kernel<DIM, K, Real, Store>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid = step_grid();
    if (kernel_sel >= 2 && nsteps > 0) {
      // both counters start at zero; consecutive steps then clear each other's
      e = cudaMemsetAsync(B.tile_ctr, 0, 2 * sizeof(unsigned), st);
      if (e != cudaSuccess) return e;
    }
    int n = 0;
    if (nsteps >= kGraphMinSteps && !P.moving) {
      for (; n < 2; ++n) {
        e = one_step(B, cur, st, grid, smem);
        if (e != cudaSuccess) return e;
      }
      if (!cap_st) {
        e = cudaStreamCreateWithFlags(&cap_st, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
      }
      const int cur0 = cur;
      const long long nstep0 = B.nstep;
      const int pending0 = B.pending, parity0 = B.last_parity;
      const long long last_nb0 = B.last_nb;
      cudaGraph_t g = nullptr;
      cudaGraphExec_t x = nullptr;
      e = cudaStreamBeginCapture(cap_st, cudaStreamCaptureModeRelaxed);
      if (e == cudaSuccess) {
        cudaError_t e1 = one_step(B, cur, cap_st, grid, smem);
        if (e1 == cudaSuccess) e1 = one_step(B, cur, cap_st, grid, smem);
        e = cudaStreamEndCapture(cap_st, &g);
        if (e == cudaSuccess) e = e1;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
      if (e == cudaSuccess) {
        // the capture advanced the bookkeeping by the pair the first launch runs
        const int pairs = (nsteps - n) / 2;
        for (int q = 0; q < pairs && e == cudaSuccess; ++q) {
          e = cudaGraphLaunch(x, st);
          if (q > 0) B.nstep += 2;
        }
        n += 2 * pairs;
      } else {
        // capture refused: undo its bookkeeping, step without a graph
        cudaGetLastError();
        cur = cur0;
        B.nstep = nstep0;
        B.pending = pending0;
        B.last_parity = parity0;
        B.last_nb = last_nb0;
        e = cudaSuccess;
      }
      if (x) cudaGraphExecDestroy(x);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) return e;
    }
    for (; n < nsteps; ++n) {
      e = one_step(B, cur, st, grid, smem);
      if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
  }
  cudaError_t finalize(Buffers& B, cudaStream_t st) override {
    if (!B.pending) return cudaSuccess;
    finalize_kernel<<<1, 32, 0, st>>>(B.partials + (size_t)4 * B.slots * B.last_parity,
                                      (unsigned)B.last_nb, B.scal, P.eos_c, P.inv_rho_ref);
    B.pending = 0;
    return cudaGetLastError();
  }
  cudaError_t moments(const Buffers& B, int cur, double* u, double* rho, double* ph,
                      cudaStream_t st) override {
    moments_kernel<DIM, K, Real, Store><<<blocks(), BLOCK, 0, st>>>(P, state(B, cur), u, rho, ph);
    return cudaGetLastError();
  }
  float g_scale() const override { return float(P.g_scale); }
  int diag_blocks() const override { return blocks(); }
  cudaError_t diagnostics(const Buffers& B, int cur, double* part, double* out,
                          cudaStream_t st) override {
    diag_kernel<DIM, K, Real, Store><<<blocks(), BLOCK, 0, st>>>(P, state(B, cur), part);
    diag_combine_kernel<<<1, 32, 0, st>>>(part, blocks(), out);
    return cudaGetLastError();
  }
};

// factories, one per translation unit (compiled in parallel)
Launcher* make_launcher_2d_fp64(int K, const pflb_domain_desc& d, const pflb_mechanism& m);
Launcher* make_launcher_2d_fp32(int K, const pflb_domain_desc& d, const pflb_mechanism& m);
Launcher* make_launcher_2d_fp16(int K, const pflb_domain_desc& d, const pflb_mechanism& m);
Launcher* make_launcher_3d_fp64(int K, const pflb_domain_desc& d, const pflb_mechanism& m);
Launcher* make_launcher_3d_fp32(int K, const pflb_domain_desc& d, const pflb_mechanism& m);
Launcher* make_launcher_3d_fp16(int K, const pflb_domain_desc& d, const pflb_mechanism& m);

}  // namespace pflb
