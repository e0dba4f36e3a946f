// pflb_kernels.cuh -- CUDA kernels of the PF-LB-FD time step (sm_103a).
//
// One fused kernel advances one time step of the low-Mach phase-field /
// lattice-Boltzmann / finite-difference model (arXiv 2310.17214, Sec. 3.3):
//   pull streaming of the pressure-based populations with the boundary rules,
//   moments with the implicit diffuse-interface drag (Sec. 3.2.1), the FD
//   transport of T, Y_k and the solid temperature with the reaction source
//   (Sec. 3.2.2 eq. 8, Sec. 3.3 eqs. diffusion-heat-flux-3,
//   energy-transport-DI-version, 9), the divergence from the low-Mach
//   constraint, the source Xi (eq. body-force) and BGK collision (eqs.
//   eq-pop-f, eq-pop-g), and the FP64 reduction for P0 (Sec. 3.1) finished
//   by the last block to arrive.
//
// Storage is SoA: g[i*N + cell], Y[k*N + cell]; cell = x + nx*(y + ny*z).
// Threads map to consecutive x so every population / field load of a warp
// is a contiguous (or one-element-shifted) 128-byte line.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace pflb {

constexpr int KMAX = 8;
constexpr int JMAX = 4;
constexpr int BLOCK = 256;

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_INLET = 2, BC_OUTLET = 3 };
enum { MODE_FP64 = 0, MODE_FP32 = 1, MODE_FP16 = 2 };

// ------------------------------------------------------------- lattices
// D2Q9 and D3Q19 velocity sets and weights (cs^2 = 1/3).  The direction
// order is the library's storage order (reported by pflb_lattice).
template <int DIM> struct Lattice;

template <> struct Lattice<2> {
  static constexpr int Q = 9;
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int t[9][3] = {{0, 0, 0},  {1, 0, 0},  {0, 1, 0},   {-1, 0, 0}, {0, -1, 0},
                             {1, 1, 0},  {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
    return t[i][a];
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr int opp(int i) {
    constexpr int t[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    return t[i];
  }
};

template <> struct Lattice<3> {
  static constexpr int Q = 19;
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int t[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                              {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                              {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                              {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    return t[i][a];
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr int opp(int i) {
    constexpr int t[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
    return t[i];
  }
};

// ------------------------------------------------------------ parameters
// Everything in lattice units, converted once on the host (pflb_api.cu).
template <class Real, int K>
struct Params {
  static constexpr int KK = K > 0 ? K : 1;
  int nx, ny, nz, N;
  int bc[6];
  Real wall_u[6][3];
  Real wall_T[6];
  double eos_c;            // rho* = P0 Mw eos_c / T, eos_c = 1 / (R rho_ref)
  double inv_rho_ref;      // dP0 / rho_ref (J/kg) in the T equation
  Real mu_lat;             // mu_ref dt / (rho_ref dx^2)
  int sutherland;
  Real inv_suth_T, suth_S, suth_TS;  // suth_TS = suth_T + suth_S
  Real inv_Pr;
  Real Au_eta2, AT_eta2;   // A_u / eta^2, A_T / eta^2
  Real Fb[3];
  int inlet_parabolic;
  Real u_in, T_in;
  Real Y_in[KK];
  Real M0, cp0;
  Real invM[KK], cp[KK], hf[KK], Dlat[KK];
  int D_Tdep;
  Real inv_DTref, D_exp;
  int Ts_field;
  Real Ts_uniform, Cs, Lams;  // solid rho cp / rho_ref, lambda_s dt / (rho_ref dx^2)
  Real phi_min;
  int chem, J;
  Real A_lat[JMAX];        // A dt / rho_ref
  Real b[JMAX], EaR[JMAX];
  Real order[JMAX][KK], stoichM[JMAX][KK];  // stoichM = s_kj M_k
  Real rho_ref_M[KK];      // rho_ref / M_k (concentration from rho* Y_k)
  Real g_scale, g_inv_scale;  // FP16 storage scale (power of two)
};

struct DevScalars {
  double P0, P0_prev, mass, I, flux_in, flux_out, mass_now;
  long long step;
  int status;
  int pad;
};

template <class Real, class Store>
struct State {
  const Store* __restrict__ g_in;
  Store* __restrict__ g_out;
  const Real* __restrict__ T_in;
  Real* __restrict__ T_out;
  const Real* __restrict__ Y_in;
  Real* __restrict__ Y_out;
  const Real* __restrict__ Ts_in;
  Real* __restrict__ Ts_out;
  const Real* __restrict__ phi;
  DevScalars* scal;
  double* partials;        // [gridDim.x][4]
  unsigned* counter;
};

// ----------------------------------------------------- storage codecs
template <class Store, class Real> struct Codec;
template <> struct Codec<double, double> {
  __device__ static double load(const double* p, double, double) { return __ldg(p); }
  __device__ static void store(double* p, double v, double, double) { *p = v; }
};
template <> struct Codec<float, float> {
  __device__ static float load(const float* p, float, float) { return __ldg(p); }
  __device__ static void store(float* p, float v, float, float) { *p = v; }
};
// FP16: h = g / w * scale (weights folded so every direction has the same range)
template <> struct Codec<__half, float> {
  __device__ static float load(const __half* p, float w_over_scale, float) {
    return __half2float(__ldg(p)) * w_over_scale;
  }
  __device__ static void store(__half* p, float v, float, float scale_over_w) {
    *p = __float2half_rn(v * scale_over_w);
  }
};

// ------------------------------------------------------------ helpers
template <class Real> __device__ __forceinline__ Real rcp(Real x) { return Real(1) / x; }

template <class Real, int K>
struct Props {
  Real rho, cp, lam, Mw;
  Real D[Params<Real, K>::KK];
};

// EOS (Sec. 3.1), Sutherland / constant viscosity and lambda = mu cp / Pr
// (Sec. 4, eqs. muT, lambdaT), D_k = Dref (T / D_Tref)^D_exp.
template <class Real, int K>
__device__ __forceinline__ Real viscosity(const Params<Real, K>& P, Real T) {
  if (!P.sutherland) return P.mu_lat;
  Real t = T * P.inv_suth_T;
  return P.mu_lat * t * sqrt(t) * P.suth_TS / (T + P.suth_S);
}

template <class Real, int K>
__device__ __forceinline__ void props(const Params<Real, K>& P, Real P0, Real T, const Real* Y,
                                      bool need_D, Props<Real, K>& o) {
  Real Mw, cp;
  if constexpr (K == 0) {
    Mw = P.M0;
    cp = P.cp0;
  } else {
    Real s = 0, c = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      s += Y[k] * P.invM[k];
      c += Y[k] * P.cp[k];
    }
    Mw = Real(1) / s;
    cp = c;
  }
  o.Mw = Mw;
  o.cp = cp;
  o.rho = P0 * Mw * Real(P.eos_c) / T;
  o.lam = viscosity(P, T) * cp * P.inv_Pr;
  if constexpr (K > 0) {
    if (need_D) {
      Real f = P.D_Tdep ? pow(T * P.inv_DTref, P.D_exp) : Real(1);
#pragma unroll
      for (int k = 0; k < K; ++k) o.D[k] = P.Dlat[k] * f;
    }
  }
}

template <class Real, int K>
__device__ __forceinline__ Real mixture_Mw(const Params<Real, K>& P, const Real* Y) {
  if constexpr (K == 0) {
    return P.M0;
  } else {
    Real s = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) s += Y[k] * P.invM[k];
    return Real(1) / s;
  }
}

// Explicit Arrhenius rates (Sec. 3.2.2 eq. 8, Sec. 3.3 eq. 9), returned per
// lattice step per rho_ref: om[k] = omega_k dt / rho_ref, omT likewise (J/kg).
template <class Real, int K>
__device__ __forceinline__ void rates(const Params<Real, K>& P, Real T, const Real* Y, Real rho,
                                      Real* om, Real& omT) {
#pragma unroll
  for (int k = 0; k < K; ++k) om[k] = 0;
  Real C[Params<Real, K>::KK];
#pragma unroll
  for (int k = 0; k < K; ++k) C[k] = rho * P.rho_ref_M[k] * (Y[k] > Real(0) ? Y[k] : Real(0));
  for (int j = 0; j < P.J; ++j) {
    Real q = P.A_lat[j] * exp(-P.EaR[j] / T);
    if (P.b[j] != Real(0)) q *= pow(T, P.b[j]);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      Real o = P.order[j][k];
      if (o == Real(1)) q *= C[k];
      else if (o == Real(2)) q *= C[k] * C[k];
      else if (o != Real(0)) q *= pow(C[k], o);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) om[k] += P.stoichM[j][k] * q;
  }
  Real wt = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) wt -= P.hf[k] * om[k];
  omT = wt;
}

template <class Real, int K>
struct Nb {
  Real T, phi, Ts;
  Real Y[Params<Real, K>::KK];
};

// Neighbour (or ghost) state along axis a, side s.  Periodic faces wrap;
// the inlet ghost carries (T_in, Y_in); a wall with a set temperature
// carries it; other faces copy the cell.  phi, Ts of ghosts are the cell's.
template <int DIM, class Real, class Store, int K>
__device__ __forceinline__ void load_nb(const Params<Real, K>& P, const State<Real, Store>& S,
                                        int c, const int xyz[3], int a, int s, const Nb<Real, K>& own,
                                        Nb<Real, K>& o) {
  const int n = a == 0 ? P.nx : (a == 1 ? P.ny : P.nz);
  const int stride = a == 0 ? 1 : (a == 1 ? P.nx : P.nx * P.ny);
  int q = xyz[a] + s;
  int face = 2 * a + (s > 0 ? 1 : 0);
  int nc;
  if (q >= 0 && q < n) {
    nc = c + s * stride;
  } else if (P.bc[face] == BC_PERIODIC) {
    nc = c + s * stride - s * n * stride;
  } else {
    o = own;
    if (P.bc[face] == BC_INLET) {
      o.T = P.T_in;
#pragma unroll
      for (int k = 0; k < K; ++k) o.Y[k] = P.Y_in[k];
    } else if (P.bc[face] == BC_WALL && P.wall_T[face] > Real(0)) {
      o.T = P.wall_T[face];
    }
    return;
  }
  o.T = __ldg(S.T_in + nc);
  o.phi = __ldg(S.phi + nc);
  o.Ts = P.Ts_field ? __ldg(S.Ts_in + nc) : P.Ts_uniform;
#pragma unroll
  for (int k = 0; k < K; ++k) o.Y[k] = __ldg(S.Y_in + (size_t)k * P.N + nc);
}

template <class Real, int K>
__device__ __forceinline__ Real inlet_u(const Params<Real, K>& P, const int xyz[3], int dim) {
  Real u = P.u_in;
  if (!P.inlet_parabolic) return u;
  for (int a = 1; a < dim; ++a) {
    if (P.bc[2 * a] != BC_WALL) continue;
    Real n = Real(a == 1 ? P.ny : P.nz);
    Real s = Real(xyz[a]) + Real(0.5);
    u *= Real(4) * s * (n - s) / (n * n);
  }
  return u;
}

// Pull streaming of every population into the cell, with the boundary rules:
// half-way bounce-back on walls (moving walls add 2 w rho c.u_w), the inlet
// as a moving wall with the inlet velocity and inlet density, the outlet as
// anti-bounce-back at P_h = 0 with wall velocity uw.
template <int DIM, class Real, class Store, int K>
__device__ __forceinline__ void pull(const Params<Real, K>& P, const State<Real, Store>& S, int c,
                                     const int xyz[3], bool edge, Real rho_c, Real rho_in,
                                     const Real* uw, Real* gin) {
  using L = Lattice<DIM>;
  const int sy = P.nx, sz = P.nx * P.ny;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const Real wos = Real(L::w(i)) * P.g_inv_scale;
    if (!edge) {
      int src = c - L::c(i, 0) - L::c(i, 1) * sy - (DIM == 3 ? L::c(i, 2) * sz : 0);
      gin[i] = Codec<Store, Real>::load(S.g_in + (size_t)i * P.N + src, wos, 0);
      continue;
    }
    int sx[3] = {xyz[0] - L::c(i, 0), xyz[1] - L::c(i, 1), DIM == 3 ? xyz[2] - L::c(i, 2) : 0};
    int wall = -1;
    bool inlet = false, outlet = false;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int n = a == 0 ? P.nx : (a == 1 ? P.ny : P.nz);
      if (sx[a] < 0 || sx[a] >= n) {
        int face = 2 * a + (sx[a] >= n ? 1 : 0);
        int bc = P.bc[face];
        if (bc == BC_PERIODIC) sx[a] = sx[a] < 0 ? sx[a] + n : sx[a] - n;
        else if (bc == BC_WALL) { if (wall < 0) wall = face; }
        else if (bc == BC_INLET) inlet = true;
        else outlet = true;
      }
    }
    const int ib = L::opp(i);
    if (wall >= 0 || inlet || outlet) {
      const Real wob = Real(L::w(ib)) * P.g_inv_scale;
      Real own = Codec<Store, Real>::load(S.g_in + (size_t)ib * P.N + c, wob, 0);
      if (wall >= 0) {
        Real cu = 0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) cu += Real(L::c(i, a)) * P.wall_u[wall][a];
        gin[i] = own + Real(2) * Real(L::w(i)) * rho_c * cu;
      } else if (inlet) {
        Real cu = Real(L::c(i, 0)) * inlet_u(P, xyz, DIM);
        gin[i] = own + Real(2) * Real(L::w(i)) * rho_in * cu;
      } else {
        Real cu = 0, uu = 0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
          cu += Real(L::c(i, a)) * uw[a];
          uu += uw[a] * uw[a];
        }
        gin[i] = -own + Real(L::w(i)) * rho_c * (Real(3) * cu * cu - uu);
      }
    } else {
      int src = sx[0] + P.nx * (sx[1] + P.ny * sx[2]);
      gin[i] = Codec<Store, Real>::load(S.g_in + (size_t)i * P.N + src, wos, 0);
    }
  }
}

// Block-wide FP64 sum of 4 values; result valid in thread 0.
__device__ __forceinline__ void block_sum4(double v[4]) {
  __shared__ double sh[BLOCK / 32][4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < 4; ++j) sh[wid][j] = v[j];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      double t = lane < (int)(blockDim.x >> 5) ? sh[lane][j] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      v[j] = t;
    }
  }
}

// Deterministic finish of the per-block partials by the last block to
// arrive: a fixed-order strided sum followed by a fixed tree.  Updates the
// scalar state (P0 closure, diagnostics) and re-arms the counter.
__device__ __forceinline__ void finish_reduction(double* partials, unsigned* counter,
                                                 DevScalars* scal, int p0_closed, bool is_init,
                                                 double init_P0, double eos_c) {
  __shared__ bool last;
  __threadfence();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double v[4] = {0, 0, 0, 0};
  const volatile double* vp = partials;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] += vp[4 * b + j];
  block_sum4(v);
  if (threadIdx.x == 0) {
    const double I = v[0];
    if (is_init) {
      scal->P0 = init_P0;
      scal->P0_prev = init_P0;
      scal->mass = init_P0 * I * eos_c;
      scal->I = I;
      scal->flux_in = scal->flux_out = 0;
      scal->mass_now = v[3];
      scal->step = 0;
      scal->status = 0;
    } else {
      const double P0 = scal->P0;
      double P0n = P0;
      if (p0_closed) P0n = scal->mass / (I * eos_c);
      scal->P0_prev = P0;
      scal->P0 = P0n;
      scal->I = I;
      scal->flux_in = v[1];
      scal->flux_out = v[2];
      scal->mass_now = v[3];
      scal->step += 1;
      if (!(I == I) || !(P0n == P0n) || I <= 0.0) scal->status = -5;
    }
    *counter = 0u;
  }
}

// ------------------------------------------------------ the fused step
template <int DIM, int K, class Real, class Store>
__global__ void __launch_bounds__(BLOCK)
step_kernel(const Params<Real, K> P, const State<Real, Store> S, int p0_closed) {
  using L = Lattice<DIM>;
  constexpr int Q = L::Q;
  constexpr int KK = Params<Real, K>::KK;
  constexpr Real CS2 = Real(1) / Real(3);
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = c < P.N;

  const double P0d = S.scal->P0, P0pd = S.scal->P0_prev;
  const Real P0 = Real(P0d);
  const Real dlnP0 = Real((P0d - P0pd) / P0d);
  const Real dP0r = Real((P0d - P0pd) * P.inv_rho_ref);

  double red[4] = {0, 0, 0, 0};
  if (active) {
    int xyz[3];
    xyz[0] = c % P.nx;
    const int yz = c / P.nx;
    xyz[1] = yz % P.ny;
    xyz[2] = DIM == 3 ? yz / P.ny : 0;
    bool edge = xyz[0] == 0 || xyz[0] == P.nx - 1 || xyz[1] == 0 || xyz[1] == P.ny - 1;
    if (DIM == 3) edge = edge || xyz[2] == 0 || xyz[2] == P.nz - 1;

    // own state
    Nb<Real, K> v0;
    v0.T = __ldg(S.T_in + c);
    v0.phi = __ldg(S.phi + c);
    v0.Ts = P.Ts_field ? __ldg(S.Ts_in + c) : P.Ts_uniform;
#pragma unroll
    for (int k = 0; k < K; ++k) v0.Y[k] = __ldg(S.Y_in + (size_t)k * P.N + c);
    Props<Real, K> d0;
    props(P, P0, v0.T, v0.Y, true, d0);
    const Real phis = v0.phi, phif = Real(1) - v0.phi;
    const Real mu = viscosity(P, v0.T);
    const Real Kd = P.Au_eta2 * mu * phif * phis * phis;
    const Real rho = d0.rho;

    // (a1) pull streaming and moments, implicit drag
    Real rho_in = 0;
    if (edge) {
      Real Yin[KK];
#pragma unroll
      for (int k = 0; k < K; ++k) Yin[k] = P.Y_in[k];
      rho_in = P0 * mixture_Mw(P, Yin) * Real(P.eos_c) / P.T_in;
    }
    Real gin[Q];
    Real u[3] = {0, 0, 0};
    Real uw[3] = {0, 0, 0};
    const bool outlet_cell = P.bc[1] == BC_OUTLET && xyz[0] == P.nx - 1;
    const Real inv_rk = Real(1) / (rho + Real(0.5) * Kd);
    for (int pass = 0; pass < (outlet_cell ? 2 : 1); ++pass) {
      pull<DIM>(P, S, c, xyz, edge, rho, rho_in, uw, gin);
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        Real m = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i)
          if (L::c(i, a) != 0) m += Real(L::c(i, a)) * gin[i];
        u[a] = (m * Real(3) + Real(0.5) * P.Fb[a]) * inv_rk;
        uw[a] = u[a];
      }
    }

    // neighbours for the FD stencils and grad(rho)
    Nb<Real, K> vm[DIM], vp[DIM];
    Props<Real, K> dm[DIM], dp[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      load_nb<DIM>(P, S, c, xyz, a, -1, v0, vm[a]);
      load_nb<DIM>(P, S, c, xyz, a, +1, v0, vp[a]);
      props(P, P0, vm[a].T, vm[a].Y, true, dm[a]);
      props(P, P0, vp[a].T, vp[a].Y, true, dp[a]);
    }

    const bool fluid_on = phif >= P.phi_min;
    const bool solid_on = P.Ts_field ? (phis >= P.phi_min) : true;
    Real SI = 0;
    if (fluid_on && solid_on) SI = P.AT_eta2 * d0.lam * phif * phis * phis * (v0.Ts - v0.T);

    // (c) reaction source
    Real om[KK], omT = 0;
#pragma unroll
    for (int k = 0; k < KK; ++k) om[k] = 0;
    if constexpr (K > 0) {
      if (P.chem == 1) rates(P, v0.T, v0.Y, rho, om, omT);
    }

    // (b) FD transport: species
    Real Yn[KK];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (!fluid_on) { Yn[k] = v0.Y[k]; continue; }
      const Real kc = phif * rho * d0.D[k];
      Real adv = 0, dif = 0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        adv += u[a] > Real(0) ? u[a] * (v0.Y[k] - vm[a].Y[k]) : u[a] * (vp[a].Y[k] - v0.Y[k]);
        const Real km = Real(0.5) * (kc + (Real(1) - vm[a].phi) * dm[a].rho * dm[a].D[k]);
        const Real kp = Real(0.5) * (kc + (Real(1) - vp[a].phi) * dp[a].rho * dp[a].D[k]);
        dif += kp * (vp[a].Y[k] - v0.Y[k]) - km * (v0.Y[k] - vm[a].Y[k]);
      }
      const Real rhs = -phif * rho * adv + dif + phif * om[k];
      Yn[k] = v0.Y[k] + rhs / (phif * rho);
    }

    // (b) FD transport: temperature
    Real Tn;
    if (fluid_on) {
      Real adv = 0, dif = 0, cross = 0;
      const Real kc = phif * d0.lam;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        adv += u[a] > Real(0) ? u[a] * (v0.T - vm[a].T) : u[a] * (vp[a].T - v0.T);
        const Real km = Real(0.5) * (kc + (Real(1) - vm[a].phi) * dm[a].lam);
        const Real kp = Real(0.5) * (kc + (Real(1) - vp[a].phi) * dp[a].lam);
        dif += kp * (vp[a].T - v0.T) - km * (v0.T - vm[a].T);
        const Real gT = Real(0.5) * (vp[a].T - vm[a].T);
#pragma unroll
        for (int k = 0; k < K; ++k)
          cross += P.cp[k] * d0.D[k] * Real(0.5) * (vp[a].Y[k] - vm[a].Y[k]) * gT;
      }
      const Real rhs = -phif * rho * d0.cp * adv + dif + phif * (rho * cross + dP0r + omT + SI);
      Tn = v0.T + rhs / (phif * rho * d0.cp);
    } else {
      Tn = v0.Ts;
    }

    // solid temperature
    if (P.Ts_field) {
      Real Tsn = v0.Ts;
      if (phis >= P.phi_min) {
        Real dif = 0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
          const Real km = Real(0.5) * (phis + vm[a].phi) * P.Lams;
          const Real kp = Real(0.5) * (phis + vp[a].phi) * P.Lams;
          dif += kp * (vp[a].Ts - v0.Ts) - km * (v0.Ts - vm[a].Ts);
        }
        Tsn = v0.Ts + (dif - phif * SI) / (phis * P.Cs);
      }
      S.Ts_out[c] = Tsn;
    }

    // low-Mach divergence D = (1/T) dT + Mw sum dY_k / M_k - dP0 / P0
    Real D = (Tn - v0.T) / v0.T;
    if constexpr (K > 0) {
      Real sY = 0;
#pragma unroll
      for (int k = 0; k < K; ++k) sY += (Yn[k] - v0.Y[k]) * P.invM[k];
      D += d0.Mw * sY;
    }
    D -= dlnP0;

    // (a) source and BGK collision
    Real G[3] = {0, 0, 0}, F[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      G[a] = CS2 * Real(0.5) * (dp[a].rho - dm[a].rho);
      F[a] = P.Fb[a] - Kd * u[a];
    }
    Real sg = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) sg += gin[i];
    const Real Ph = sg + Real(0.5) * rho * CS2 * D;
    const Real omega = Real(1) / (Real(0.5) + mu / (rho * CS2));
    const Real src_w = Real(1) - Real(0.5) * omega;
    Real uu = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) uu += u[a] * u[a];
    const Real rD = rho * CS2 * D;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const Real w = Real(L::w(i));
      Real cu = 0;
#pragma unroll
      for (int a = 0; a < DIM; ++a)
        if (L::c(i, a) != 0) cu += Real(L::c(i, a)) * u[a];
      // f_eq / rho - w = w e,   g_eq = w (P_h + rho (cu + 3/2 cu^2 - uu/2))
      const Real e = Real(3) * cu + Real(4.5) * cu * cu - Real(1.5) * uu;
      const Real geq = w * (Ph + rho * (cu + Real(1.5) * cu * cu - Real(0.5) * uu));
      Real xs = 0;
#pragma unroll
      for (int a = 0; a < DIM; ++a)
        xs += (Real(L::c(i, a)) - u[a]) * (G[a] * e + F[a] * (Real(1) + e));
      const Real xi = w * (xs + rD);
      const Real g = gin[i] + omega * (geq - gin[i]) + src_w * xi;
      Codec<Store, Real>::store(S.g_out + (size_t)i * P.N + c, g, 0, P.g_scale / w);
    }

    S.T_out[c] = Tn;
#pragma unroll
    for (int k = 0; k < K; ++k) S.Y_out[(size_t)k * P.N + c] = Yn[k];

    // (d) contributions to the FP64 reduction
    const Real Mwn = mixture_Mw(P, Yn);
    red[0] = double(phif) * double(Mwn) / double(Tn);
    const double fx = double(phif) * double(rho) * double(u[0]);
    if (xyz[0] == 0 && P.bc[0] == BC_INLET) red[1] = fx;
    if (outlet_cell) red[2] = fx;
    red[3] = double(phif) * double(rho);
  }
  block_sum4(red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) S.partials[4 * blockIdx.x + j] = red[j];
  }
  finish_reduction(S.partials, S.counter, S.scal, p0_closed, false, 0.0, P.eos_c);
}

// ------------------------------------------------ initial equilibrium
// g = g_eq(P_h = 0, rho, u); reduction of I = sum phi_f Mw / T for the mass m.
template <int DIM, int K, class Real, class Store>
__global__ void __launch_bounds__(BLOCK)
init_kernel(const Params<Real, K> P, const State<Real, Store> S, const Real* __restrict__ u_init,
            double P0_init) {
  using L = Lattice<DIM>;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double red[4] = {0, 0, 0, 0};
  if (c < P.N) {
    Real T = S.T_in[c];
    Real Y[Params<Real, K>::KK];
#pragma unroll
    for (int k = 0; k < K; ++k) Y[k] = S.Y_in[(size_t)k * P.N + c];
    const Real Mw = mixture_Mw(P, Y);
    const Real rho = Real(P0_init) * Mw * Real(P.eos_c) / T;
    Real u[3] = {0, 0, 0};
    if (u_init)
      for (int a = 0; a < DIM; ++a) u[a] = u_init[(size_t)a * P.N + c];
    Real uu = 0;
    for (int a = 0; a < DIM; ++a) uu += u[a] * u[a];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const Real w = Real(L::w(i));
      Real cu = 0;
      for (int a = 0; a < DIM; ++a) cu += Real(L::c(i, a)) * u[a];
      const Real geq = w * rho * (cu + Real(1.5) * cu * cu - Real(0.5) * uu);
      Codec<Store, Real>::store(S.g_out + (size_t)i * P.N + c, geq, 0, P.g_scale / w);
    }
    const Real phif = Real(1) - S.phi[c];
    red[0] = double(phif) * double(Mw) / double(T);
    red[3] = double(phif) * double(rho);
  }
  block_sum4(red);
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < 4; ++j) S.partials[4 * blockIdx.x + j] = red[j];
  finish_reduction(S.partials, S.counter, S.scal, 0, true, P0_init, P.eos_c);
}

// --------------------------------------------------- moments (get_fields)
// u, rho and sum g that the next step sees (pull + boundary rules + drag).
template <int DIM, int K, class Real, class Store>
__global__ void __launch_bounds__(BLOCK)
moments_kernel(const Params<Real, K> P, const State<Real, Store> S, double* __restrict__ u_out,
               double* __restrict__ rho_out, double* __restrict__ ph_out) {
  using L = Lattice<DIM>;
  constexpr int Q = L::Q;
  constexpr int KK = Params<Real, K>::KK;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P.N) return;
  const Real P0 = Real(S.scal->P0);
  int xyz[3];
  xyz[0] = c % P.nx;
  xyz[1] = (c / P.nx) % P.ny;
  xyz[2] = DIM == 3 ? c / (P.nx * P.ny) : 0;
  Real T = S.T_in[c];
  Real Y[KK];
#pragma unroll
  for (int k = 0; k < K; ++k) Y[k] = S.Y_in[(size_t)k * P.N + c];
  const Real rho = P0 * mixture_Mw(P, Y) * Real(P.eos_c) / T;
  const Real phis = S.phi[c];
  const Real Kd = P.Au_eta2 * viscosity(P, T) * (Real(1) - phis) * phis * phis;
  Real Yin[KK];
#pragma unroll
  for (int k = 0; k < K; ++k) Yin[k] = P.Y_in[k];
  const Real rho_in = P0 * mixture_Mw(P, Yin) * Real(P.eos_c) / P.T_in;
  const bool outlet_cell = P.bc[1] == BC_OUTLET && xyz[0] == P.nx - 1;
  Real gin[Q], u[3] = {0, 0, 0}, uw[3] = {0, 0, 0};
  for (int pass = 0; pass < (outlet_cell ? 2 : 1); ++pass) {
    pull<DIM>(P, S, c, xyz, true, rho, rho_in, uw, gin);
    for (int a = 0; a < DIM; ++a) {
      Real m = 0;
      for (int i = 0; i < Q; ++i) m += Real(L::c(i, a)) * gin[i];
      u[a] = (m * Real(3) + Real(0.5) * P.Fb[a]) / (rho + Real(0.5) * Kd);
      uw[a] = u[a];
    }
  }
  Real sg = 0;
  for (int i = 0; i < Q; ++i) sg += gin[i];
  for (int a = 0; a < DIM; ++a) u_out[(size_t)a * P.N + c] = double(u[a]);
  rho_out[c] = double(rho);
  ph_out[c] = double(sg);
}

}  // namespace pflb
