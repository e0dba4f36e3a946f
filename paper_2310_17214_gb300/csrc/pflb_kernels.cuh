// pflb_kernels.cuh -- CUDA kernels of the PF-LB-FD time step (sm_103a).
//
// One fused kernel advances one time step of the low-Mach phase-field /
// lattice-Boltzmann / finite-difference model (arXiv 2310.17214, Sec. 3.3):
//   pull streaming of the pressure-based populations with the boundary rules,
//   moments with the implicit diffuse-interface drag (Sec. 3.2.1), FD
//   transport of T, Y_k and the solid temperature with the reaction source
//   (Sec. 3.2.2 eq. 8, Sec. 3.3 eqs. diffusion-heat-flux-3,
//   energy-transport-DI-version, 9), the divergence from the low-Mach
//   constraint, the source Xi (eq. body-force) and BGK collision (eqs.
//   eq-pop-f, eq-pop-g), and the FP64 reduction for P0 (Sec. 3.1) finished by
//   the last block to arrive.
//
// Layout: SoA in HBM, g[i*N + cell], Y[k*N + cell]; cell = x + nx*(y + ny*z).
// A block owns a TX x TY tile of one or more z-planes.  It stages T, Y, phi,
// Ts of the tile plus a one-cell halo in shared memory and evaluates the
// per-cell properties (EOS density, viscosity, conductivity, diffusivity
// factor) once per staged cell; the FD stencils and grad(rho) then read their
// neighbours from shared memory.  In 3-D the block marches along z with a
// ring of three staged planes (2.5-D blocking).  The populations are pulled
// straight from HBM: warps map to 32 consecutive x, so every load is a
// contiguous or one-element-shifted 128-byte line.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace pflb {

constexpr int KMAX = 8;
constexpr int JMAX = 4;
constexpr int BLOCK = 256;  // threads per block (one cell each per plane)
// default bound of a device-side wait: 2^31 SM clock cycles, about a second
constexpr long long kDefaultWaitCycles = 1LL << 31;

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

// Tile shape: TX x (256 / TX) RPT cells per plane, 256 threads; in 2-D every
// thread can own RPT rows and issues the population loads of its cells before
// the staging barrier (PREFETCH), so the two load phases overlap.  Measured
// on GB300 for the single-domain step: 32 x 8 with one row per thread is
// fastest (two rows spill at the 64-register cap); the prefetch helps the
// FP16-stored path.  The batched step lets its autotuner pick among shapes.
// 3-D blocks march over ZC planes.
template <int DIM, int TXv = 32, int RPTv = 1> struct Tile {
  static constexpr int RPT = RPTv;
  static constexpr bool PREFETCH = DIM == 2;
  static constexpr int TX = TXv, TY = (256 / TXv) * RPT;
  static constexpr int ZC = DIM == 3 ? 16 : 1;
  static constexpr int HX = TX + 2, HY = TY + 2, HP = HX * HY;
  static constexpr int NPL = DIM == 3 ? 3 : 1;  // staged planes
};

// ------------------------------------------------------------ parameters
// FP64 chemistry data of the implicit integrator.
template <int K>
struct Chem64 {
  static constexpr int KK = K > 0 ? K : 1;
  double A[JMAX], b[JMAX], EaR[JMAX], dH[JMAX], dS[JMAX], dn[JMAX];
  int rev[JMAX];
  double order[JMAX][KK], rorder[JMAX][KK], stoich[JMAX][KK];
  double Ms[JMAX][KK];          // M_k s_kj
  double dS_R[JMAX], dH_R[JMAX];  // dS / R, dH / R
  double M[KK], invM[KK], cp[KK], hf[KK];
  double p_ref, ln_pref_R, rho_ref, dt;  // ln_pref_R = ln(p_ref / R)
};

// FP32 copy of the chemistry for the Newton fallback of the surrogate in FP32
// domains (rate constants as logarithms: ln k = ln A + b ln T - EaR / T).
template <int K>
struct Chem32 {
  static constexpr int KK = K > 0 ? K : 1;
  float lnA[JMAX], b[JMAX], EaR[JMAX], dn[JMAX], dS_R[JMAX], dH_R[JMAX];
  int on[JMAX], rev[JMAX];
  float order[JMAX][KK], rorder[JMAX][KK];
  float Ms[JMAX][KK];  // M_k s_kj
  float invM[KK], cp[KK], hf[KK];
  float ln_pref_R, dt;
};

// Everything in lattice units, converted once on the host (pflb_launch.cuh).
template <class Real, int K>
struct Params {
  static constexpr int KK = K > 0 ? K : 1;
  int nx, ny, nz, N;
  int bc[6];
  Real wall_u[6][3];
  Real wall_T[6];
  double eos_c;            // rho* = P0 Mw eos_c / T, eos_c = 1 / (R rho_ref)
  double inv_rho_ref;      // dP0 / rho_ref (J/kg) in the T equation
  Real eos_cr;             // eos_c in the compute type
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
  Real cpD[KK];            // cp_k Dlat_k (enthalpy-flux cross term)
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
  // reversible reactions in the compute type (explicit rates)
  int rev[JMAX];
  Real rorder[JMAX][KK];
  Real dS_R[JMAX], dH_R[JMAX], dn[JMAX], p_ref_R;  // dS/R, dH/R, sum_k s_kj, p_ref/R
  // FP64 copy of the chemistry for the implicit Newton integrator (FP64 in
  // every precision mode: the stiff chemistry keeps double precision)
  Chem64<K> c64;
  Chem32<K> c32;
  // mixture-averaged transport (Sec. 4.4): species Sutherland laws (lattice
  // units), modified Eucken factors, Wilke's constant factors
  int mix;
  Real mu_lat_k[KK], inv_suth_Tk[KK], suth_Sk[KK], suth_TSk[KK], eucken_k[KK];
  Real wA[KK][KK];         // (M_j / M_k)^(1/4)
  Real wB[KK][KK];         // 1 / (sqrt(8) sqrt(1 + M_k / M_j))
  // inlet mass-flow feedback (Sec. 4.4.1): on, species index, and
  // feed_c = 1 / (rho_in / P0 Y_in[k] A) so that u_in = fuel feed_c / P0
  int feed, feed_k;
  double feed_c;
  // characteristic outlet (Sec. 4.1): on, and K = sigma cs / nx
  int nscbc;
  double nscbc_K;
  // moving solid (Sec. 2, interface velocity): rigid translation velocity
  int moving;
  Real u_s[3];
};

// Scalar state on the device.  The per-step quantities the cells need (P0,
// dP0/P0, dP0/rho_ref) are precomputed by the block that finishes the
// reduction, in FP64 and in FP32.
struct DevScalars {
  double P0, P0_prev, mass, I, flux_in, flux_out, mass_now;
  double flux_in_sum, flux_out_sum;  // inlet / outlet mass flux summed over the steps
  long long step;
  int status;
  int pad;
  double dlnP0, dP0r;
  float P0_f, dlnP0_f, dP0r_f, pad_f;
  // inlet peak speed of the next step and the consumption it was set from
  // (inlet feedback; otherwise u_in stays the description's value)
  double u_in, fuel;
  float u_in_f, pad_f2;
  // boundary pressure of the next step at the characteristic outlet
  double pb;
  float pb_f, pad_f3;
};

// FP16 storage keeps, per cell, the FP32 moments (P, j) = (sum g*, sum c g*)
// of the post-collision populations and, per direction, the FP16 residual
// h_i = (g*_i - w_i (P + 3 c_i . j)) S / w_i (the first-order equilibrium of
// the cell's own moments removed, so that the narrowed quantity is second
// order in u).  A reader adds w_i (P + 3 c_i . j) of the source cell back.
template <class Store> struct IsHalf { static constexpr bool value = false; };
template <> struct IsHalf<__half> { static constexpr bool value = true; };
template <int DIM, class Store>
__host__ __device__ constexpr int n_mom() { return IsHalf<Store>::value ? DIM + 1 : 0; }

template <class Real, class Store>
struct State {
  const Store* __restrict__ g_in;
  Store* __restrict__ g_out;
  const Real* __restrict__ M_in;   // FP16 storage: moments [DIM+1][N] of g_in (else null)
  Real* __restrict__ M_out;        // FP16 storage: moments of g_out
  const Real* __restrict__ T_in;
  Real* __restrict__ T_out;
  const Real* __restrict__ Y_in;
  Real* __restrict__ Y_out;
  const Real* __restrict__ Ts_in;
  Real* __restrict__ Ts_out;
  const Real* __restrict__ phi;
  const Real* __restrict__ src;  // precomputed chemistry increments [K+1][N] (implicit/surrogate)
  DevScalars* scal;
  double* partials;        // this step's block partials: [blocks][4]
  unsigned* counter;
  Real* ob;                // characteristic outlet: P_h, u_x of columns nx-1 and nx-2 and rho
                           // of column nx-1 of this step, [5][ny nz] (else null)
};

// ----------------------------------------------------- storage codecs
template <class Store, class Real> struct Codec;
// load: from global memory (read-only path); get: from shared memory.
// raw: the stored value as a number; dec(raw, w/S, fo): the population from it
// and the first-order part fo of the source cell (FP16 storage: one FMA, the
// same on every path that decodes, so all paths round alike).
template <> struct Codec<double, double> {
  __device__ static double raw(const double* p) { return __ldg(p); }
  __device__ static double dec(double r, double, double) { return r; }
  __device__ static double load(const double* p, double) { return __ldg(p); }
  __device__ static double get(const double* p, double) { return *p; }
  __device__ static void store(double* p, double v, double) { *p = v; }
};
template <> struct Codec<float, float> {
  __device__ static float raw(const float* p) { return __ldg(p); }
  __device__ static float dec(float r, float, float) { return r; }
  __device__ static float load(const float* p, float) { return __ldg(p); }
  __device__ static float get(const float* p, float) { return *p; }
  __device__ static void store(float* p, float v, float) { *p = v; }
};
// FP16: residual r_i = g_i - w_i (P + 3 c_i . j), stored as h = r / w * scale
// (weights folded so every direction has the same range); load/get return
// r_i, the caller adds the first-order part of the source cell.
template <> struct Codec<__half, float> {
  __device__ static float raw(const __half* p) { return __half2float(__ldg(p)); }
  __device__ static float dec(float r, float w_over_scale, float fo) {
    return __fmaf_rn(r, w_over_scale, fo);
  }
  __device__ static float load(const __half* p, float w_over_scale) {
    return __half2float(__ldg(p)) * w_over_scale;
  }
  __device__ static float get(const __half* p, float w_over_scale) {
    return __half2float(*p) * w_over_scale;
  }
  __device__ static void store(__half* p, float v, float scale_over_w) {
    *p = __float2half_rn(v * scale_over_w);
  }
};

// ---------------------------------------------------------- arithmetic
// FP32 uses the fast hardware approximations (a few ulp); FP64 stays IEEE.
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }

// Packed FP32 pairs (the f32x2 arithmetic of sm_100 and later: one
// instruction for two lanes of independent FP32 work).
__device__ __forceinline__ uint64_t f2_bits(float2 v) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
  return r;
}
__device__ __forceinline__ float2 f2_of(uint64_t r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  uint64_t d;
  asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)),
      "l"(f2_bits(c)));
  return f2_of(d);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  uint64_t d;
  asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_of(d);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  uint64_t d;
  asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_of(d);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  uint64_t d;
  asm("add.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_of(d);
}
__device__ __forceinline__ float2 splat2(float a) { return make_float2(a, a); }

__device__ __forceinline__ float fexp(float x) { return __expf(x); }
__device__ __forceinline__ double fexp(double x) { return exp(x); }
__device__ __forceinline__ float fpow(float x, float y) { return __powf(x, y); }
__device__ __forceinline__ double fpow(double x, double y) { return pow(x, y); }

template <class Real> __device__ __forceinline__ Real scal_P0(const DevScalars* s);
template <> __device__ __forceinline__ double scal_P0<double>(const DevScalars* s) { return s->P0; }
template <> __device__ __forceinline__ float scal_P0<float>(const DevScalars* s) { return s->P0_f; }
template <class Real> __device__ __forceinline__ Real scal_u_in(const DevScalars* s);
template <> __device__ __forceinline__ double scal_u_in<double>(const DevScalars* s) { return s->u_in; }
template <> __device__ __forceinline__ float scal_u_in<float>(const DevScalars* s) { return s->u_in_f; }
template <class Real> __device__ __forceinline__ Real scal_pb(const DevScalars* s);
template <> __device__ __forceinline__ double scal_pb<double>(const DevScalars* s) { return s->pb; }
template <> __device__ __forceinline__ float scal_pb<float>(const DevScalars* s) { return s->pb_f; }
template <class Real> __device__ __forceinline__ Real scal_dlnP0(const DevScalars* s);
template <> __device__ __forceinline__ double scal_dlnP0<double>(const DevScalars* s) { return s->dlnP0; }
template <> __device__ __forceinline__ float scal_dlnP0<float>(const DevScalars* s) { return s->dlnP0_f; }
template <class Real> __device__ __forceinline__ Real scal_dP0r(const DevScalars* s);
template <> __device__ __forceinline__ double scal_dP0r<double>(const DevScalars* s) { return s->dP0r; }
template <> __device__ __forceinline__ float scal_dP0r<float>(const DevScalars* s) { return s->dP0r_f; }

// ------------------------------------------------------------ physics
// Viscosity: Sutherland (Sec. 4, eq. muT) or constant, lattice units.
template <class Real, int K>
__device__ __forceinline__ Real viscosity(const Params<Real, K>& P, Real T) {
  if (!P.sutherland) return P.mu_lat;
  Real t = T * P.inv_suth_T;
  return P.mu_lat * t * sqrt(t) * fdiv(P.suth_TS, T + P.suth_S);
}

// Viscosity and conductivity of the gas of composition Y at T (lattice
// units).  Single-gas mode: the viscosity law above and lambda = mu cp / Pr.
// Mixture mode (Sec. 4.4, eqs. muT_mix, phi_mix, conduct_mix): mole fractions
// X_k = Y_k Mw / M_k, species viscosities from their Sutherland laws,
// mu = sum_k mu_k X_k / sum_j Phi_kj X_j with
// Phi_kj = (1 + sqrt(mu_k / mu_j) (M_j / M_k)^(1/4))^2 / (sqrt(8) sqrt(1 + M_k / M_j)),
// lambda = (sum_k X_k lambda_k + 1 / sum_k X_k / lambda_k) / 2 with
// lambda_k = mu_k (1.32 cv_k + 1.77 R / M_k).
template <class Real, int K>
__device__ __forceinline__ void transport(const Params<Real, K>& P, Real T, const Real* Y,
                                          Real invMw, Real cp, Real& mu, Real& lam) {
  if constexpr (K > 0) {
    if (P.mix) {
      Real X[K], m[K], sm[K], ism[K];
      const Real Mw = fdiv(Real(1), invMw);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        X[k] = Y[k] * P.invM[k] * Mw;
        const Real t = T * P.inv_suth_Tk[k];
        m[k] = P.mu_lat_k[k] * t * sqrt(t) * fdiv(P.suth_TSk[k], T + P.suth_Sk[k]);
        sm[k] = sqrt(m[k]);
        ism[k] = fdiv(Real(1), sm[k]);
      }
      Real mm = 0, l1 = 0, l2 = 0;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        Real den = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
          const Real a = Real(1) + sm[k] * ism[j] * P.wA[k][j];
          den += a * a * P.wB[k][j] * X[j];
        }
        mm += m[k] * X[k] * fdiv(Real(1), den);
        const Real lk = m[k] * P.eucken_k[k];
        l1 += X[k] * lk;
        l2 += X[k] * fdiv(Real(1), lk);
      }
      mu = mm;
      lam = Real(0.5) * (l1 + fdiv(Real(1), l2));
      return;
    }
  }
  mu = viscosity(P, T);
  lam = mu * cp * P.inv_Pr;
}

template <class Real, int K>
__device__ __forceinline__ Real mixture_invMw(const Params<Real, K>& P, const Real* Y) {
  if constexpr (K == 0) {
    return Real(1) / P.M0;
  } else {
    Real s = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) s += Y[k] * P.invM[k];
    return s;
  }
}

template <class Real, int K>
__device__ __forceinline__ Real mixture_cp(const Params<Real, K>& P, const Real* Y) {
  if constexpr (K == 0) {
    return P.cp0;
  } else {
    Real s = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) s += Y[k] * P.cp[k];
    return s;
  }
}

// Explicit Arrhenius rates (Sec. 3.2.2 eq. 8, Sec. 3.3 eq. 9), per lattice
// step per rho_ref: om[k] = omega_k dt / rho_ref, omT likewise (J/kg).
template <class Real, int K>
__device__ __forceinline__ void rates(const Params<Real, K>& P, Real T, const Real* Y, Real rho,
                                      Real invT, Real* om, Real& omT) {
#pragma unroll
  for (int k = 0; k < K; ++k) om[k] = 0;
  Real C[Params<Real, K>::KK];
#pragma unroll
  for (int k = 0; k < K; ++k) C[k] = rho * P.rho_ref_M[k] * (Y[k] > Real(0) ? Y[k] : Real(0));
#pragma unroll 1
  for (int j = 0; j < P.J; ++j) {
    Real kf = P.A_lat[j] * fexp(-P.EaR[j] * invT);
    if (P.b[j] != Real(0)) kf *= fpow(T, P.b[j]);
    Real q = kf;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const Real o = P.order[j][k];
      if (o == Real(1)) q *= C[k];
      else if (o == Real(2)) q *= C[k] * C[k];
      else if (o != Real(0)) q *= fpow(C[k], o);
    }
    if (P.rev[j]) {
      // k_r = k_f / K_c, K_c = exp(dS/R - dH/(R T)) (p_ref/(R T))^(sum s)
      const Real Kc = fexp(P.dS_R[j] - P.dH_R[j] * invT) * fpow(P.p_ref_R * invT, P.dn[j]);
      Real qr = fdiv(kf, Kc);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const Real o = P.rorder[j][k];
        if (o == Real(1)) qr *= C[k];
        else if (o == Real(2)) qr *= C[k] * C[k];
        else if (o != Real(0)) qr *= fpow(C[k], o);
      }
      q -= qr;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) om[k] += P.stoichM[j][k] * q;
  }
  Real wt = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) wt -= P.hf[k] * om[k];
  omT = wt;
}

// Power C^o of a concentration for the reaction orders that occur (0, 1, 2,
// 1/2: multiplications and a square root), pow() otherwise; d = dC^o/dC for
// C > 0, in the precision LA of the Jacobian.
template <class LA>
__device__ __forceinline__ double conc_power(double C, double o, LA& d) {
  if (o == 1.0) { d = LA(1); return C; }
  if (o == 0.0) { d = LA(0); return 1.0; }
  if (o == 2.0) { d = LA(2) * LA(C); return C * C; }
  if (o == 0.5) {
    const double s = sqrt(C);
    d = s > 0.0 ? LA(0.5) / LA(s) : LA(0);
    return s;
  }
  d = C > 0.0 ? LA(o * pow(C, o - 1.0)) : LA(0);
  return pow(C, o);
}

// Rates w_k (kg/(m^3 s), FP64) and their Jacobian dw_k/dz_m, z = (Y_1..Y_K,
// T), in the precision LA: FP64 for FP64 domains; FP32 for FP32 domains,
// where the Jacobian only steers the Newton iteration and the FP64 residual
// decides where it converges.
template <int K, class LA>
__device__ __forceinline__ void rates_jacobian64(const Chem64<K>& c, const double* z, double rho,
                                                 double* w, LA (*dw)[K + 1]) {
  constexpr int KK = K > 0 ? K : 1;
  constexpr int n = K + 1;
  const double T = z[K], invT = 1.0 / T;
  double Cc[KK];
  LA dC[KK];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double d = z[k] > 0 ? rho * c.invM[k] : 0.0;
    dC[k] = LA(d);
    Cc[k] = z[k] > 0 ? z[k] * d : 0.0;
    w[k] = 0;
#pragma unroll
    for (int m = 0; m < n; ++m) dw[k][m] = LA(0);
  }
  double lnT = 0.0;
  bool have_lnT = false;
#pragma unroll
  for (int j = 0; j < JMAX; ++j) {
    if (c.A[j] == 0.0) continue;
    double kf = c.A[j] * exp(-c.EaR[j] * invT);
    if (c.b[j] != 0.0) kf *= pow(T, c.b[j]);
    const double dlkf = (c.EaR[j] * invT + c.b[j]) * invT;
    double kr = 0.0, dlkr = dlkf;
    if (c.rev[j]) {
      // K_c = exp(dS/R - dH/(R T)) (p_ref / (R T))^dn
      double lnKc = c.dS_R[j] - c.dH_R[j] * invT;
      if (c.dn[j] != 0.0) {
        if (!have_lnT) { lnT = log(T); have_lnT = true; }
        lnKc += c.dn[j] * (c.ln_pref_R - lnT);
      }
      kr = kf * exp(-lnKc);
      dlkr = dlkf - (c.dH_R[j] * invT + c.dn[j]) * invT;
    }
    LA dq[K + 1];
#pragma unroll
    for (int m = 0; m < n; ++m) dq[m] = LA(0);
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      if (dir == 1 && !c.rev[j]) break;
      const double kk = dir == 0 ? kf : -kr;
      double Pw[KK], pre[K + 1];
      LA Dp[KK], suf[K + 1];
#pragma unroll
      for (int k = 0; k < K; ++k)
        Pw[k] = conc_power(Cc[k], dir == 0 ? c.order[j][k] : c.rorder[j][k], Dp[k]);
      // prefix / suffix products: the product without factor m, no division
      pre[0] = 1.0;
      suf[K] = LA(1);
#pragma unroll
      for (int k = 0; k < K; ++k) pre[k + 1] = pre[k] * Pw[k];
#pragma unroll
      for (int k = K - 1; k >= 0; --k) suf[k] = LA(Pw[k]) * suf[k + 1];
      const double q = kk * pre[K];
#pragma unroll
      for (int k = 0; k < K; ++k) w[k] += c.Ms[j][k] * q;
      dq[K] += LA(q) * LA(dir == 0 ? dlkf : dlkr);
#pragma unroll
      for (int m = 0; m < K; ++m) dq[m] += LA(kk * pre[m]) * suf[m + 1] * Dp[m] * dC[m];
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int m = 0; m < n; ++m) dw[k][m] += LA(c.Ms[j][k]) * dq[m];
  }
}

// Solve A x = r in place (r <- x) by Gaussian elimination with partial
// pivoting; false if a pivot is zero.  The compiler keeps a 7 x 7 matrix in
// local memory here (the row swap after the pivot search defeats its scalar
// replacement); a fully unrolled form with the matrix in registers was tried
// and is slower, its register pressure spilling more than the matrix.
template <int n, class LA>
__device__ __forceinline__ bool solve_pivoted(LA (*A)[n], LA* r) {
  LA dinv[n];
#pragma unroll
  for (int col = 0; col < n; ++col) {
    int piv = col;
    LA best = fabs(A[col][col]);
#pragma unroll
    for (int rr = col + 1; rr < n; ++rr) {
      const LA v = fabs(A[rr][col]);
      if (v > best) { best = v; piv = rr; }
    }
    if (best == LA(0)) return false;
#pragma unroll
    for (int rr = col + 1; rr < n; ++rr) {
      if (rr == piv) {
#pragma unroll
        for (int k = col; k < n; ++k) { const LA t = A[col][k]; A[col][k] = A[rr][k]; A[rr][k] = t; }
        const LA t = r[col]; r[col] = r[rr]; r[rr] = t;
      }
    }
    const LA inv = LA(1) / A[col][col];
    dinv[col] = inv;
#pragma unroll
    for (int rr = col + 1; rr < n; ++rr) {
      const LA f = A[rr][col] * inv;
#pragma unroll
      for (int k = col + 1; k < n; ++k) A[rr][k] -= f * A[col][k];
      r[rr] -= f * r[col];
    }
  }
#pragma unroll
  for (int rr = n - 1; rr >= 0; --rr) {
    LA s = r[rr];
#pragma unroll
    for (int k = rr + 1; k < n; ++k) s -= A[rr][k] * r[k];
    r[rr] = s * dinv[rr];
  }
  return true;
}

// ----------------------------------------------- implicit chemistry (FP64)
// One lattice step of the chemistry alone at frozen density (operator
// splitting), backward Euler: z = (Y_1..Y_K, T), dY/dt = omega/rho,
// dT/dt = -sum hf omega / (rho cp(Y)).  Newton with the analytic Jacobian and
// Gaussian elimination with partial pivoting (tolerance 1e-13, <= 30
// iterations); if it fails the step is split into 2, 4, ..., 64 backward-Euler
// sub-steps.  Kept out of line so that it does not weigh on the register
// allocation of the rest of the step.  The arithmetic is laid out for a short
// dependency chain (FP64 latency sets the time of a warp): reciprocals taken
// once, square roots for half orders, no dynamic array indices.
// The state, the rates and the residual are FP64 in every mode; the Jacobian,
// the Newton matrix and its elimination take the precision LA (FP64 for FP64
// domains, FP32 for FP32 domains).  A direction from an FP32 elimination is
// off by about cond(A) x 6e-8 of itself, so the iteration still contracts and
// stops where the FP64 residual puts the root (the update test is relative
// to the update, not to the FP32 rounding), and the elimination runs on the
// FP32 pipe instead of GB300's narrow FP64 one.
template <int K, class LA>
__device__ __forceinline__ void chem_be_newton(const Chem64<K>* C0,
                                            double T0, const double* Y0, double rho,
                                            double* dY, double* dT) {
  constexpr int n = K + 1;
  const auto& c = *C0;
  const double inv_rho = 1.0 / rho;
  double zs[K + 1], z[K + 1], y0[K + 1];
#pragma unroll
  for (int k = 0; k < K; ++k) y0[k] = Y0[k];
  y0[K] = T0;
  int ok = -1;
  // the sub-step and Newton loops stay rolled: unrolled, they multiply the
  // fully unrolled Jacobian and elimination by up to 7 x 30 copies
#pragma unroll 1
  for (int nsub = 1; nsub <= 64 && ok != 0; nsub *= 2) {
#pragma unroll
    for (int m = 0; m < n; ++m) zs[m] = y0[m];
    ok = 0;
    const double h = c.dt / nsub, hr = h * inv_rho;
#pragma unroll 1
    for (int sub = 0; sub < nsub && ok == 0; ++sub) {
#pragma unroll
      for (int m = 0; m < n; ++m) z[m] = zs[m];
      const double inv_Ts = 1.0 / zs[K];  // temperature scale of the update test
      ok = -1;
#pragma unroll 1
      for (int it = 0; it < 30; ++it) {
        double w[K + 1];
        LA A[K + 1][K + 1];  // rows 0..K-1: dw_k/dz_m, then the Newton matrix
        rates_jacobian64<K, LA>(c, z, rho, w, A);
        double cp = 0, hw = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          cp += z[k] * c.cp[k];
          hw += c.hf[k] * w[k];
        }
        const double inv_rcp = inv_rho / cp;
        // Newton system (I - h dF/dz) dz = -(z - zs - h F): residual in FP64,
        // matrix in LA, built in place (the T row first, from the rates'
        // Jacobian, then the species rows)
        const LA hrL = LA(hr), hL = LA(h), inv_rcpL = LA(inv_rcp);
        const LA hwcL = LA(hw * inv_rcp / cp);
        LA r[K + 1];
#pragma unroll
        for (int m = 0; m < n; ++m) {
          LA dhw = LA(0);
#pragma unroll
          for (int k = 0; k < K; ++k) dhw += LA(c.hf[k]) * A[k][m];
          LA dFT = -dhw * inv_rcpL;
          if (m < K) dFT += hwcL * LA(c.cp[m]);
          A[K][m] = LA(m == K ? 1 : 0) - hL * dFT;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
          r[k] = LA(-(z[k] - zs[k] - hr * w[k]));
#pragma unroll
          for (int m = 0; m < n; ++m) A[k][m] = LA(k == m ? 1 : 0) - hrL * A[k][m];
        }
        r[K] = LA(-(z[K] - zs[K] + h * hw * inv_rcp));
        if (!solve_pivoted<K + 1, LA>(A, r)) break;
        double big = 0;
        bool bad = false;
#pragma unroll
        for (int m = 0; m < n; ++m) {
          z[m] += double(r[m]);
          const double e = fabs(double(r[m])) * (m < K ? 1.0 : inv_Ts);
          if (!(e == e)) bad = true;
          if (e > big) big = e;
        }
        if (bad || !(z[K] > 0)) break;
        if (big < 1e-13) { ok = 0; break; }
      }
#pragma unroll
      for (int m = 0; m < n; ++m) zs[m] = z[m];
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) dY[k] = zs[k] - y0[k];
  *dT = zs[K] - T0;
}

// ------------------------------------ Newton fallback of FP32 domains (FP32)
// Rates w_k (kg/(m^3 s)) and their Jacobian dw_k/dz_m in FP32, z = (Y, T);
// k_f and k_r are taken as exponentials of their logarithms, so that neither
// over- nor underflows on the way (k_r = exp(ln k_f - ln K_c)).
template <int K>
__device__ __forceinline__ void rates_jacobian32(const Chem32<K>& c, const float* z, float rho,
                                                 float* w, float (*dw)[K + 1]) {
  constexpr int KK = K > 0 ? K : 1;
  constexpr int n = K + 1;
  const float T = z[K], invT = 1.f / T, lnT = logf(T);
  float Cc[KK], dC[KK];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    dC[k] = z[k] > 0.f ? rho * c.invM[k] : 0.f;
    Cc[k] = z[k] > 0.f ? z[k] * dC[k] : 0.f;
    w[k] = 0.f;
#pragma unroll
    for (int m = 0; m < n; ++m) dw[k][m] = 0.f;
  }
#pragma unroll
  for (int j = 0; j < JMAX; ++j) {
    if (!c.on[j]) continue;
    const float lkf = c.lnA[j] + c.b[j] * lnT - c.EaR[j] * invT;
    const float kf = expf(lkf);
    const float dlkf = (c.EaR[j] * invT + c.b[j]) * invT;
    float kr = 0.f, dlkr = dlkf;
    if (c.rev[j]) {
      const float lnKc = c.dS_R[j] - c.dH_R[j] * invT + c.dn[j] * (c.ln_pref_R - lnT);
      kr = expf(lkf - lnKc);
      dlkr = dlkf - (c.dH_R[j] * invT + c.dn[j]) * invT;
    }
    float dq[K + 1];
#pragma unroll
    for (int m = 0; m < n; ++m) dq[m] = 0.f;
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      if (dir == 1 && !c.rev[j]) break;
      const float kk = dir == 0 ? kf : -kr;
      float Pw[KK], Dp[KK], pre[K + 1], suf[K + 1];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float o = dir == 0 ? c.order[j][k] : c.rorder[j][k];
        const float C = Cc[k];
        if (o == 1.f) { Pw[k] = C; Dp[k] = 1.f; }
        else if (o == 0.f) { Pw[k] = 1.f; Dp[k] = 0.f; }
        else if (o == 2.f) { Pw[k] = C * C; Dp[k] = 2.f * C; }
        else if (o == 0.5f) {
          const float sq = sqrtf(C);
          Pw[k] = sq;
          Dp[k] = sq > 0.f ? 0.5f / sq : 0.f;
        } else {
          Pw[k] = powf(C, o);
          Dp[k] = C > 0.f ? o * powf(C, o - 1.f) : 0.f;
        }
      }
      pre[0] = 1.f;
      suf[K] = 1.f;
#pragma unroll
      for (int k = 0; k < K; ++k) pre[k + 1] = pre[k] * Pw[k];
#pragma unroll
      for (int k = K - 1; k >= 0; --k) suf[k] = Pw[k] * suf[k + 1];
      const float q = kk * pre[K];
#pragma unroll
      for (int k = 0; k < K; ++k) w[k] += c.Ms[j][k] * q;
      dq[K] += q * (dir == 0 ? dlkf : dlkr);
#pragma unroll
      for (int m = 0; m < K; ++m) dq[m] += kk * (pre[m] * suf[m + 1]) * Dp[m] * dC[m];
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int m = 0; m < n; ++m) dw[k][m] += c.Ms[j][k] * dq[m];
  }
}

// The backward-Euler step of chem_be_newton in FP32 for the cells that the
// surrogate rejects in FP32 domains.  FP32 cannot hold the root to the FP64
// integrator's 1e-13, so the unknown is the sub-step's increment d = z - zs
// (small numbers keep their relative precision), the residual is
// d - h F(zs + d), and the iteration stops once every update is below
// 1e-5 |d_m| + 1e-6 |zs_m| (a few units in the last place of the FP32 field
// that receives the increment).  On GB300 the FP64 pipe issues one warp
// instruction every 16 cycles per SM, so the FP64 integrator's chain on a
// short list of cells takes tens of microseconds; this one runs on the FP32
// pipe and the special-function unit.
template <int K>
__device__ __forceinline__ void chem_be_newton32(const Chem32<K>& c, float T0, const float* Y0,
                                                 float rho, float* dY, float* dT) {
  constexpr int n = K + 1;
  const float inv_rho = 1.f / rho;
  float y0[K + 1], acc[K + 1];
#pragma unroll
  for (int k = 0; k < K; ++k) y0[k] = Y0[k];
  y0[K] = T0;
#pragma unroll
  for (int m = 0; m < n; ++m) acc[m] = 0.f;
  int ok = -1;
#pragma unroll 1
  for (int nsub = 1; nsub <= 64 && ok != 0; nsub *= 2) {
    float zs[K + 1];
#pragma unroll
    for (int m = 0; m < n; ++m) {
      zs[m] = y0[m];
      acc[m] = 0.f;
    }
    ok = 0;
    const float h = c.dt / float(nsub), hr = h * inv_rho;
#pragma unroll 1
    for (int sub = 0; sub < nsub && ok == 0; ++sub) {
      float d[K + 1];
#pragma unroll
      for (int m = 0; m < n; ++m) d[m] = 0.f;
      ok = -1;
#pragma unroll 1
      for (int it = 0; it < 30; ++it) {
        float z[K + 1], w[K + 1];
#pragma unroll
        for (int m = 0; m < n; ++m) z[m] = zs[m] + d[m];
        if (!(z[K] > 0.f)) break;
        float A[K + 1][K + 1];
        rates_jacobian32<K>(c, z, rho, w, A);
        float cp = 0.f, hw = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          cp += z[k] * c.cp[k];
          hw += c.hf[k] * w[k];
        }
        const float inv_rcp = inv_rho / cp;
        const float hwc = hw * inv_rcp / cp;
        float r[K + 1];
#pragma unroll
        for (int m = 0; m < n; ++m) {
          float dhw = 0.f;
#pragma unroll
          for (int k = 0; k < K; ++k) dhw += c.hf[k] * A[k][m];
          float dFT = -dhw * inv_rcp;
          if (m < K) dFT += hwc * c.cp[m];
          A[K][m] = (m == K ? 1.f : 0.f) - h * dFT;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
          r[k] = -(d[k] - hr * w[k]);
#pragma unroll
          for (int m = 0; m < n; ++m) A[k][m] = (k == m ? 1.f : 0.f) - hr * A[k][m];
        }
        r[K] = -(d[K] + h * hw * inv_rcp);
        if (!solve_pivoted<K + 1, float>(A, r)) break;
        bool bad = false, done = true;
#pragma unroll
        for (int m = 0; m < n; ++m) {
          d[m] += r[m];
          if (!(r[m] == r[m])) bad = true;
          if (fabsf(r[m]) > 1e-5f * fabsf(d[m]) + 1e-6f * fabsf(zs[m])) done = false;
        }
        if (bad) break;
        if (done) { ok = 0; break; }
      }
#pragma unroll
      for (int m = 0; m < n; ++m) {
        zs[m] += d[m];
        acc[m] += d[m];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) dY[k] = acc[k];
  *dT = acc[K];
}

// Moments read straight from global memory (the moments kernel, no staging).
template <class Real>
struct GlobalMom {
  const Real* M;
  int N;
  __device__ __forceinline__ Real mom(int a, int src, int, int, int) const {
    return M[(size_t)a * N + src];
  }
};

// First-order part w_i (P + 3 c_i . j) of direction i at the source cell
// (global index src, offset (dx, dy, dz) from the pulling cell).
template <int DIM, class Real, class MA>
__device__ __forceinline__ Real first_order(const MA& A, int i, int src, int dx, int dy, int dz) {
  using L = Lattice<DIM>;
  Real cj = 0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (L::c(i, a) > 0) cj += A.mom(1 + a, src, dx, dy, dz);
    if (L::c(i, a) < 0) cj -= A.mom(1 + a, src, dx, dy, dz);
  }
  return Real(L::w(i)) * (A.mom(0, src, dx, dy, dz) + Real(3) * cj);
}

template <class Real, int K>
__device__ __forceinline__ Real inlet_u(const Params<Real, K>& P, Real u, const int xyz[3],
                                        int dim) {
  if (P.inlet_parabolic != 1) return u;
  for (int a = 1; a < dim; ++a) {
    if (P.bc[2 * a] != BC_WALL) continue;
    Real n = Real(a == 1 ? P.ny : P.nz);
    Real s = Real(xyz[a]) + Real(0.5);
    u *= Real(4) * s * (n - s) / (n * n);
  }
  return u;
}

// The cell's own post-collision population of direction ib (bounce-back).
template <int DIM, class Real, class Store, int K, class MA>
__device__ __forceinline__ Real own_pop(const Params<Real, K>& P, const State<Real, Store>& S,
                                        int c, int ib, const MA& mom) {
  const Real r = Codec<Store, Real>::raw(S.g_in + (size_t)ib * P.N + c);
  if constexpr (IsHalf<Store>::value)
    return Codec<Store, Real>::dec(r, Real(Lattice<DIM>::w(ib)) * P.g_inv_scale,
                                   first_order<DIM, Real>(mom, ib, c, 0, 0, 0));
  else return r;
}

// Half-way bounce-back with the wall velocity for the directions entering
// through face F, when the cell lies on it (on) and it is a wall.
template <int DIM, int F, class Real, class Store, int K, class MA>
__device__ __forceinline__ void wall_pops(const Params<Real, K>& P, const State<Real, Store>& S,
                                          int c, bool on, Real rho_c, Real* gin, const MA& mom) {
  using L = Lattice<DIM>;
  constexpr int a = F >> 1, s = (F & 1) ? -1 : 1;
  if (!(on && P.bc[F] == BC_WALL)) return;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    if (L::c(i, a) != s) continue;
    Real cu = 0;
#pragma unroll
    for (int b = 0; b < DIM; ++b) cu += Real(L::c(i, b)) * P.wall_u[F][b];
    gin[i] = own_pop<DIM, Real, Store>(P, S, c, L::opp(i), mom) +
             Real(2) * Real(L::w(i)) * rho_c * cu;
  }
}

// Pull streaming of every population into the cell.  A cell off every face
// reads its upstream neighbours at fixed offsets.  On a face, along each axis
// the upstream neighbour coordinate wraps across a periodic face and is
// clamped to the cell itself across any other face; every direction is read
// from there.  Directions that cross a non-periodic face are then replaced by the
// boundary rules, in the order outlet, inlet, walls (the wall of the lowest
// axis last, so it wins on edges and corners): half-way bounce-back on walls
// (moving walls add 2 w rho c.u_w), the inlet as a moving wall with the inlet
// velocity and inlet density, the outlet as anti-bounce-back at P_h = 0 with
// wall velocity uw.
template <int DIM, class Real, class Store, int K, class MA>
__device__ __forceinline__ void pull(const Params<Real, K>& P, const State<Real, Store>& S, int c,
                                     const int xyz[3], Real rho_c, Real rho_in, const Real* uw,
                                     Real* gin, const MA& mom) {
  using L = Lattice<DIM>;
  constexpr bool FO = IsHalf<Store>::value;  // residual storage: add the first-order part
  // cells off every domain face: fixed offsets from the cell (the common case)
  const bool inner = xyz[0] > 0 && xyz[0] < P.nx - 1 && xyz[1] > 0 && xyz[1] < P.ny - 1 &&
                     (DIM == 2 || (xyz[2] > 0 && xyz[2] < P.nz - 1));
  if (inner) {
    const int sy = P.nx, sz = P.nx * P.ny;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const int cx = L::c(i, 0), cy = L::c(i, 1), cz = DIM == 3 ? L::c(i, 2) : 0;
      const int src = c - cx - cy * sy - cz * sz;
      const Real r = Codec<Store, Real>::raw(S.g_in + (size_t)i * P.N + src);
      if constexpr (FO)
        gin[i] = Codec<Store, Real>::dec(r, Real(L::w(i)) * P.g_inv_scale,
                                         first_order<DIM, Real>(mom, i, src, -cx, -cy, -cz));
      else gin[i] = r;
    }
    return;
  }
  // upstream neighbour coordinates along each axis: m (coordinate - 1) and
  // p (coordinate + 1), wrapped across periodic faces, clamped otherwise
  const int x = xyz[0], y = xyz[1], z = DIM == 3 ? xyz[2] : 0;
  const bool per0 = P.bc[0] == BC_PERIODIC, per1 = P.bc[1] == BC_PERIODIC;
  const bool per2 = P.bc[2] == BC_PERIODIC, per3 = P.bc[3] == BC_PERIODIC;
  const bool per4 = P.bc[4] == BC_PERIODIC, per5 = P.bc[5] == BC_PERIODIC;
  const int xm = x > 0 ? x - 1 : (per0 ? P.nx - 1 : x);
  const int xp = x < P.nx - 1 ? x + 1 : (per1 ? 0 : x);
  const int ym = y > 0 ? y - 1 : (per2 ? P.ny - 1 : y);
  const int yp = y < P.ny - 1 ? y + 1 : (per3 ? 0 : y);
  const int zm = DIM == 3 ? (z > 0 ? z - 1 : (per4 ? P.nz - 1 : z)) : 0;
  const int zp = DIM == 3 ? (z < P.nz - 1 ? z + 1 : (per5 ? 0 : z)) : 0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const int cx = L::c(i, 0), cy = L::c(i, 1), cz = DIM == 3 ? L::c(i, 2) : 0;
    const int sx = cx > 0 ? xm : (cx < 0 ? xp : x);
    const int sy = cy > 0 ? ym : (cy < 0 ? yp : y);
    const int sz = cz > 0 ? zm : (cz < 0 ? zp : z);
    const int src = sx + P.nx * (sy + P.ny * sz);
    const Real r = Codec<Store, Real>::raw(S.g_in + (size_t)i * P.N + src);
    // a periodic source: the staged halo holds its image at the same offset
    if constexpr (FO)
      gin[i] = Codec<Store, Real>::dec(r, Real(L::w(i)) * P.g_inv_scale,
                                       first_order<DIM, Real>(mom, i, src, -cx, -cy, -cz));
    else gin[i] = r;
  }
  // non-periodic faces the cell lies on
  const bool f0 = x == 0 && !per0, f1 = x == P.nx - 1 && !per1;
  const bool f2 = y == 0 && !per2, f3 = y == P.ny - 1 && !per3;
  const bool f4 = DIM == 3 && z == 0 && !per4, f5 = DIM == 3 && z == P.nz - 1 && !per5;
  if (!(f0 || f1 || f2 || f3 || f4 || f5)) return;
  if (f1 && P.bc[1] == BC_OUTLET) {
    Real uu = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) uu += uw[a] * uw[a];
    const Real pb2 = P.nscbc ? Real(2) * scal_pb<Real>(S.scal) : Real(0);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      if (L::c(i, 0) != -1) continue;
      Real cu = 0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) cu += Real(L::c(i, a)) * uw[a];
      gin[i] = -own_pop<DIM, Real, Store>(P, S, c, L::opp(i), mom) +
               Real(L::w(i)) * (pb2 + rho_c * (Real(3) * cu * cu - uu));
    }
  }
  if (f0 && P.bc[0] == BC_INLET) {
    Real ui = inlet_u(P, P.feed ? scal_u_in<Real>(S.scal) : P.u_in, xyz, DIM);
    if (P.inlet_parabolic == 2) ui *= Real(1) - S.phi[c];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      if (L::c(i, 0) != 1) continue;
      gin[i] = own_pop<DIM, Real, Store>(P, S, c, L::opp(i), mom) +
               Real(2) * Real(L::w(i)) * rho_in * ui;
    }
  }
  // walls, the highest axis first so that the lowest axis wins on edges
  if (DIM == 3) {
    wall_pops<DIM, 5>(P, S, c, f5, rho_c, gin, mom);
    wall_pops<DIM, 4>(P, S, c, f4, rho_c, gin, mom);
  }
  wall_pops<DIM, 3>(P, S, c, f3, rho_c, gin, mom);
  wall_pops<DIM, 2>(P, S, c, f2, rho_c, gin, mom);
  wall_pops<DIM, 1>(P, S, c, f1, rho_c, gin, mom);
  wall_pops<DIM, 0>(P, S, c, f0, rho_c, gin, mom);
}

// ----------------------------------------------------------- reductions
// Error-free sum of two floats (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Block sum of one per-thread value into FP64 (result in thread 0).  FP32
// values are summed within the warp with compensation (the pair s + e is
// exact up to the final rounding), warps are combined in FP64.
// Warp part of the sums below (result in lane 0).
template <class Real>
__device__ __forceinline__ double warp_sum(Real v) {
  if constexpr (sizeof(Real) == 4) {
    float s = v, e = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float so = __shfl_down_sync(0xffffffffu, s, o);
      const float eo = __shfl_down_sync(0xffffffffu, e, o);
      float t, err;
      two_sum(s, so, t, err);
      s = t;
      e = e + eo + err;
    }
    return double(s) + double(e);
  } else {
    double w = v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
    return w;
  }
}

// The three sums of a tile (I, and the two fluxes when `bc` holds) with one
// barrier, grouped exactly as block_sum; results valid in thread 0.  `sh`
// holds 96 doubles and is free again after the block's next barrier.
template <class Real>
__device__ __forceinline__ void block_sum3(Real a, Real b, Real c, bool bc, double* sh,
                                           double& ra, double& rb, double& rc) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double wa = warp_sum(a);
  const double wb = bc ? warp_sum(b) : 0.0, wc = bc ? warp_sum(c) : 0.0;
  if (lane == 0) {
    sh[wid] = wa;
    sh[32 + wid] = wb;
    sh[64 + wid] = wc;
  }
  __syncthreads();
  ra = rb = rc = 0.0;
  if (wid == 0) {
    const bool in = lane < (int)(blockDim.x >> 5);
    double x = in ? sh[lane] : 0.0, y = in ? sh[32 + lane] : 0.0, z = in ? sh[64 + lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_down_sync(0xffffffffu, x, o);
      y += __shfl_down_sync(0xffffffffu, y, o);
      z += __shfl_down_sync(0xffffffffu, z, o);
    }
    ra = x;
    rb = bc ? y : 0.0;
    rc = bc ? z : 0.0;
  }
}

template <class Real>
__device__ __forceinline__ double block_sum(Real v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double w;
  if constexpr (sizeof(Real) == 4) {
    float s = v, e = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float so = __shfl_down_sync(0xffffffffu, s, o);
      const float eo = __shfl_down_sync(0xffffffffu, e, o);
      float t, err;
      two_sum(s, so, t, err);
      s = t;
      e = e + eo + err;
    }
    w = double(s) + double(e);
  } else {
    w = v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
  }
  if (lane == 0) sh[wid] = w;
  __syncthreads();
  double r = 0;
  if (wid == 0) {
    r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;
}

// Combine the per-block partials (I, inlet flux, outlet flux) of one step in
// a fixed order (lane-strided sums, then a fixed shuffle tree) and update the
// scalar state: the P0 closure when the domain is closed, the diagnostics and
// the per-step constants the cells of the next step read.  Run by one warp.
__device__ __forceinline__ void combine_partials(const double* partials, unsigned nb,
                                                 DevScalars* scal, int p0_closed, bool is_init,
                                                 double init_P0, double eos_c,
                                                 double inv_rho_ref) {
  const int lane = threadIdx.x & 31;
  double v0 = 0, v1 = 0, v2 = 0;
  unsigned b = lane;
  for (; b + 96 < nb; b += 128) {
    const double a0 = __ldcg(partials + 4 * b), a1 = __ldcg(partials + 4 * (b + 32));
    const double a2 = __ldcg(partials + 4 * (b + 64)), a3 = __ldcg(partials + 4 * (b + 96));
    const double f0 = __ldcg(partials + 4 * b + 1), f1 = __ldcg(partials + 4 * (b + 32) + 1);
    const double f2 = __ldcg(partials + 4 * (b + 64) + 1), f3 = __ldcg(partials + 4 * (b + 96) + 1);
    const double o0 = __ldcg(partials + 4 * b + 2), o1 = __ldcg(partials + 4 * (b + 32) + 2);
    const double o2 = __ldcg(partials + 4 * (b + 64) + 2), o3 = __ldcg(partials + 4 * (b + 96) + 2);
    v0 += a0; v0 += a1; v0 += a2; v0 += a3;
    v1 += f0; v1 += f1; v1 += f2; v1 += f3;
    v2 += o0; v2 += o1; v2 += o2; v2 += o3;
  }
  for (; b < nb; b += 32) {
    v0 += __ldcg(partials + 4 * b + 0);
    v1 += __ldcg(partials + 4 * b + 1);
    v2 += __ldcg(partials + 4 * b + 2);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_down_sync(0xffffffffu, v0, o);
    v1 += __shfl_down_sync(0xffffffffu, v1, o);
    v2 += __shfl_down_sync(0xffffffffu, v2, o);
  }
  if (lane == 0) {
    const double I = v0;
    double P0, P0p;
    if (is_init) {
      P0 = P0p = init_P0;
      scal->mass = init_P0 * I * eos_c;
      scal->flux_in = scal->flux_out = 0;
      scal->flux_in_sum = scal->flux_out_sum = 0;
      scal->step = 0;
      scal->status = 0;
    } else {
      P0p = scal->P0;
      P0 = P0p;
      if (p0_closed) P0 = scal->mass / (I * eos_c);
      scal->flux_in = v1;
      scal->flux_out = v2;
      scal->flux_in_sum += v1;
      scal->flux_out_sum += v2;
      scal->step += 1;
      // latch only the first failure (a timeout is not overwritten)
      if (scal->status == 0 && (!(I == I) || !(P0 == P0) || I <= 0.0)) scal->status = -5;
    }
    scal->P0_prev = P0p;
    scal->P0 = P0;
    scal->I = I;
    scal->mass_now = P0 * I * eos_c;
    scal->dlnP0 = (P0 - P0p) / P0;
    scal->dP0r = (P0 - P0p) * inv_rho_ref;
    scal->P0_f = float(P0);
    scal->dlnP0_f = float(scal->dlnP0);
    scal->dP0r_f = float(scal->dP0r);
  }
}

// Publish the block sums (valid in thread 0) of this step.  Closed domains
// need P0 of the next step before it starts, so the warp that draws the last
// arrival ticket combines at once (lane 0 fences its own writes before taking
// the ticket; the other warps retire).  With a fixed P0 the combine is
// deferred: block 0 of the next launch, or the on-demand finalize kernel,
// does it, and the step ends without a serial tail.
// Publish into slot `bid` of `nb`; `now` combines at the last arrival.
__device__ __forceinline__ void publish_partials_at(double sI, double sIn, double sOut,
                                                    double* partials, unsigned* counter,
                                                    DevScalars* scal, int p0_closed, bool is_init,
                                                    double init_P0, double eos_c,
                                                    double inv_rho_ref, unsigned bid,
                                                    unsigned nb, bool now) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  unsigned last = 0;
  if (lane == 0) {
    partials[4 * bid + 0] = sI;
    partials[4 * bid + 1] = sIn;
    partials[4 * bid + 2] = sOut;
    if (now) {
      __threadfence();
      last = (atomicAdd(counter, 1u) == nb - 1) ? 1u : 0u;
    }
  }
  if (!now) return;
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return;
  __threadfence();
  combine_partials(partials, nb, scal, p0_closed, is_init, init_P0, eos_c, inv_rho_ref);
  if (lane == 0) *counter = 0u;
}

__device__ __forceinline__ void publish_partials(double sI, double sIn, double sOut,
                                                 double* partials, unsigned* counter,
                                                 DevScalars* scal, int p0_closed, bool is_init,
                                                 double init_P0, double eos_c,
                                                 double inv_rho_ref) {
  publish_partials_at(sI, sIn, sOut, partials, counter, scal, p0_closed, is_init, init_P0, eos_c,
                      inv_rho_ref,
                      blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z),
                      gridDim.x * gridDim.y * gridDim.z, p0_closed || is_init);
}

// On-demand combine of the deferred partials of the last step (one warp).
static __global__ void finalize_kernel(const double* partials, unsigned nb, DevScalars* scal,
                                double eos_c, double inv_rho_ref) {
  combine_partials(partials, nb, scal, 0, false, 0.0, eos_c, inv_rho_ref);
}

// ------------------------------------------------ staged tile (smem)
// Fields per staged cell: T, phi_s, rho, kappa_T = phi_f lambda, mu, f_D
// (diffusivity factor), Ts, phi_f rho f_D, then Y_k.
enum { F_T = 0, F_PHI, F_RHO, F_KT, F_MU, F_FD, F_TS, F_RF, F_Y0 };

template <class Real, int K, int HP, int NM = 0>
struct Plane {
  Real f[F_Y0 + K + NM][HP];  // NM moment fields (P, j) after the species
};

// Stage plane z (may be -1 or nz: ghost plane) of the block's tile with its
// xy halo.  Out-of-domain halo cells follow the ghost rules: periodic faces
// wrap; otherwise the adjacent cell's values, with the inlet state (T_in,
// Y_in) on the inlet face and the wall temperature on a wall that has one.
template <int DIM, class Real, class Store, int K, int HP, class T_ = Tile<DIM>,
          int NM = n_mom<DIM, Store>()>
__device__ __forceinline__ void stage_plane(const Params<Real, K>& P, const State<Real, Store>& S,
                                            Plane<Real, K, HP, NM>& pl, int x0, int y0, int z,
                                            Real P0) {
  static_assert(T_::HP == HP, "plane and tile shape disagree");
  // tiles whose halo lies inside the lattice need no ghost rules
  const bool inner = x0 >= 1 && y0 >= 1 && x0 + T_::TX < P.nx && y0 + T_::TY < P.ny &&
                     (DIM == 2 || (z >= 0 && z < P.nz));
  for (int h = threadIdx.x; h < HP; h += blockDim.x) {
    const int hx = h % T_::HX, hy = h / T_::HX;
    int q[3] = {x0 - 1 + hx, y0 - 1 + hy, z};
    int ghost_face = -1;
    int nout = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      if (inner) break;
      const int n = a == 0 ? P.nx : (a == 1 ? P.ny : P.nz);
      if (q[a] < 0 || q[a] >= n) {
        const int face = 2 * a + (q[a] >= n ? 1 : 0);
        if (P.bc[face] == BC_PERIODIC) {
          q[a] = q[a] < 0 ? q[a] + n : q[a] - n;
          if (q[a] < 0 || q[a] >= n) q[a] = q[a] < 0 ? 0 : n - 1;  // tiles wider than n
        } else {
          q[a] = q[a] < 0 ? 0 : n - 1;
          ghost_face = face;
          ++nout;
        }
      }
    }
    const int c = q[0] + P.nx * (q[1] + P.ny * q[2]);
    Real T = __ldg(S.T_in + c);
    const Real phis = __ldg(S.phi + c);
    const Real Ts = P.Ts_field ? __ldg(S.Ts_in + c) : P.Ts_uniform;
    Real Y[Params<Real, K>::KK];
#pragma unroll
    for (int k = 0; k < K; ++k) Y[k] = __ldg(S.Y_in + (size_t)k * P.N + c);
    if (nout == 1) {
      const int bc = P.bc[ghost_face];
      if (bc == BC_INLET) {
        T = P.T_in;
#pragma unroll
        for (int k = 0; k < K; ++k) Y[k] = P.Y_in[k];
      } else if (bc == BC_WALL && P.wall_T[ghost_face] > Real(0)) {
        T = P.wall_T[ghost_face];
      }
    }
    const Real phif = Real(1) - phis;
    const Real invMw = mixture_invMw(P, Y);
    const Real rho = fdiv(P0 * P.eos_cr, T * invMw);
    const Real cp = mixture_cp(P, Y);
    Real mu, lam;
    transport(P, T, Y, invMw, cp, mu, lam);
    Real fD = Real(1);
    if constexpr (K > 0) {
      if (P.D_Tdep) fD = fpow(T * P.inv_DTref, P.D_exp);
    }
    pl.f[F_T][h] = T;
    pl.f[F_PHI][h] = phis;
    pl.f[F_RHO][h] = rho;
    pl.f[F_KT][h] = phif * lam;
    pl.f[F_MU][h] = mu;
    pl.f[F_FD][h] = fD;
    pl.f[F_TS][h] = Ts;
    pl.f[F_RF][h] = phif * rho * fD;
#pragma unroll
    for (int k = 0; k < K; ++k) pl.f[F_Y0 + k][h] = Y[k];
    if constexpr (NM > 0) {
#pragma unroll
      for (int a = 0; a < NM; ++a) pl.f[F_Y0 + K + a][h] = __ldg(S.M_in + (size_t)a * P.N + c);
    }
  }
}

// Staged-plane accessor: own and neighbour values of the staged fields and
// properties (the populations come from global memory).
template <int DIM, class Real, bool PRE = false, class TL = Tile<DIM>, int MF = 0,
          bool STASH = false>
struct PlaneAcc {
  static constexpr int HP = TL::HP;
  static constexpr bool has_pops = PRE;  // populations prefetched into registers
  static constexpr bool kStash = STASH;  // pulled populations wait in shared memory
  const Real* __restrict__ cen;
  const Real* __restrict__ zm;
  const Real* __restrict__ zp;
  int h;
  const Real* pre;
  bool pv;  // pre holds this cell's populations
  Real* st; // stash, [Q][BLOCK] (STASH)
  __device__ __forceinline__ Real c(int f) const { return cen[f * HP + h]; }
  __device__ __forceinline__ Real n(int f, int a, int s) const {
    if (a == 0) return cen[f * HP + h + s];
    if (a == 1) return cen[f * HP + h + s * TL::HX];
    return (s < 0 ? zm : zp)[f * HP + h];
  }
  template <class Store>
  __device__ __forceinline__ Real pop(int i, Real) const { return PRE ? pre[i] : Real(0); }
  // moment a of the staged cell at offset (dx, dy, dz) (FP16 storage; MF is
  // the first moment field, src the cell's global index, unused here)
  __device__ __forceinline__ Real mom(int a, int, int dx, int dy, int dz) const {
    const Real* p = dz < 0 ? zm : (dz > 0 ? zp : cen);
    return p[(MF + a) * HP + h + dx + dy * TL::HX];
  }
};


// ------------------------------------------------------ the fused step
// Per cell: (a1) pull + moments + implicit drag, (c) reaction source,
// (b) FD transport of Y_k, T, Ts, low-Mach divergence, (a) source + BGK
// collision + store, (d) contribution to the FP64 reduction.
template <int DIM, int K, class Real, class Store, class Acc>
__device__ __forceinline__ Real cell_update(const Params<Real, K>& P, const State<Real, Store>& S,
                                            const Acc& A, int c, const int xyz[3], Real P0,
                                            Real dlnP0, Real dP0r, Real& fin, Real& fout) {
  using L = Lattice<DIM>;
  constexpr int Q = L::Q;
  constexpr int KK = Params<Real, K>::KK;
  constexpr Real CS2 = Real(1) / Real(3);
  auto at = [&](int f, int a, int s) -> Real { return A.n(f, a, s); };

  const Real T0 = A.c(F_T);
  const Real phis = A.c(F_PHI);
  const Real phif = Real(1) - phis;
  const Real rho = A.c(F_RHO);
  const Real mu = A.c(F_MU);
  const Real fD = A.c(F_FD);
  const Real Ts0 = A.c(F_TS);
  Real Y0[KK];
#pragma unroll
  for (int k = 0; k < K; ++k) Y0[k] = A.c(F_Y0 + k);
  const Real invMw = mixture_invMw(P, Y0);
  const Real cp = mixture_cp(P, Y0);
  const Real lam = mu * cp * P.inv_Pr;
  const Real Kd = P.Au_eta2 * mu * phif * phis * phis;
  const Real invT = fdiv(Real(1), T0);

  // cells on a non-periodic face (their pull takes the boundary rules)
  bool edge = (xyz[0] == 0 && P.bc[0] != BC_PERIODIC) || (xyz[0] == P.nx - 1 && P.bc[1] != BC_PERIODIC) ||
              (xyz[1] == 0 && P.bc[2] != BC_PERIODIC) || (xyz[1] == P.ny - 1 && P.bc[3] != BC_PERIODIC);
  if (DIM == 3)
    edge = edge || (xyz[2] == 0 && P.bc[4] != BC_PERIODIC) ||
           (xyz[2] == P.nz - 1 && P.bc[5] != BC_PERIODIC);

  // (a1) pull streaming, moments, implicit drag
  Real rho_in = 0;
  if (edge && P.bc[0] == BC_INLET) {
    Real Yin[KK];
#pragma unroll
    for (int k = 0; k < K; ++k) Yin[k] = P.Y_in[k];
    rho_in = fdiv(P0 * P.eos_cr, P.T_in * mixture_invMw(P, Yin));
  }
  constexpr bool FO = IsHalf<Store>::value;  // FP16 residual storage
  Real gin[Q];
  Real u[3] = {0, 0, 0}, uw[3] = {0, 0, 0}, mraw[3] = {0, 0, 0};
  const bool outlet_cell = P.bc[1] == BC_OUTLET && xyz[0] == P.nx - 1;
  const Real inv_rk = fdiv(Real(1), rho + Real(0.5) * Kd);
  for (int pass = 0; pass < (outlet_cell ? 2 : 1); ++pass) {
    if (Acc::has_pops && A.pv) {  // populations prefetched for this cell
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        // prefetched values are raw stored numbers (scaled residuals with FP16)
        gin[i] = A.template pop<Store>(i, Real(L::w(i)) * P.g_inv_scale);
        if constexpr (FO)
          gin[i] = Codec<Store, Real>::dec(gin[i], Real(L::w(i)) * P.g_inv_scale,
                                           first_order<DIM, Real>(A, i, 0, -L::c(i, 0), -L::c(i, 1),
                                                                  DIM == 3 ? -L::c(i, 2) : 0));
      }
    } else {
      pull<DIM>(P, S, c, xyz, rho, rho_in, uw, gin, A);
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      Real m = 0;
#pragma unroll
      for (int i = 0; i < Q; ++i)
        if (L::c(i, a) != 0) m += Real(L::c(i, a)) * gin[i];
      mraw[a] = m;
      u[a] = (m * Real(3) + Real(0.5) * (P.Fb[a] + Kd * P.u_s[a])) * inv_rk;
      uw[a] = u[a];
    }
  }
  Real sg = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) sg += gin[i];

  // the pulled populations are needed again only by the collision: with a
  // stash they wait in shared memory instead of 9 / 19 registers
  if constexpr (Acc::kStash) {
#pragma unroll
    for (int i = 0; i < Q; ++i) A.st[i * BLOCK + threadIdx.x] = gin[i];
  }

  const bool fluid_on = phif >= P.phi_min;
  const bool solid_on = P.Ts_field ? (phis >= P.phi_min) : true;
  Real SI = 0;
  if (fluid_on && solid_on)
    SI = P.mix ? P.AT_eta2 * A.c(F_KT) * phis * phis * (Ts0 - T0)  // staged phi_f lambda
               : P.AT_eta2 * lam * phif * phis * phis * (Ts0 - T0);

  // (c) reaction source
  Real om[KK], omT = 0;
#pragma unroll
  for (int k = 0; k < KK; ++k) om[k] = 0;
  if constexpr (K > 0) {
    if (P.chem == 1) rates(P, T0, Y0, rho, invT, om, omT);
    if (P.chem >= 2) {
      // increments of the chemistry pre-pass (implicit integrator or surrogate)
#pragma unroll
      for (int k = 0; k < K; ++k) om[k] = __ldg(S.src + (size_t)k * P.N + c);
      omT = __ldg(S.src + (size_t)K * P.N + c);
    }
  }

  const Real iphr = fluid_on ? fdiv(Real(1), phif * rho) : Real(0);
  const Real rf0 = A.c(F_RF);

  // (b) species; the face factors (phi_f rho f_D averaged over the face) are
  // shared by every species, and the central differences of Y_k feed the
  // enthalpy-flux cross term of the temperature equation
  Real Yn[KK];
  Real sYm = 0;  // sum_k (1/M_k) DY_k/Dt dt for the divergence
  Real sx[3] = {0, 0, 0};  // sum_k cp_k D_k (Y_k(+) - Y_k(-)) per axis
  {
    Real fm[DIM], fp[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      fm[a] = Real(0.5) * (rf0 + at(F_RF, a, -1));
      fp[a] = Real(0.5) * (rf0 + at(F_RF, a, +1));
    }
    // FP32: species in pairs with packed f32x2 arithmetic; the last one of an
    // odd count (and every species in FP64) one at a time
    constexpr int KP = sizeof(Real) == 4 ? (K / 2) * 2 : 0;
    if constexpr (KP > 0) {
      float2 sx2[3] = {splat2(0.f), splat2(0.f), splat2(0.f)}, sYm2 = splat2(0.f);
      const float2 prf = splat2(-phif * rho), pf = splat2(phif), ip = splat2(iphr);
#pragma unroll
      for (int k = 0; k < KP; k += 2) {
        const float2 y0 = make_float2(Y0[k], Y0[k + 1]);
        float2 adv = splat2(0.f), dif = splat2(0.f), cen = splat2(0.f);
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
          const float2 dm = sub2(y0, make_float2(at(F_Y0 + k, a, -1), at(F_Y0 + k + 1, a, -1)));
          const float2 dp = sub2(make_float2(at(F_Y0 + k, a, +1), at(F_Y0 + k + 1, a, +1)), y0);
          adv = fma2(splat2(u[a]), u[a] > 0.f ? dm : dp, adv);
          dif = fma2(splat2(fp[a]), dp, dif);
          dif = fma2(splat2(-fm[a]), dm, dif);
          const float2 sd = add2(dp, dm);
          cen = fma2(splat2(u[a]), sd, cen);
          sx2[a] = fma2(make_float2(P.cpD[k], P.cpD[k + 1]), sd, sx2[a]);
        }
        float2 dY = fma2(prf, adv, fma2(make_float2(P.Dlat[k], P.Dlat[k + 1]), dif,
                                        mul2(pf, make_float2(om[k], om[k + 1]))));
        dY = fluid_on ? mul2(dY, ip) : splat2(0.f);
        const float2 yn = add2(y0, dY);
        Yn[k] = yn.x;
        Yn[k + 1] = yn.y;
        // material increment: the step's increment plus u.grad Y_k (central)
        const float2 dm2 = fluid_on ? fma2(splat2(0.5f), cen, dY) : splat2(0.f);
        sYm2 = fma2(make_float2(P.invM[k], P.invM[k + 1]), dm2, sYm2);
      }
#pragma unroll
      for (int a = 0; a < DIM; ++a) sx[a] += sx2[a].x + sx2[a].y;
      sYm += sYm2.x + sYm2.y;
    }
#pragma unroll
    for (int k = KP; k < K; ++k) {
      Real adv = 0, dif = 0, cen = 0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const Real dm = Y0[k] - at(F_Y0 + k, a, -1), dp = at(F_Y0 + k, a, +1) - Y0[k];
        adv += u[a] * (u[a] > Real(0) ? dm : dp);
        dif += fp[a] * dp - fm[a] * dm;
        cen += u[a] * (dp + dm);
        sx[a] += P.cpD[k] * (dp + dm);
      }
      const Real dY = fluid_on ? (-phif * rho * adv + P.Dlat[k] * dif + phif * om[k]) * iphr
                               : Real(0);
      Yn[k] = Y0[k] + dY;
      // material increment: the step's increment plus u.grad Y_k (central)
      sYm += (fluid_on ? dY + Real(0.5) * cen : Real(0)) * P.invM[k];
    }
  }

  // (b) temperature
  Real Tn = Ts0, dTm = Ts0 - T0;  // frozen cells take the solid temperature
  if (fluid_on) {
    Real adv = 0, dif = 0, cross = 0, cen = 0;
    const Real kc = A.c(F_KT);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const Real tm = at(F_T, a, -1), tp = at(F_T, a, +1);
      adv += u[a] > Real(0) ? u[a] * (T0 - tm) : u[a] * (tp - T0);
      cen += u[a] * (tp - tm);
      const Real km = Real(0.5) * (kc + at(F_KT, a, -1));
      const Real kp = Real(0.5) * (kc + at(F_KT, a, +1));
      dif += kp * (tp - T0) - km * (T0 - tm);
      if constexpr (K > 0) cross += Real(0.25) * fD * sx[a] * (tp - tm);
    }
    const Real rhs = -phif * rho * cp * adv + dif + phif * (rho * cross + dP0r + omT + SI);
    const Real dTn = rhs * iphr * fdiv(Real(1), cp);
    Tn = T0 + dTn;
    dTm = dTn + Real(0.5) * cen;  // plus u.grad T (central)
  }

  // solid temperature
  if (P.Ts_field) {
    Real Tsn = Ts0;
    if (phis >= P.phi_min) {
      Real dif = 0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const Real km = Real(0.5) * (phis + at(F_PHI, a, -1)) * P.Lams;
        const Real kp = Real(0.5) * (phis + at(F_PHI, a, +1)) * P.Lams;
        dif += kp * (at(F_TS, a, +1) - Ts0) - km * (Ts0 - at(F_TS, a, -1));
      }
      Tsn = Ts0 + fdiv(dif - phif * SI, phis * P.Cs);
      if (P.moving) {
        // a moving solid carries its temperature with u_s (upwind)
        Real advs = 0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
          const Real us = P.u_s[a];
          if (us > Real(0)) advs += us * (Ts0 - at(F_TS, a, -1));
          else if (us < Real(0)) advs += us * (at(F_TS, a, +1) - Ts0);
        }
        Tsn -= advs;
      }
    }
    S.Ts_out[c] = Tsn;
  }

  // low-Mach divergence: continuity with the EOS at uniform P0,
  // D = (1/T) DT/Dt + Mw sum_k (1/M_k) DY_k/Dt - (1/P0) dP0/dt, the material
  // increments taken as the step's increments plus u.grad with central
  // differences, the gradient the source takes of rho (with the upwind
  // gradient the discrete continuity would keep a first-order mass defect)
  Real D = dTm * invT;
  if constexpr (K > 0) D += fdiv(sYm, invMw);
  D -= dlnP0;

  // (a) source and BGK collision: omega = 1/tau = 2 rho / (rho + 6 mu)
  Real G[3] = {0, 0, 0}, F[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    G[a] = CS2 * Real(0.5) * (at(F_RHO, a, +1) - at(F_RHO, a, -1));
    F[a] = P.Fb[a] - Kd * (u[a] - P.u_s[a]);
  }
  // P_h: the pulled zeroth moment plus half the zeroth moment of the source,
  // sum_i Xi_i = u.G + rho cs^2 D, so that a step adds the whole source
  Real uG = 0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) uG += u[a] * G[a];
  const Real Ph = sg + Real(0.5) * (rho * CS2 * D + uG);
  if (P.nscbc && xyz[0] >= P.nx - 2) {
    // the two outlet columns of this step for the characteristic outlet
    const int NF = P.ny * P.nz, f = xyz[1] + P.ny * xyz[2];
    const int col = xyz[0] == P.nx - 1 ? 0 : 1;
    S.ob[(size_t)(2 * col) * NF + f] = Ph;
    S.ob[(size_t)(2 * col + 1) * NF + f] = u[0];
    if (col == 0) S.ob[(size_t)4 * NF + f] = rho;
  }
  const Real omega = fdiv(Real(2) * rho, rho + Real(6) * mu);
  const Real src_w = Real(1) - Real(0.5) * omega;
  // f_eq / rho - w = w e with e = 3 cu + 9/2 cu^2 - 3/2 uu;
  // g_eq = cs2 f_eq + w (P_h - rho cs2) = w (P_h + rho e / 3);
  // Xi = w [(c - u).(G e + F (1 + e)) + rho cs2 D] = w [(c.H - u.H) e + c.F - u.F + rho cs2 D]
  // with H = G + F.  Collected per cell: g* = (1 - omega) g + w [A0 + B e + src_w x],
  // A0 = omega P_h + src_w rho cs2 D, B = omega rho cs2, x = (c.H - u.H) e + c.F - u.F.
  Real H[3] = {0, 0, 0};
  Real uu = 0, uH = 0, uF = 0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    H[a] = G[a] + F[a];
    uu += u[a] * u[a];
    uH += u[a] * H[a];
    uF += u[a] * F[a];
  }
  const Real rho3 = rho * CS2;
  const Real A0 = omega * Ph + src_w * (rho3 * D);
  const Real B = omega * rho3;
  const Real uu15 = Real(1.5) * uu;
  const Real keep = Real(1) - omega;
  // FP16 storage: the post-collision moments of this cell in closed form
  // (sum_i w_i e_i = 0, sum_i w_i x_i = u.G, sum_i w_i c_i e_i = u,
  // sum_i w_i c_i x_i = F / 3 on the isotropic lattice); any values would do,
  // since readers add back exactly what is subtracted here, but these leave
  // a residual of second order in u
  Real Pst = 0, jst[3] = {0, 0, 0};
  if constexpr (FO) {
    Pst = keep * sg + A0 + src_w * (uH - uF);
#pragma unroll
    for (int a = 0; a < DIM; ++a) jst[a] = keep * mraw[a] + B * u[a] + src_w * CS2 * F[a];
  }
  // FP32 updates a direction and its opposite together with packed f32x2
  // arithmetic (c.u, c.H, c.F of the opposite are the negated ones); the rest
  // direction, and every direction in FP64, one at a time
  constexpr bool PAIRS = sizeof(Real) == 4;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if constexpr (PAIRS) {
      if (L::opp(i) < i) continue;  // done with its opposite
    }
    Real cu = 0, cH = 0, cF = 0, cj = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      if (L::c(i, a) > 0) { cu += u[a]; cH += H[a]; cF += F[a]; cj += jst[a]; }
      if (L::c(i, a) < 0) { cu -= u[a]; cH -= H[a]; cF -= F[a]; cj -= jst[a]; }
    }
    Real gi = gin[i];
    if constexpr (Acc::kStash) gi = A.st[i * BLOCK + threadIdx.x];
    if constexpr (PAIRS) {
      if (i > 0) {
        const int j = L::opp(i);
        Real gj = gin[j];
        if constexpr (Acc::kStash) gj = A.st[j * BLOCK + threadIdx.x];
        const float2 cu2 = make_float2(cu, -cu);
        const float2 e = fma2(cu2, fma2(cu2, splat2(4.5f), splat2(3.f)), splat2(-uu15));
        const float2 x = fma2(sub2(make_float2(cH, -cH), splat2(uH)), e,
                              sub2(make_float2(cF, -cF), splat2(uF)));
        float2 t = fma2(splat2(B), e, splat2(A0));
        t = fma2(splat2(src_w), x, t);
        const float w = float(L::w(i));
        float2 g = fma2(splat2(keep), make_float2(gi, gj), mul2(splat2(w), t));
        if constexpr (FO)
          g = sub2(g, mul2(splat2(w), fma2(splat2(3.f), make_float2(cj, -cj), splat2(Pst))));
        Codec<Store, Real>::store(S.g_out + (size_t)i * P.N + c, g.x,
                                  P.g_scale * Real(1.0 / L::w(i)));
        Codec<Store, Real>::store(S.g_out + (size_t)j * P.N + c, g.y,
                                  P.g_scale * Real(1.0 / L::w(j)));
        continue;
      }
    }
    const Real w = Real(L::w(i));
    const Real e = cu * (Real(3) + Real(4.5) * cu) - uu15;
    const Real x = (cH - uH) * e + (cF - uF);
    Real g = keep * gi + w * (A0 + B * e + src_w * x);
    if constexpr (FO) g -= w * (Pst + Real(3) * cj);
    Codec<Store, Real>::store(S.g_out + (size_t)i * P.N + c, g, P.g_scale * Real(1.0 / L::w(i)));
  }
  if constexpr (FO) {
    S.M_out[c] = Pst;
#pragma unroll
    for (int a = 0; a < DIM; ++a) S.M_out[(size_t)(1 + a) * P.N + c] = jst[a];
  }

  S.T_out[c] = Tn;
#pragma unroll
  for (int k = 0; k < K; ++k) S.Y_out[(size_t)k * P.N + c] = Yn[k];

  // (d) contributions to the reduction
  const Real fx = phif * rho * u[0];
  fin = (xyz[0] == 0 && P.bc[0] == BC_INLET) ? fx : Real(0);
  fout = outlet_cell ? fx : Real(0);
  // 0 * P_h is NaN when any pulled population is: a NaN confined to the
  // populations reaches the FP64 reduction (and the status word) this step
  return phif * fdiv(Real(1), Tn * mixture_invMw(P, Yn)) + Real(0) * Ph;
}

// Resident blocks per SM requested from the register allocator: 2-D FP32 /
// FP16 storage at <= 64 registers (4 blocks), 3-D FP32 at <= 80 (3 blocks),
// 3-D FP16 storage, whose decode holds the source cells' moments, at <= 128
// (2 blocks); FP64 is bound by the FP64 pipe and keeps the registers it needs.
template <int DIM, class Real, class Store> struct MinBlocks {
  static constexpr int value =
      sizeof(Real) == 8 ? (DIM == 3 ? 1 : 2) : (DIM == 2 ? 4 : (IsHalf<Store>::value ? 2 : 3));
};

// One tile of the fused step (tile (bx, by) of the xy grid, z-chunk bz in
// 3-D): stages the tile's planes in `planes` (shared memory), updates its
// cells and returns the block sums of the reduction in thread 0 (I, inlet
// flux, outlet flux).  Every thread of the block calls it.
template <int DIM, int K, class Real, class Store, class T_ = Tile<DIM>>
__device__ __forceinline__ void step_tile(const Params<Real, K>& P, const State<Real, Store>& S,
                                          int bx, int by, int bz,
                                          Plane<Real, K, T_::HP, n_mom<DIM, Store>()>* planes,
                                          double* red_sh,
                                          double& sI, double& sIn, double& sOut) {
  const Real P0 = scal_P0<Real>(S.scal);
  const Real dlnP0 = scal_dlnP0<Real>(S.scal);
  const Real dP0r = scal_dP0r<Real>(S.scal);

  const int tx = threadIdx.x % T_::TX, ty = threadIdx.x / T_::TX;
  const int x0 = bx * T_::TX, y0 = by * T_::TY;
  const int x = x0 + tx, y = y0 + ty;
  const int h = (ty + 1) * T_::HX + (tx + 1);
  const bool in_xy = x < P.nx && y < P.ny;
  const int z_begin = bz * T_::ZC;
  const int z_end = DIM == 3 ? min(z_begin + T_::ZC, P.nz) : 1;
  const bool flux_block = (x0 == 0 && P.bc[0] == BC_INLET) ||
                          (x0 + T_::TX >= P.nx && P.bc[1] == BC_OUTLET);

  Real accI = 0, accIn = 0, accOut = 0;
  if constexpr (DIM == 2) {
    using L = Lattice<2>;
    constexpr int RPT = T_::RPT;
    constexpr int RS = T_::TY / RPT;  // row stride between a thread's cells
    // population loads of the thread's interior cells, issued before staging
    Real pre[RPT][L::Q];
    bool pv[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) pv[r] = false;
    if constexpr (T_::PREFETCH) {
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const int yr = y0 + ty + r * RS;
        const bool inner = x > 0 && x < P.nx - 1 && yr > 0 && yr < P.ny - 1;
        pv[r] = inner;
        if (inner) {
          const int c = x + P.nx * yr;
#pragma unroll
          for (int i = 0; i < L::Q; ++i)
            pre[r][i] = Codec<Store, Real>::raw(
                S.g_in + (size_t)i * P.N + c - L::c(i, 0) - L::c(i, 1) * P.nx);
        }
      }
    }
    stage_plane<DIM, Real, Store, K, T_::HP, T_>(P, S, planes[0], x0, y0, 0, P0);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int yr = y0 + ty + r * RS;
      if (x < P.nx && yr < P.ny) {
        const int c = x + P.nx * yr;
        const int xyz[3] = {x, yr, 0};
        const int hr = (ty + r * RS + 1) * T_::HX + (tx + 1);
        Real fi, fo;
        const PlaneAcc<DIM, Real, T_::PREFETCH, T_, F_Y0 + K> A{&planes[0].f[0][0], nullptr,
                                                                nullptr, hr, pre[r], pv[r],
                                                                nullptr};
        accI += cell_update<DIM, K, Real, Store>(P, S, A, c, xyz, P0, dlnP0, dP0r, fi, fo);
        accIn += fi;
        accOut += fo;
      }
    }
  } else {
    // ring of three staged planes: slot (z mod 3)
    stage_plane<DIM, Real, Store, K, T_::HP, T_>(P, S, planes[(z_begin + 2) % 3], x0, y0,
                                                 z_begin - 1, P0);
    stage_plane<DIM, Real, Store, K, T_::HP, T_>(P, S, planes[z_begin % 3], x0, y0, z_begin, P0);
    for (int z = z_begin; z < z_end; ++z) {
      stage_plane<DIM, Real, Store, K, T_::HP, T_>(P, S, planes[(z + 1) % 3], x0, y0, z + 1, P0);
      __syncthreads();
      if (in_xy) {
        const int c = x + P.nx * (y + P.ny * z);
        const int xyz[3] = {x, y, z};
        Real fi, fo;
        const PlaneAcc<DIM, Real, false, T_, F_Y0 + K, true> A{
            &planes[z % 3].f[0][0], &planes[(z + 2) % 3].f[0][0],
            &planes[(z + 1) % 3].f[0][0], h, nullptr, false,
            reinterpret_cast<Real*>(planes + T_::NPL)};
        accI += cell_update<DIM, K, Real, Store>(P, S, A, c, xyz, P0, dlnP0, dP0r, fi, fo);
        accIn += fi;
        accOut += fo;
      }
      __syncthreads();
    }
  }

  // (d) block partials in FP64 (one barrier)
  block_sum3<Real>(accI, accIn, accOut, flux_block, red_sh, sI, sIn, sOut);
}

template <int DIM, int K, class Real, class Store>
__global__ void __launch_bounds__(BLOCK, MinBlocks<DIM, Real, Store>::value)
step_kernel(const Params<Real, K> P, const State<Real, Store> S, int p0_closed,
            const double* __restrict__ prev_partials, unsigned prev_nb) {
  using T_ = Tile<DIM>;
  using PL = Plane<Real, K, T_::HP, n_mom<DIM, Store>()>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PL* planes = reinterpret_cast<PL*>(smem_raw);
  __shared__ double red_sh[96];

  // deferred combine of the previous step's partials (fixed P0 only): block
  // 0's first warp does it while the other blocks start on their cells
  if (prev_partials && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 &&
      threadIdx.x < 32)
    combine_partials(prev_partials, prev_nb, S.scal, 0, false, 0.0, P.eos_c, P.inv_rho_ref);

  double sI, sIn, sOut;
  step_tile<DIM, K, Real, Store, T_>(P, S, blockIdx.x, blockIdx.y, blockIdx.z, planes, red_sh,
                                     sI, sIn, sOut);
  // deterministic finish by the last block (closed P0) or deferred
  publish_partials(sI, sIn, sOut, S.partials, S.counter, S.scal, p0_closed, false, 0.0, P.eos_c,
                   P.inv_rho_ref);
}

// Persistent variant of the 2-D step: one grid of resident blocks walks the
// tiles, handed out by an atomic counter (one per step parity; each launch
// clears the other one for the next step), so no block waits for a second
// wave and cheap tiles do not leave SMs idle.  Reduction slots are the tile
// indices, as in step_kernel.
template <int DIM, int K, class Real, class Store, class T_>
__global__ void __launch_bounds__(BLOCK, (sizeof(Real) == 8 ? 2 : (T_::RPT > 1 ? 3 : 4)))
step_persistent_kernel(const Params<Real, K> P, const State<Real, Store> S, int p0_closed,
                       const double* __restrict__ prev_partials, unsigned prev_nb,
                       unsigned* __restrict__ tile_ctr, int parity) {
  static_assert(DIM == 2, "the persistent step walks 2-D tiles");
  using PL = Plane<Real, K, T_::HP, n_mom<DIM, Store>()>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PL* planes = reinterpret_cast<PL*>(smem_raw);
  __shared__ double red_sh[96];
  __shared__ int next_sh[2];

  if (prev_partials && blockIdx.x == 0 && threadIdx.x < 32)
    combine_partials(prev_partials, prev_nb, S.scal, 0, false, 0.0, P.eos_c, P.inv_rho_ref);

  const int nbx = (P.nx + T_::TX - 1) / T_::TX;
  const int total = nbx * ((P.ny + T_::TY - 1) / T_::TY);
  unsigned* ctr = tile_ctr + parity;
  if (threadIdx.x == 0) {
    if (blockIdx.x == 0) tile_ctr[parity ^ 1] = 0u;  // the next step's counter
    next_sh[0] = (int)atomicAdd(ctr, 1u);
  }
  __syncthreads();
  int par = 0;
  for (int t = next_sh[0]; t < total; t = next_sh[par]) {
    // draw the next tile now; the tile's staging barrier publishes it
    par ^= 1;
    if (threadIdx.x == 0) next_sh[par] = (int)atomicAdd(ctr, 1u);
    double sI, sIn, sOut;
    step_tile<DIM, K, Real, Store, T_>(P, S, t % nbx, t / nbx, 0, planes, red_sh, sI, sIn,
                                       sOut);
    publish_partials_at(sI, sIn, sOut, S.partials, S.counter, S.scal, p0_closed, false, 0.0,
                        P.eos_c, P.inv_rho_ref, (unsigned)t, (unsigned)total, p0_closed != 0);
  }
}

// staged planes, and in 3-D the stash of the pulled populations
template <int DIM, int K, class Real, class Store, class T_ = Tile<DIM>>
constexpr size_t step_smem_bytes() {
  return sizeof(Plane<Real, K, T_::HP, n_mom<DIM, Store>()>) * T_::NPL +
         (DIM == 3 ? sizeof(Real) * Lattice<DIM>::Q * BLOCK : 0);
}

// ------------------------------------------- chemistry pre-pass (implicit)
// Per cell: backward-Euler Newton increments over the step at (T^n, Y^n,
// rho^n), stored as the FD source terms rho* dY_k and rho* cp dT.
template <int K, class Real, class Store>
__global__ void __launch_bounds__(BLOCK)
chem_implicit_kernel(const __grid_constant__ Params<Real, K> P, const State<Real, Store> S,
                     Real* __restrict__ src) {
  constexpr int KK = K > 0 ? K : 1;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P.N) return;
  const Real T = S.T_in[c];
  Real Y[KK];
#pragma unroll
  for (int k = 0; k < K; ++k) Y[k] = S.Y_in[(size_t)k * P.N + c];
  const Real phif = Real(1) - S.phi[c];
  Real om[KK], omT = 0;
#pragma unroll
  for (int k = 0; k < KK; ++k) om[k] = 0;
  if (phif >= P.phi_min) {
    const Real P0 = scal_P0<Real>(S.scal);
    const Real rho = fdiv(P0 * P.eos_cr, T * mixture_invMw(P, Y));
    double Yd[KK], dY[KK], dT;
#pragma unroll
    for (int k = 0; k < K; ++k) Yd[k] = double(Y[k]);
    chem_be_newton<K, Real>(&P.c64, double(T), Yd, double(rho) * P.c64.rho_ref, dY, &dT);
#pragma unroll
    for (int k = 0; k < K; ++k) om[k] = rho * Real(dY[k]);
    omT = rho * mixture_cp(P, Y) * Real(dT);
  }
#pragma unroll
  for (int k = 0; k < K; ++k) src[(size_t)k * P.N + c] = om[k];
  src[(size_t)K * P.N + c] = omT;
}

// ------------------------------------------------ inlet feedback
// Sec. 4.4.1: the inflow of species feed_k is matched to its consumption.
// After the step kernel of step n, whose inputs (T, Y and the pre-pass
// increments) are still in place, feed_kernel sums phi_f (-omega_k) of that
// state over the cells (FP64 block partials, grid-stride over at most
// kFeedBlocks blocks) and feed_combine_kernel sums the partials in a fixed
// order and sets the inlet peak speed of step n + 1.
constexpr int kFeedBlocks = 1024;

template <int K, class Real, class Store>
__global__ void __launch_bounds__(BLOCK)
feed_kernel(const Params<Real, K> P, const State<Real, Store> S, double* __restrict__ part) {
  constexpr int KK = Params<Real, K>::KK;
  __shared__ double red_sh[32];
  double acc = 0;
  if constexpr (K > 0) {
    const Real P0 = scal_P0<Real>(S.scal);
    for (int c = blockIdx.x * BLOCK + threadIdx.x; c < P.N; c += gridDim.x * BLOCK) {
      const Real phif = Real(1) - S.phi[c];
      if (!(phif >= P.phi_min)) continue;
      Real om[KK], omT = 0;
      if (P.chem == 1) {
        const Real T = S.T_in[c];
        Real Y[KK];
#pragma unroll
        for (int k = 0; k < K; ++k) Y[k] = S.Y_in[(size_t)k * P.N + c];
        const Real rho = fdiv(P0 * P.eos_cr, T * mixture_invMw(P, Y));
        rates(P, T, Y, rho, fdiv(Real(1), T), om, omT);
        acc += double(phif * -om[P.feed_k]);
      } else if (P.chem >= 2) {
        acc += double(phif * -S.src[(size_t)P.feed_k * P.N + c]);
      }
    }
  }
  const double s = block_sum<double>(acc, red_sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// One warp: u_in = fuel feed_c / P0, held in [0, 0.3].
static __global__ void feed_combine_kernel(const double* __restrict__ part, unsigned nb,
                                           DevScalars* scal, double feed_c) {
  const int lane = threadIdx.x;
  double v = 0;
  for (unsigned b = lane; b < nb; b += 32) v += part[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) {
    double u = v * feed_c / scal->P0;
    u = u > 0.3 ? 0.3 : (u > 0.0 ? u : 0.0);  // NaN -> 0
    scal->fuel = v;
    scal->u_in = u;
    scal->u_in_f = float(u);
  }
}

// The inlet speed of the first step (and no consumption yet); the
// characteristic outlet starts at the ambient pressure.
static __global__ void set_inlet_kernel(DevScalars* scal, double u_in) {
  scal->u_in = u_in;
  scal->u_in_f = float(u_in);
  scal->fuel = 0.0;
  scal->pb = 0.0;
  scal->pb_f = 0.f;
}

// ------------------------------------------------ moving solid
// Phase field of step n of a rigidly translating solid: the step-0 field phi0
// displaced by s = n u_s, multilinear interpolation between the cells around
// x - s; per axis the host passes the whole shift ish and the fraction fr in
// [0, 1).  Periodic axes wrap, other axes clamp.
template <int DIM, class Real>
__global__ void __launch_bounds__(BLOCK)
phase_shift_kernel(const Real* __restrict__ phi0, Real* __restrict__ phi, int nx, int ny, int nz,
                   int per_mask, int3 ish, Real fx, Real fy, Real fz) {
  const int c = blockIdx.x * BLOCK + threadIdx.x;
  const int N = nx * ny * nz;
  if (c >= N) return;
  const int xyz[3] = {c % nx, (c / nx) % ny, c / (nx * ny)};
  const int ext[3] = {nx, ny, nz}, sh[3] = {ish.x, ish.y, ish.z};
  const Real fr[3] = {fx, fy, fz};
  Real v = 0;
#pragma unroll
  for (int corner = 0; corner < (1 << DIM); ++corner) {
    Real w = 1;
    int q[3] = {xyz[0], xyz[1], xyz[2]};
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int up = (corner >> a) & 1;
      w *= up ? fr[a] : Real(1) - fr[a];
      int qa = xyz[a] - sh[a] - up;
      if ((per_mask >> a) & 1) qa = ((qa % ext[a]) + ext[a]) % ext[a];
      else qa = qa < 0 ? 0 : (qa >= ext[a] ? ext[a] - 1 : qa);
      q[a] = qa;
    }
    v += w * phi0[q[0] + nx * (q[1] + ny * q[2])];
  }
  phi[c] = v;
}

// ------------------------------------------------ characteristic outlet
// Sec. 4.1 (Poinsot and Lele): after a step, one block forms the face means
// of the outlet columns it wrote (fixed-order FP64 sums) and advances the
// boundary pressure, P_b <- P_b - (L5 + K P_b) / 2 with
// L5 = (u + cs)((P1 - P2) + rho cs (u1 - u2)).
template <class Real>
__global__ void __launch_bounds__(BLOCK)
outlet_kernel(const Real* __restrict__ ob, int NF, DevScalars* scal, double K) {
  __shared__ double red_sh[32];
  double v[5] = {0, 0, 0, 0, 0};
  for (int f = threadIdx.x; f < NF; f += BLOCK)
#pragma unroll
    for (int q = 0; q < 5; ++q) v[q] += double(ob[(size_t)q * NF + f]);
  double m[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) m[q] = block_sum<double>(v[q], red_sh) / NF;
  if (threadIdx.x == 0) {
    const double cs = 0.57735026918962576;  // sqrt(1/3)
    const double P1 = m[0], u1 = m[1], P2 = m[2], u2 = m[3], r = m[4];
    const double pb = scal->pb;
    const double L5 = (u1 + cs) * ((P1 - P2) + r * cs * (u1 - u2));
    const double nb = pb - 0.5 * (L5 + K * pb);
    scal->pb = nb;
    scal->pb_f = float(nb);
  }
}

// ------------------------------------------------ initial equilibrium
// g = g_eq(P_h = 0, rho, u); reduction of I = sum phi_f Mw / T for the mass m.
template <int DIM, int K, class Real, class Store>
__global__ void __launch_bounds__(BLOCK)
init_kernel(const Params<Real, K> P, const State<Real, Store> S, const Real* __restrict__ u_init,
            double P0_init) {
  using L = Lattice<DIM>;
  __shared__ double red_sh[32];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  Real acc = 0;
  if (c < P.N) {
    const Real T = S.T_in[c];
    Real Y[Params<Real, K>::KK];
#pragma unroll
    for (int k = 0; k < K; ++k) Y[k] = S.Y_in[(size_t)k * P.N + c];
    const Real invMw = mixture_invMw(P, Y);
    const Real rho = Real(P0_init) * Real(P.eos_c) / (T * invMw);
    Real u[3] = {0, 0, 0};
    if (u_init)
      for (int a = 0; a < DIM; ++a) u[a] = u_init[(size_t)a * P.N + c];
    Real uu = 0;
    for (int a = 0; a < DIM; ++a) uu += u[a] * u[a];
    // FP16 storage: moments P = 0, j = rho u / 3 of g_eq; the stored residual
    // drops the first-order part w rho c.u
    constexpr bool FO = IsHalf<Store>::value;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const Real w = Real(L::w(i));
      Real cu = 0;
      for (int a = 0; a < DIM; ++a) cu += Real(L::c(i, a)) * u[a];
      const Real geq = w * rho * ((FO ? Real(0) : cu) + Real(1.5) * cu * cu - Real(0.5) * uu);
      Codec<Store, Real>::store(S.g_out + (size_t)i * P.N + c, geq, P.g_scale * Real(1.0 / L::w(i)));
    }
    if constexpr (FO) {
      S.M_out[c] = Real(0);
      for (int a = 0; a < DIM; ++a) S.M_out[(size_t)(1 + a) * P.N + c] = rho * u[a] * Real(1.0 / 3.0);
    }
    acc = (Real(1) - S.phi[c]) / (T * invMw);
  }
  const double s = block_sum<Real>(acc, red_sh);
  publish_partials(s, 0.0, 0.0, S.partials, S.counter, S.scal, 0, true, P0_init, P.eos_c,
                   P.inv_rho_ref);
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
  const Real T = S.T_in[c];
  Real Y[KK];
#pragma unroll
  for (int k = 0; k < K; ++k) Y[k] = S.Y_in[(size_t)k * P.N + c];
  const Real rho = P0 * Real(P.eos_c) / (T * mixture_invMw(P, Y));
  const Real phis = S.phi[c];
  Real mu_c, lam_c;
  transport(P, T, Y, mixture_invMw(P, Y), mixture_cp(P, Y), mu_c, lam_c);
  const Real Kd = P.Au_eta2 * mu_c * (Real(1) - phis) * phis * phis;
  Real Yin[KK];
#pragma unroll
  for (int k = 0; k < K; ++k) Yin[k] = P.Y_in[k];
  const Real rho_in = P0 * Real(P.eos_c) / (P.T_in * mixture_invMw(P, Yin));
  const bool outlet_cell = P.bc[1] == BC_OUTLET && xyz[0] == P.nx - 1;
  Real gin[Q], u[3] = {0, 0, 0}, uw[3] = {0, 0, 0};
  for (int pass = 0; pass < (outlet_cell ? 2 : 1); ++pass) {
    pull<DIM>(P, S, c, xyz, rho, rho_in, uw, gin, GlobalMom<Real>{S.M_in, P.N});
    for (int a = 0; a < DIM; ++a) {
      Real m = 0;
      for (int i = 0; i < Q; ++i) m += Real(L::c(i, a)) * gin[i];
      u[a] = (m * Real(3) + Real(0.5) * (P.Fb[a] + Kd * P.u_s[a])) / (rho + Real(0.5) * Kd);
      uw[a] = u[a];
    }
  }
  Real sg = 0;
  for (int i = 0; i < Q; ++i) sg += gin[i];
  for (int a = 0; a < DIM; ++a) u_out[(size_t)a * P.N + c] = double(u[a]);
  rho_out[c] = double(rho);
  ph_out[c] = double(sg);
}

// ------------------------------------------------- diagnostics (on demand)
// Per-cell terms of the domain diagnostics of the state the next step sees,
// summed per block in FP64: drag sum K_d u (the force of the fluid on the
// solid phase, Sec. 3.2.1), heat sum phi_f S_I (Sec. 3.3, eq.
// diffusion-heat-flux-3), fluid mass sum phi_f rho, and over the outlet
// column rho u_x cp T and rho u_x cp (mixing-cup temperature, Sec. 4.2).
constexpr int NDIAG = 8;
template <int DIM, int K, class Real, class Store>
__global__ void __launch_bounds__(BLOCK)
diag_kernel(const Params<Real, K> P, const State<Real, Store> S, double* __restrict__ part) {
  using L = Lattice<DIM>;
  constexpr int Q = L::Q;
  constexpr int KK = Params<Real, K>::KK;
  __shared__ double red_sh[32];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double v[NDIAG] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (c < P.N) {
    const Real P0 = Real(S.scal->P0);
    int xyz[3];
    xyz[0] = c % P.nx;
    xyz[1] = (c / P.nx) % P.ny;
    xyz[2] = DIM == 3 ? c / (P.nx * P.ny) : 0;
    const Real T = S.T_in[c];
    Real Y[KK];
#pragma unroll
    for (int k = 0; k < K; ++k) Y[k] = S.Y_in[(size_t)k * P.N + c];
    const Real rho = P0 * Real(P.eos_c) / (T * mixture_invMw(P, Y));
    const Real phis = S.phi[c], phif = Real(1) - phis;
    const Real cp = mixture_cp(P, Y);
    Real mu, lam;
    transport(P, T, Y, mixture_invMw(P, Y), cp, mu, lam);
    const Real Kd = P.Au_eta2 * mu * phif * phis * phis;
    Real Yin[KK];
#pragma unroll
    for (int k = 0; k < K; ++k) Yin[k] = P.Y_in[k];
    const Real rho_in = P0 * Real(P.eos_c) / (P.T_in * mixture_invMw(P, Yin));
    const bool outlet_cell = P.bc[1] == BC_OUTLET && xyz[0] == P.nx - 1;
    Real gin[Q], u[3] = {0, 0, 0}, uw[3] = {0, 0, 0};
    for (int pass = 0; pass < (outlet_cell ? 2 : 1); ++pass) {
      pull<DIM>(P, S, c, xyz, rho, rho_in, uw, gin, GlobalMom<Real>{S.M_in, P.N});
      for (int a = 0; a < DIM; ++a) {
        Real m = 0;
        for (int i = 0; i < Q; ++i) m += Real(L::c(i, a)) * gin[i];
        u[a] = (m * Real(3) + Real(0.5) * (P.Fb[a] + Kd * P.u_s[a])) / (rho + Real(0.5) * Kd);
        uw[a] = u[a];
      }
    }
    for (int a = 0; a < DIM; ++a) v[a] = double(Kd * (u[a] - P.u_s[a]));
    const Real Ts = P.Ts_field ? S.Ts_in[c] : P.Ts_uniform;
    const bool fluid_on = phif >= P.phi_min;
    const bool solid_on = P.Ts_field ? (phis >= P.phi_min) : true;
    if (fluid_on && solid_on)
      v[3] = double(phif * (P.AT_eta2 * lam * phif * phis * phis * (Ts - T)));
    v[4] = double(phif * rho);
    if (outlet_cell) {
      v[5] = double(rho * u[0] * cp * T);
      v[6] = double(rho * u[0] * cp);
    }
  }
#pragma unroll
  for (int k = 0; k < NDIAG; ++k) {
    const double s = block_sum<double>(v[k], red_sh);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * NDIAG + k] = s;
  }
}

// Fixed-order sum of the block partials (one warp).
static __global__ void diag_combine_kernel(const double* __restrict__ part, int nb,
                                           double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  for (int k = 0; k < NDIAG; ++k) {
    double s = 0;
    for (int b = lane; b < nb; b += 32) s += part[(size_t)b * NDIAG + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[k] = s;
  }
}

}  // namespace pflb
