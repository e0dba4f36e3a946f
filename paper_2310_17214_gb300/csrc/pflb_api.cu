// pflb_api.cu -- the extern "C" boundary of libpflb.so (declared in
// include/pflb.h): domain lifetime, field transfer, stepping, scalars.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "../../include/pflb.h"
#include "pflb_launch.cuh"
#include "pflb_validate.cuh"

using namespace pflb;

struct pflb_domain {
  pflb_domain_desc desc;
  pflb_mechanism mech;
  int K = 0, Q = 0, N = 0, mode = 0, dim = 2;
  size_t real_sz = 8, store_sz = 8;
  cudaStream_t stream = nullptr;
  Buffers B;
  int cur = 0;
  bool has_mech = false, has_phase = false, has_fields = false;
  Launcher* L = nullptr;
  long long wait_limit = kDefaultWaitCycles;
  std::string err;
};

static thread_local std::string g_create_err;

namespace {

int fail(pflb_domain* d, int code, const char* fmt, const char* a = "") {
  char buf[512];
  std::snprintf(buf, sizeof(buf), fmt, a);
  if (d) d->err = buf;
  else g_create_err = buf;
  return code;
}

#define CK(d, call)                                                     \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) return fail(d, PFLB_ERR_CUDA, "%s", cudaGetErrorString(e_)); \
  } while (0)

template <class S, class D>
__global__ void convert_kernel(const S* __restrict__ s, D* __restrict__ d, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    d[i] = D(s[i]);
}

struct Weights {
  float w_over_scale[19], w[19];
  int c[19][3];
  int Q, dim;
};

// Stored populations -> populations.  FP16 storage keeps residuals from the
// cell's first-order equilibrium: g_i = w_i (P + 3 c_i . j) + h_i w_i / S.
template <class Store, class D>
__global__ void decode_g_kernel(const Store* __restrict__ s, const float* __restrict__ M,
                                D* __restrict__ d, size_t N, Weights W) {
  const size_t n = N * (size_t)W.Q;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    if constexpr (sizeof(Store) == 2) {
      const size_t q = i / N, c = i - q * N;
      float cj = 0.f;
      for (int a = 0; a < W.dim; ++a) cj += float(W.c[q][a]) * M[(1 + a) * N + c];
      d[i] = D(__half2float(s[i]) * W.w_over_scale[q] + W.w[q] * (M[c] + 3.f * cj));
    } else {
      d[i] = D(s[i]);
    }
  }
}

template <class D>
__global__ void fill_kernel(D* __restrict__ d, D v, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    d[i] = v;
}

template <class S, class D>
cudaError_t convert(const void* s, void* d, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  convert_kernel<S, D><<<blocks, 256, 0, st>>>(static_cast<const S*>(s), static_cast<D*>(d), n);
  return cudaGetLastError();
}

// copy n values of dtype `dt` at `src` (host or device) into the compute-type
// device array `dst` (double or float)
int upload(pflb_domain* d, const void* src, int dt, int where, void* dst, size_t n) {
  const size_t esz = dt == PFLB_DTYPE_F64 ? 8 : 4;
  const void* dev = src;
  void* stage = nullptr;
  if (where == PFLB_HOST) {
    CK(d, cudaMallocAsync(&stage, n * esz, d->stream));
    CK(d, cudaMemcpyAsync(stage, src, n * esz, cudaMemcpyHostToDevice, d->stream));
    dev = stage;
  }
  cudaError_t e;
  if (d->real_sz == 8) e = dt == PFLB_DTYPE_F64 ? convert<double, double>(dev, dst, n, d->stream)
                                                : convert<float, double>(dev, dst, n, d->stream);
  else e = dt == PFLB_DTYPE_F64 ? convert<double, float>(dev, dst, n, d->stream)
                                : convert<float, float>(dev, dst, n, d->stream);
  if (stage) cudaFreeAsync(stage, d->stream);
  CK(d, e);
  return PFLB_OK;
}

int check_dtype_where(pflb_domain* d, int dt, int where) {
  if (dt != PFLB_DTYPE_F64 && dt != PFLB_DTYPE_F32) return fail(d, PFLB_ERR_ARG, "bad dtype");
  if (where != PFLB_HOST && where != PFLB_DEVICE) return fail(d, PFLB_ERR_ARG, "bad where");
  return PFLB_OK;
}

Launcher* make_launcher(const pflb_domain* d) {
  const int K = d->K, m = d->mode;
  if (d->dim == 2) {
    if (m == MODE_FP64) return make_launcher_2d_fp64(K, d->desc, d->mech);
    if (m == MODE_FP32) return make_launcher_2d_fp32(K, d->desc, d->mech);
    return make_launcher_2d_fp16(K, d->desc, d->mech);
  }
  if (m == MODE_FP64) return make_launcher_3d_fp64(K, d->desc, d->mech);
  if (m == MODE_FP32) return make_launcher_3d_fp32(K, d->desc, d->mech);
  return make_launcher_3d_fp16(K, d->desc, d->mech);
}

void free_buffers(pflb_domain* d) {
  void* ptrs[] = {d->B.g[0], d->B.g[1], d->B.M[0], d->B.M[1], d->B.T[0], d->B.T[1], d->B.Y[0], d->B.Y[1],
                  d->B.Ts[0], d->B.Ts[1], d->B.phi, d->B.scal, d->B.partials, d->B.counter,
                  d->B.src, d->B.fb_idx, d->B.fb_count, d->B.chem_stats, d->B.tile_ctr,
                  d->B.feed_part, d->B.ob, d->B.phi0};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  std::memset(&d->B, 0, sizeof(d->B));
}

}  // namespace

namespace pflb {

void set_global_error(const std::string& msg) { g_create_err = msg; }

const char* status_message(int status) {
  switch (status) {
    case PFLB_ERR_UNSTABLE: return "instability (NaN or non-positive temperature sum)";
    case PFLB_ERR_TIMEOUT: return "a bounded device wait ran out";
    case PFLB_ERR_UNSUPPORTED: return "a kernel's self-check failed (shared-memory alignment)";
    default: return "device status set";
  }
}

int validate_desc(const pflb_domain_desc& D, std::string& msg) {
  auto bad = [&](int code, const char* why) { msg = why; return code; };
  if (D.dim != 2 && D.dim != 3) return bad(PFLB_ERR_UNSUPPORTED, "dim must be 2 or 3");
  if (D.nx < 2 || D.ny < 1 || (D.dim == 3 && D.nz < 1)) return bad(PFLB_ERR_ARG, "bad lattice extent");
  const long long N = (long long)D.nx * D.ny * (D.dim == 3 ? D.nz : 1);
  if (N > (1LL << 31) / 32) return bad(PFLB_ERR_ARG, "lattice too large for int indexing");
  if (D.precision < PFLB_FP64 || D.precision > PFLB_FP32_FP16STORE)
    return bad(PFLB_ERR_ARG, "bad precision");
  for (int a = 0; a < D.dim; ++a) {
    const int lo = D.bc[2 * a], hi = D.bc[2 * a + 1];
    if (lo < 0 || lo > 3 || hi < 0 || hi > 3) return bad(PFLB_ERR_ARG, "bad bc kind");
    if ((lo == PFLB_BC_PERIODIC) != (hi == PFLB_BC_PERIODIC))
      return bad(PFLB_ERR_ARG, "periodic faces must come in pairs");
    if ((lo == PFLB_BC_INLET && a != 0) || (hi == PFLB_BC_OUTLET && a != 0) ||
        lo == PFLB_BC_OUTLET || hi == PFLB_BC_INLET)
      return bad(PFLB_ERR_ARG, "inlet only at x-lo, outlet only at x-hi");
  }
  const double pos[] = {D.dx, D.dt, D.rho_ref, D.Pr, D.eta, D.P0, D.mu_ref};
  for (double v : pos)
    if (!(v > 0 && std::isfinite(v)))
      return bad(PFLB_ERR_ARG, "dx, dt, rho_ref, Pr, eta, P0, mu_ref must be positive and finite");
  if (D.sutherland && !(D.suth_T > 0 && D.suth_S >= 0))
    return bad(PFLB_ERR_ARG, "Sutherland constants must be positive");
  if (!(D.T_in > 0) || !(D.Ts_uniform > 0)) return bad(PFLB_ERR_ARG, "T_in, Ts_uniform must be > 0");
  if (!(D.M0 > 0 && D.cp0 > 0)) return bad(PFLB_ERR_ARG, "M0, cp0 must be > 0");
  if (D.p0_mode != PFLB_P0_FIXED && D.p0_mode != PFLB_P0_CLOSED) return bad(PFLB_ERR_ARG, "bad p0_mode");
  if (D.Ts_field && !(D.rhocp_s > 0)) return bad(PFLB_ERR_ARG, "rhocp_s must be > 0");
  if (!(D.A_u >= 0 && D.A_T >= 0 && D.lambda_s >= 0 && D.phi_min >= 0 && D.T_max >= 0))
    return bad(PFLB_ERR_ARG, "A_u, A_T, lambda_s, phi_min, T_max must be >= 0");
  if (D.inlet_parabolic < 0 || D.inlet_parabolic > 2) return bad(PFLB_ERR_ARG, "bad inlet profile");
  if (D.outlet_nscbc != 0 && D.outlet_nscbc != 1) return bad(PFLB_ERR_ARG, "bad outlet_nscbc");
  if (D.outlet_nscbc && D.bc[1] != PFLB_BC_OUTLET)
    return bad(PFLB_ERR_ARG, "the characteristic outlet needs an outlet face");
  if (D.outlet_nscbc && !(D.nscbc_sigma > 0 && std::isfinite(D.nscbc_sigma)))
    return bad(PFLB_ERR_ARG, "nscbc_sigma must be positive");
  for (int a = 0; a < 3; ++a)
    if (!(std::fabs(D.u_s[a]) < 0.3)) return bad(PFLB_ERR_ARG, "|u_s| must be below 0.3");
  return PFLB_OK;
}

int validate_mech(const pflb_mechanism& m, std::string& msg) {
  auto bad = [&](int code, const char* why) { msg = why; return code; };
  if (m.K != 0 && m.K != 5 && m.K != 6) return bad(PFLB_ERR_UNSUPPORTED, "species count must be 0, 5 or 6");
  if (m.J < 0 || m.J > PFLB_JMAX) return bad(PFLB_ERR_ARG, "bad reaction count");
  if (m.chem_mode != PFLB_CHEM_NONE && m.chem_mode != PFLB_CHEM_EXPLICIT &&
      m.chem_mode != PFLB_CHEM_IMPLICIT && m.chem_mode != PFLB_CHEM_SURROGATE)
    return bad(PFLB_ERR_UNSUPPORTED, "chem_mode");
  if (m.chem_mode == PFLB_CHEM_SURROGATE && m.K != 6)
    return bad(PFLB_ERR_UNSUPPORTED, "the surrogate needs the six-species mechanism");
  for (int j = 0; j < m.J; ++j)
    if (m.rev[j] && !(m.p_ref > 0)) return bad(PFLB_ERR_ARG, "p_ref must be > 0");
  for (int k = 0; k < m.K; ++k)
    if (!(m.M[k] > 0 && m.cp[k] > 0 && m.Dref[k] >= 0))
      return bad(PFLB_ERR_ARG, "species data must be positive");
  if (m.K > 0 && m.D_exp != 0.0 && !(m.D_Tref > 0)) return bad(PFLB_ERR_ARG, "D_Tref must be > 0");
  if (m.transport != PFLB_TRANSPORT_SINGLE && m.transport != PFLB_TRANSPORT_MIXTURE)
    return bad(PFLB_ERR_ARG, "bad transport mode");
  if (m.transport == PFLB_TRANSPORT_MIXTURE)
    for (int k = 0; k < m.K; ++k)
      if (!(m.mu_k[k] > 0 && m.suth_Tk[k] > 0 && m.suth_Sk[k] >= 0))
        return bad(PFLB_ERR_ARG, "species viscosity laws must be positive");
  if (m.inlet_feedback < 0 || m.inlet_feedback > m.K)
    return bad(PFLB_ERR_ARG, "inlet_feedback must be 0 (off) or a species index + 1");
  if (m.inlet_feedback > 0 && !(m.Y_in[m.inlet_feedback - 1] > 0))
    return bad(PFLB_ERR_ARG, "the inlet feedback species must have Y_in > 0");
  return PFLB_OK;
}

// Mixture-averaged viscosity and conductivity (SI) of composition Y at T, the
// rules of the device's transport() in double precision.
static void mixture_mu_lam(const pflb_mechanism& m, double T, const double* Y, double& mu,
                           double& lam) {
  double invMw = 0, X[PFLB_KMAX], mk[PFLB_KMAX], lk[PFLB_KMAX];
  for (int k = 0; k < m.K; ++k) invMw += Y[k] / m.M[k];
  for (int k = 0; k < m.K; ++k) {
    X[k] = Y[k] / m.M[k] / invMw;
    mk[k] = m.mu_k[k] * std::pow(T / m.suth_Tk[k], 1.5) * (m.suth_Tk[k] + m.suth_Sk[k]) /
            (T + m.suth_Sk[k]);
    const double RM = 8.314 / m.M[k];
    lk[k] = mk[k] * (1.32 * (m.cp[k] - RM) + 1.77 * RM);
  }
  double s = 0, l1 = 0, l2 = 0;
  for (int k = 0; k < m.K; ++k) {
    double den = 0;
    for (int j = 0; j < m.K; ++j) {
      const double q = 1.0 + std::sqrt(mk[k] / mk[j]) * std::pow(m.M[j] / m.M[k], 0.25);
      den += q * q / (std::sqrt(8.0) * std::sqrt(1.0 + m.M[k] / m.M[j])) * X[j];
    }
    s += mk[k] * X[k] / den;
    l1 += X[k] * lk[k];
    l2 += X[k] / lk[k];
  }
  mu = s;
  lam = 0.5 * (l1 + 1.0 / l2);
}

int check_stability(const pflb_domain_desc& D, const pflb_mechanism* m, std::string& msg) {
  const bool mix = m && m->K > 0;
  double invMw = 1.0 / D.M0;
  if (mix) {
    invMw = 0.0;
    for (int k = 0; k < m->K; ++k) invMw += m->Y_in[k] / m->M[k];
    if (!(invMw > 0)) { msg = "inlet composition has no mass"; return PFLB_ERR_ARG; }
  }
  const double h2 = D.dt / (D.dx * D.dx);
  const double lim = 1.0 / (2.0 * D.dim);
  double temps[9];
  int nt = 0;
  temps[nt++] = D.T_in;
  temps[nt++] = D.Ts_uniform;
  if (D.T_max > 0) temps[nt++] = D.T_max;
  for (int f = 0; f < 2 * D.dim; ++f)
    if (D.bc[f] == PFLB_BC_WALL && D.wall_T[f] > 0) temps[nt++] = D.wall_T[f];
  char buf[256];
  for (int i = 0; i < nt; ++i) {
    const double T = temps[i];
    double mu = D.mu_ref;
    if (D.sutherland) mu *= std::pow(T / D.suth_T, 1.5) * (D.suth_T + D.suth_S) / (T + D.suth_S);
    const double rho_lat = D.P0 / (8.314 * T * invMw * D.rho_ref);
    double a;        // lambda / (rho cp), lattice units
    double lam_lat;  // lambda dt / (rho_ref dx^2) (J/kg/K)
    if (mix && m->transport == PFLB_TRANSPORT_MIXTURE) {
      double lam, cp = 0;
      mixture_mu_lam(*m, T, m->Y_in, mu, lam);
      for (int k = 0; k < m->K; ++k) cp += m->Y_in[k] * m->cp[k];
      a = lam * h2 / D.rho_ref / (rho_lat * cp);
      lam_lat = lam * h2 / D.rho_ref;
    } else {
      double cp = D.cp0;
      if (mix) {
        cp = 0;
        for (int k = 0; k < m->K; ++k) cp += m->Y_in[k] * m->cp[k];
      }
      a = mu * h2 / D.rho_ref / (rho_lat * D.Pr);
      lam_lat = mu * h2 / D.rho_ref * cp / D.Pr;
    }
    // the solid side of the exchange: phi_f S_I / (phi_s (rho cp)_s) relaxes Ts
    // at a rate A_T lambda phi_f^2 phi_s / (eta^2 (rho cp)_s), largest at
    // phi_s = 1/3 (4/27); forward Euler needs it below 2
    if (D.Ts_field && D.A_T > 0) {
      const double rs = D.A_T * lam_lat * (4.0 / 27.0) / (D.eta * D.eta * (D.rhocp_s / D.rho_ref));
      if (!(rs < 2.0)) {
        std::snprintf(buf, sizeof(buf),
                      "solid-side exchange number %.4g not below 2 at T = %g K (raise rhocp_s)",
                      rs, T);
        msg = buf;
        return PFLB_ERR_UNSTABLE;
      }
    }
    const double mu_lat = mu * h2 / D.rho_ref;
    const double tau = 0.5 + 3.0 * mu_lat / rho_lat;  // tau = 1/2 + nu / cs^2
    if (!(tau > 0.5) || !std::isfinite(tau)) {
      std::snprintf(buf, sizeof(buf), "relaxation time tau = %.6g <= 1/2 at T = %g K", tau, T);
      msg = buf;
      return PFLB_ERR_UNSTABLE;
    }
    if (!(a <= lim)) {
      std::snprintf(buf, sizeof(buf),
                    "thermal diffusion number %.4g above %.4g at T = %g K (reduce dt)", a, lim, T);
      msg = buf;
      return PFLB_ERR_UNSTABLE;
    }
    // forward-Euler relaxation toward Ts: stable while the rate per step,
    // at most A_T a / eta^2 (phi_s = 1), stays below 2
    if (!(D.A_T * a / (D.eta * D.eta) < 2.0)) {
      std::snprintf(buf, sizeof(buf), "interface exchange number A_T a / eta^2 = %.4g not below 2 at T = %g K",
                    D.A_T * a / (D.eta * D.eta), T);
      msg = buf;
      return PFLB_ERR_UNSTABLE;
    }
    if (mix) {
      for (int k = 0; k < m->K; ++k) {
        double Dk = m->Dref[k] * h2;
        if (m->D_exp != 0.0) Dk *= std::pow(T / m->D_Tref, m->D_exp);
        if (!(Dk <= lim)) {
          std::snprintf(buf, sizeof(buf),
                        "species %d diffusion number %.4g above %.4g at T = %g K (reduce dt)", k,
                        Dk, lim, T);
          msg = buf;
          return PFLB_ERR_UNSTABLE;
        }
      }
    }
  }
  if (D.Ts_field) {
    const double as = D.lambda_s * D.dt / (D.rhocp_s * D.dx * D.dx);
    if (!(as <= lim)) {
      std::snprintf(buf, sizeof(buf), "solid diffusion number %.4g above %.4g", as, lim);
      msg = buf;
      return PFLB_ERR_UNSTABLE;
    }
  }
  if (!(std::fabs(D.u_in) < std::sqrt(1.0 / 3.0))) {
    msg = "inlet speed at or above the lattice sound speed";
    return PFLB_ERR_UNSTABLE;
  }
  return PFLB_OK;
}

}  // namespace pflb

extern "C" {

int pflb_lattice(int dim, int* c_out, double* w_out) {
  if (dim == 2) {
    for (int i = 0; i < 9; ++i) {
      for (int a = 0; a < 3; ++a) c_out[3 * i + a] = Lattice<2>::c(i, a);
      w_out[i] = Lattice<2>::w(i);
    }
    return 9;
  }
  if (dim == 3) {
    for (int i = 0; i < 19; ++i) {
      for (int a = 0; a < 3; ++a) c_out[3 * i + a] = Lattice<3>::c(i, a);
      w_out[i] = Lattice<3>::w(i);
    }
    return 19;
  }
  return PFLB_ERR_ARG;
}

const char* pflb_last_error(const pflb_domain* d) {
  return d ? d->err.c_str() : g_create_err.c_str();
}

int pflb_validate(const pflb_domain_desc* desc, const pflb_mechanism* mech) {
  if (!desc) return fail(nullptr, PFLB_ERR_ARG, "desc is NULL");
  std::string why;
  int rc = validate_desc(*desc, why);
  if (rc == PFLB_OK && mech) rc = validate_mech(*mech, why);
  if (rc == PFLB_OK) rc = check_stability(*desc, mech, why);
  if (rc != PFLB_OK) return fail(nullptr, rc, "%s", why.c_str());
  g_create_err.clear();
  return PFLB_OK;
}

int pflb_create_domain(const pflb_domain_desc* desc, pflb_domain** out) {
  if (!out) return fail(nullptr, PFLB_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!desc) return fail(nullptr, PFLB_ERR_ARG, "desc is NULL");
  const pflb_domain_desc& D = *desc;
  std::string why;
  int rc = validate_desc(D, why);
  if (rc == PFLB_OK) rc = check_stability(D, nullptr, why);
  if (rc != PFLB_OK) return fail(nullptr, rc, "%s", why.c_str());
  const long long N = (long long)D.nx * D.ny * (D.dim == 3 ? D.nz : 1);

  pflb_domain* d = new (std::nothrow) pflb_domain();
  if (!d) return fail(nullptr, PFLB_ERR_OOM, "host allocation failed");
  d->desc = D;
  if (d->desc.dim == 2) d->desc.nz = 1;
  std::memset(&d->mech, 0, sizeof(d->mech));
  std::memset(&d->B, 0, sizeof(d->B));
  d->dim = D.dim;
  d->Q = D.dim == 2 ? 9 : 19;
  d->N = (int)N;
  d->B.N = (int)N;
  d->mode = D.precision == PFLB_FP64 ? MODE_FP64 : (D.precision == PFLB_FP32 ? MODE_FP32 : MODE_FP16);
  d->real_sz = d->mode == MODE_FP64 ? 8 : 4;
  d->store_sz = d->mode == MODE_FP64 ? 8 : (d->mode == MODE_FP32 ? 4 : 2);
  d->stream = static_cast<cudaStream_t>(D.stream);
  cudaError_t e = cudaSetDevice(D.device);
  if (e != cudaSuccess) {
    delete d;
    return fail(nullptr, PFLB_ERR_CUDA, "%s", cudaGetErrorString(e));
  }
  const size_t n = (size_t)N;
  // partial sums: one slot per block of the 1-D init grid or of any tile grid
  // (the step's 32 x 8 tiles and the batch's tile shapes)
  long long tiles = 0;
  for (int cfg = 0; cfg < BATCH_SHAPES; ++cfg)
    tiles = std::max<long long>(tiles, (long long)((D.nx + batch_tx(cfg) - 1) / batch_tx(cfg)) *
                                           ((D.ny + batch_ty(cfg) - 1) / batch_ty(cfg)) *
                                           (D.dim == 3 ? (D.nz + 15) / 16 : 1));
  const long long blocks = std::max<long long>((N + BLOCK - 1) / BLOCK, tiles);
  bool ok = true;
  auto al = [&](void** p, size_t bytes) {
    if (!ok) return;
    if (cudaMalloc(p, bytes) != cudaSuccess) { ok = false; *p = nullptr; }
    else cudaMemset(*p, 0, bytes);
  };
  for (int b = 0; b < 2; ++b) {
    al(&d->B.g[b], n * d->Q * d->store_sz);
    if (d->mode == MODE_FP16) al(&d->B.M[b], n * (D.dim + 1) * sizeof(float));
    al(&d->B.T[b], n * d->real_sz);
    if (D.Ts_field) al(&d->B.Ts[b], n * d->real_sz);
  }
  al(&d->B.phi, n * d->real_sz);
  al((void**)&d->B.scal, sizeof(DevScalars));
  d->B.slots = blocks;
  al((void**)&d->B.partials, (size_t)blocks * 2 * 4 * sizeof(double));
  al((void**)&d->B.counter, sizeof(unsigned));
  al((void**)&d->B.tile_ctr, 2 * sizeof(unsigned));
  al((void**)&d->B.feed_part, kFeedBlocks * sizeof(double));
  if (D.outlet_nscbc) al(&d->B.ob, (size_t)5 * D.ny * (D.dim == 3 ? D.nz : 1) * d->real_sz);
  if (D.u_s[0] != 0.0 || D.u_s[1] != 0.0 || (D.dim == 3 && D.u_s[2] != 0.0))
    al(&d->B.phi0, n * d->real_sz);
  if (!ok) {
    cudaGetLastError();
    free_buffers(d);
    delete d;
    return fail(nullptr, PFLB_ERR_OOM, "device allocation failed");
  }
  *out = d;
  return PFLB_OK;
}

int pflb_set_mechanism(pflb_domain* d, const pflb_mechanism* m) {
  if (!d || !m) return fail(d, PFLB_ERR_ARG, "NULL argument");
  {
    std::string why;
    int rc = validate_mech(*m, why);
    if (rc == PFLB_OK) rc = check_stability(d->desc, m, why);
    if (rc != PFLB_OK) return fail(d, rc, "%s", why.c_str());
    if (m->inlet_feedback > 0 &&
        (d->desc.bc[0] != PFLB_BC_INLET || d->desc.p0_mode != PFLB_P0_FIXED))
      return fail(d, PFLB_ERR_ARG, "the inlet feedback needs an inlet face and a fixed P0");
    if (m->inlet_feedback > 0 && d->desc.inlet_parabolic == 2)
      return fail(d, PFLB_ERR_UNSUPPORTED,
                  "the inlet feedback needs an inlet profile of fixed shape (0 or 1)");
  }
  if (d->has_fields) return fail(d, PFLB_ERR_STATE, "set_mechanism must precede set_fields");
  cudaSetDevice(d->desc.device);
  const size_t n = (size_t)d->N;
  for (int b = 0; b < 2; ++b) {
    if (d->B.Y[b]) { cudaFree(d->B.Y[b]); d->B.Y[b] = nullptr; }
    if (m->K > 0 && cudaMalloc(&d->B.Y[b], n * m->K * d->real_sz) != cudaSuccess)
      return fail(d, PFLB_ERR_OOM, "device allocation failed");
  }
  void* old_bufs[] = {d->B.src, d->B.fb_idx, d->B.fb_count, d->B.chem_stats};
  for (void* q : old_bufs)
    if (q) cudaFree(q);
  d->B.src = nullptr;
  d->B.fb_idx = nullptr;
  d->B.fb_count = nullptr;
  d->B.chem_stats = nullptr;
  if (m->K > 0 && m->chem_mode >= PFLB_CHEM_IMPLICIT &&
      cudaMalloc(&d->B.src, n * (m->K + 1) * d->real_sz) != cudaSuccess)
    return fail(d, PFLB_ERR_OOM, "device allocation failed");
  if (m->chem_mode == PFLB_CHEM_SURROGATE) {
    if (cudaMalloc((void**)&d->B.fb_idx, n * sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&d->B.fb_count, sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc((void**)&d->B.chem_stats, 2 * sizeof(double)) != cudaSuccess)
      return fail(d, PFLB_ERR_OOM, "device allocation failed");
    cudaMemset(d->B.fb_count, 0, sizeof(unsigned));
    cudaMemset(d->B.chem_stats, 0, 2 * sizeof(double));
  }
  d->mech = *m;
  d->K = m->K;
  d->has_mech = true;
  return PFLB_OK;
}

int pflb_set_phase_field(pflb_domain* d, const void* phi, const void* Ts, int dtype, int where) {
  if (!d || !phi) return fail(d, PFLB_ERR_ARG, "NULL argument");
  int r = check_dtype_where(d, dtype, where);
  if (r) return r;
  CK(d, cudaSetDevice(d->desc.device));
  if ((r = upload(d, phi, dtype, where, d->B.phi, d->N))) return r;
  if (d->B.phi0)  // a moving solid: this is the phase field of step 0
    CK(d, cudaMemcpyAsync(d->B.phi0, d->B.phi, (size_t)d->N * d->real_sz,
                          cudaMemcpyDeviceToDevice, d->stream));
  if (d->desc.Ts_field) {
    if (Ts) {
      if ((r = upload(d, Ts, dtype, where, d->B.Ts[d->cur], d->N))) return r;
    } else {
      const int blocks = (d->N + 255) / 256 > 4096 ? 4096 : (d->N + 255) / 256;
      if (d->real_sz == 8)
        fill_kernel<double><<<blocks, 256, 0, d->stream>>>((double*)d->B.Ts[d->cur],
                                                           d->desc.Ts_uniform, d->N);
      else
        fill_kernel<float><<<blocks, 256, 0, d->stream>>>((float*)d->B.Ts[d->cur],
                                                          (float)d->desc.Ts_uniform, d->N);
      CK(d, cudaGetLastError());
    }
  }
  d->has_phase = true;
  return PFLB_OK;
}

int pflb_set_fields(pflb_domain* d, unsigned mask, const void* src, int dtype, int where) {
  if (!d || !src) return fail(d, PFLB_ERR_ARG, "NULL argument");
  int r = check_dtype_where(d, dtype, where);
  if (r) return r;
  if (!d->has_phase) return fail(d, PFLB_ERR_STATE, "set_phase_field must come first");
  if (!(mask & PFLB_FIELD_T)) return fail(d, PFLB_ERR_ARG, "T is required");
  if (d->K > 0 && !(mask & PFLB_FIELD_Y)) return fail(d, PFLB_ERR_ARG, "Y is required when K > 0");
  if (mask & ~(PFLB_FIELD_T | PFLB_FIELD_Y | PFLB_FIELD_U))
    return fail(d, PFLB_ERR_ARG, "set_fields accepts T, Y, U only");
  CK(d, cudaSetDevice(d->desc.device));
  const size_t esz = dtype == PFLB_DTYPE_F64 ? 8 : 4;
  const char* p = static_cast<const char*>(src);
  const size_t n = (size_t)d->N;
  if ((r = upload(d, p, dtype, where, d->B.T[d->cur], n))) return r;
  p += n * esz;
  if (d->K > 0) {
    if ((r = upload(d, p, dtype, where, d->B.Y[d->cur], n * d->K))) return r;
    p += n * d->K * esz;
  }
  void* u = nullptr;
  if (mask & PFLB_FIELD_U) {
    CK(d, cudaMallocAsync(&u, n * d->dim * d->real_sz, d->stream));
    if ((r = upload(d, p, dtype, where, u, n * d->dim))) { cudaFreeAsync(u, d->stream); return r; }
  }
  delete d->L;
  d->L = make_launcher(d);
  if (!d->L) return fail(d, PFLB_ERR_UNSUPPORTED, "no kernel compiled for this combination");
  d->L->set_wait_limit(d->wait_limit);
  d->B.pending = 0;
  cudaError_t e = d->L->init(d->B, d->cur, u, d->desc.P0, d->stream);
  if (e == cudaSuccess) e = d->L->set_step(d->B, 0, d->stream);
  if (u) cudaFreeAsync(u, d->stream);
  CK(d, e);
  d->has_fields = true;
  return PFLB_OK;
}

int pflb_step(pflb_domain* d, int nsteps) {
  if (!d) return fail(d, PFLB_ERR_ARG, "NULL domain");
  if (!d->has_fields || !d->L) return fail(d, PFLB_ERR_STATE, "set_fields must come first");
  if (nsteps < 0) return fail(d, PFLB_ERR_ARG, "nsteps < 0");
  CK(d, cudaSetDevice(d->desc.device));
  CK(d, d->L->step(d->B, d->cur, nsteps, d->stream));
  return PFLB_OK;
}

int pflb_get_scalars(pflb_domain* d, pflb_scalars* out) {
  if (!d || !out) return fail(d, PFLB_ERR_ARG, "NULL argument");
  CK(d, cudaSetDevice(d->desc.device));
  if (d->L) CK(d, d->L->finalize(d->B, d->stream));
  DevScalars h;
  CK(d, cudaMemcpyAsync(&h, d->B.scal, sizeof(h), cudaMemcpyDeviceToHost, d->stream));
  CK(d, cudaStreamSynchronize(d->stream));
  out->P0 = h.P0;
  out->P0_prev = h.P0_prev;
  out->mass = h.mass;
  out->I = h.I;
  out->flux_in = h.flux_in;
  out->flux_out = h.flux_out;
  out->step = h.step;
  out->status = h.status;
  out->u_in = h.u_in;
  out->fuel = h.fuel;
  out->outlet_pb = h.pb;
  if (h.status != 0) return fail(d, h.status, "%s", status_message(h.status));
  return PFLB_OK;
}

int pflb_get_diagnostics(pflb_domain* d, pflb_diagnostics* out) {
  if (!d || !out) return fail(d, PFLB_ERR_ARG, "NULL argument");
  if (!d->has_fields || !d->L) return fail(d, PFLB_ERR_STATE, "no fields yet");
  CK(d, cudaSetDevice(d->desc.device));
  CK(d, d->L->finalize(d->B, d->stream));
  double* buf = nullptr;
  const int nb = d->L->diag_blocks();
  CK(d, cudaMallocAsync((void**)&buf, ((size_t)nb + 1) * NDIAG * sizeof(double), d->stream));
  cudaError_t e = d->L->diagnostics(d->B, d->cur, buf + NDIAG, buf, d->stream);
  double h[NDIAG];
  DevScalars s;
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, buf, sizeof(h), cudaMemcpyDeviceToHost, d->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&s, d->B.scal, sizeof(s), cudaMemcpyDeviceToHost, d->stream);
  cudaFreeAsync(buf, d->stream);
  CK(d, e);
  CK(d, cudaStreamSynchronize(d->stream));
  for (int a = 0; a < 3; ++a) out->drag[a] = h[a];
  out->heat = h[3];
  out->mass = h[4];
  out->outlet_Tm = h[6] != 0.0 ? h[5] / h[6] : 0.0;
  out->flux_in_total = s.flux_in_sum;
  out->flux_out_total = s.flux_out_sum;
  out->step = s.step;
  if (s.status != 0) return fail(d, s.status, "%s", status_message(s.status));
  return PFLB_OK;
}

int pflb_get_fields(pflb_domain* d, unsigned mask, void* dst, size_t bytes, int dtype, int where) {
  if (!d || !dst) return fail(d, PFLB_ERR_ARG, "NULL argument");
  int r = check_dtype_where(d, dtype, where);
  if (r) return r;
  if (!d->has_fields) return fail(d, PFLB_ERR_STATE, "no fields yet");
  if ((mask & PFLB_FIELD_TS) && !d->desc.Ts_field)
    return fail(d, PFLB_ERR_ARG, "no solid temperature field");
  if ((mask & PFLB_FIELD_Y) && d->K == 0) return fail(d, PFLB_ERR_ARG, "no species");
  const size_t n = (size_t)d->N, esz = dtype == PFLB_DTYPE_F64 ? 8 : 4;
  size_t need = 0;
  if (mask & PFLB_FIELD_T) need += n;
  if (mask & PFLB_FIELD_Y) need += n * d->K;
  if (mask & PFLB_FIELD_TS) need += n;
  if (mask & PFLB_FIELD_U) need += n * d->dim;
  if (mask & PFLB_FIELD_RHO) need += n;
  if (mask & PFLB_FIELD_PH) need += n;
  if (mask & PFLB_FIELD_G) need += n * d->Q;
  if (bytes < need * esz) return fail(d, PFLB_ERR_ARG, "destination too small");
  CK(d, cudaSetDevice(d->desc.device));
  CK(d, d->L->finalize(d->B, d->stream));
  char* out = nullptr;
  if (where == PFLB_HOST) CK(d, cudaMallocAsync((void**)&out, need * esz, d->stream));
  else out = static_cast<char*>(dst);
  char* p = out;
  auto put_real = [&](const void* srcp, size_t cnt) -> cudaError_t {
    cudaError_t e;
    if (d->real_sz == 8) e = esz == 8 ? convert<double, double>(srcp, p, cnt, d->stream)
                                      : convert<double, float>(srcp, p, cnt, d->stream);
    else e = esz == 8 ? convert<float, double>(srcp, p, cnt, d->stream)
                      : convert<float, float>(srcp, p, cnt, d->stream);
    p += cnt * esz;
    return e;
  };
  cudaError_t e = cudaSuccess;
  if (mask & PFLB_FIELD_T) e = put_real(d->B.T[d->cur], n);
  if (e == cudaSuccess && (mask & PFLB_FIELD_Y)) e = put_real(d->B.Y[d->cur], n * d->K);
  if (e == cudaSuccess && (mask & PFLB_FIELD_TS)) e = put_real(d->B.Ts[d->cur], n);
  if (e == cudaSuccess && (mask & (PFLB_FIELD_U | PFLB_FIELD_RHO | PFLB_FIELD_PH))) {
    double* mom = nullptr;
    e = cudaMallocAsync((void**)&mom, n * (d->dim + 2) * sizeof(double), d->stream);
    if (e == cudaSuccess) e = d->L->moments(d->B, d->cur, mom, mom + n * d->dim,
                                            mom + n * (d->dim + 1), d->stream);
    auto put_d = [&](const double* srcp, size_t cnt) {
      cudaError_t ee = esz == 8 ? convert<double, double>(srcp, p, cnt, d->stream)
                                : convert<double, float>(srcp, p, cnt, d->stream);
      p += cnt * esz;
      return ee;
    };
    if (e == cudaSuccess && (mask & PFLB_FIELD_U)) e = put_d(mom, n * d->dim);
    if (e == cudaSuccess && (mask & PFLB_FIELD_RHO)) e = put_d(mom + n * d->dim, n);
    if (e == cudaSuccess && (mask & PFLB_FIELD_PH)) e = put_d(mom + n * (d->dim + 1), n);
    if (mom) cudaFreeAsync(mom, d->stream);
  }
  if (e == cudaSuccess && (mask & PFLB_FIELD_G)) {
    Weights W;
    W.Q = d->Q;
    W.dim = d->dim;
    const float s = d->L->g_scale();
    for (int i = 0; i < d->Q; ++i) {
      double w = d->dim == 2 ? Lattice<2>::w(i) : Lattice<3>::w(i);
      W.w_over_scale[i] = float(w / s);
      W.w[i] = float(w);
      for (int a = 0; a < 3; ++a) W.c[i][a] = d->dim == 2 ? Lattice<2>::c(i, a) : Lattice<3>::c(i, a);
    }
    const float* Mc = static_cast<const float*>(d->B.M[d->cur]);
    const size_t cnt = n * d->Q;
    int blocks = (int)((cnt + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    const void* g = d->B.g[d->cur];
    if (d->mode == MODE_FP64) {
      if (esz == 8) decode_g_kernel<double, double><<<blocks, 256, 0, d->stream>>>((const double*)g, Mc, (double*)p, n, W);
      else decode_g_kernel<double, float><<<blocks, 256, 0, d->stream>>>((const double*)g, Mc, (float*)p, n, W);
    } else if (d->mode == MODE_FP32) {
      if (esz == 8) decode_g_kernel<float, double><<<blocks, 256, 0, d->stream>>>((const float*)g, Mc, (double*)p, n, W);
      else decode_g_kernel<float, float><<<blocks, 256, 0, d->stream>>>((const float*)g, Mc, (float*)p, n, W);
    } else {
      if (esz == 8) decode_g_kernel<__half, double><<<blocks, 256, 0, d->stream>>>((const __half*)g, Mc, (double*)p, n, W);
      else decode_g_kernel<__half, float><<<blocks, 256, 0, d->stream>>>((const __half*)g, Mc, (float*)p, n, W);
    }
    e = cudaGetLastError();
    p += cnt * esz;
  }
  if (e == cudaSuccess && where == PFLB_HOST)
    e = cudaMemcpyAsync(dst, out, need * esz, cudaMemcpyDeviceToHost, d->stream);
  if (where == PFLB_HOST && out) cudaFreeAsync(out, d->stream);
  CK(d, e);
  CK(d, cudaStreamSynchronize(d->stream));
  DevScalars h;
  CK(d, cudaMemcpy(&h, d->B.scal, sizeof(h), cudaMemcpyDeviceToHost));
  if (h.status != 0) return fail(d, h.status, "%s", status_message(h.status));
  return PFLB_OK;
}

}  // extern "C"

namespace {
struct StateHeader {
  char magic[8];
  int version, dim, nx, ny, nz, precision, K, Ts_field;
  long long N;
  int reserved[4];
};

size_t mom_bytes(const pflb_domain* d) {
  return d->mode == MODE_FP16 ? (size_t)d->N * (d->dim + 1) * sizeof(float) : 0;
}

size_t state_bytes(const pflb_domain* d) {
  const size_t n = (size_t)d->N;
  size_t b = sizeof(StateHeader) + sizeof(DevScalars);
  b += n * d->Q * d->store_sz + mom_bytes(d) + n * d->real_sz + n * d->K * d->real_sz;
  if (d->desc.Ts_field) b += n * d->real_sz;
  return b;
}

// (pointer into the serialised buffer, device array, bytes) for each array
template <class F>
int for_each_array(pflb_domain* d, F f) {
  const size_t n = (size_t)d->N;
  size_t off = sizeof(StateHeader) + sizeof(DevScalars);
  struct A { void* p; size_t b; } arr[5] = {
      {d->B.g[d->cur], n * d->Q * d->store_sz}, {d->B.M[d->cur], mom_bytes(d)},
      {d->B.T[d->cur], n * d->real_sz},
      {d->B.Y[d->cur], n * d->K * d->real_sz},
      {d->desc.Ts_field ? d->B.Ts[d->cur] : nullptr, d->desc.Ts_field ? n * d->real_sz : 0}};
  for (auto& a : arr) {
    if (!a.b) continue;
    int r = f(off, a.p, a.b);
    if (r) return r;
    off += a.b;
  }
  return PFLB_OK;
}
}  // namespace

extern "C" {

int pflb_state_bytes(const pflb_domain* d, size_t* bytes) {
  if (!d || !bytes) return PFLB_ERR_ARG;
  *bytes = state_bytes(d);
  return PFLB_OK;
}

int pflb_get_state(pflb_domain* d, void* dst, size_t bytes, int where) {
  if (!d || !dst) return fail(d, PFLB_ERR_ARG, "NULL argument");
  if (!d->has_fields) return fail(d, PFLB_ERR_STATE, "no state yet");
  if (bytes < state_bytes(d)) return fail(d, PFLB_ERR_ARG, "destination too small");
  if (where != PFLB_HOST && where != PFLB_DEVICE) return fail(d, PFLB_ERR_ARG, "bad where");
  CK(d, cudaSetDevice(d->desc.device));
  CK(d, d->L->finalize(d->B, d->stream));
  StateHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "PFLBSTv3", 8);
  h.version = 1;
  h.dim = d->dim; h.nx = d->desc.nx; h.ny = d->desc.ny; h.nz = d->desc.nz;
  h.precision = d->desc.precision; h.K = d->K; h.Ts_field = d->desc.Ts_field; h.N = d->N;
  char* out = static_cast<char*>(dst);
  const cudaMemcpyKind k = where == PFLB_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  const cudaMemcpyKind kh = where == PFLB_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice;
  CK(d, cudaMemcpyAsync(out, &h, sizeof(h), kh, d->stream));
  CK(d, cudaMemcpyAsync(out + sizeof(h), d->B.scal, sizeof(DevScalars), k, d->stream));
  int r = for_each_array(d, [&](size_t off, void* p, size_t b) {
    CK(d, cudaMemcpyAsync(out + off, p, b, k, d->stream));
    return PFLB_OK;
  });
  if (r) return r;
  CK(d, cudaStreamSynchronize(d->stream));
  return PFLB_OK;
}

int pflb_set_state(pflb_domain* d, const void* src, size_t bytes, int where) {
  if (!d || !src) return fail(d, PFLB_ERR_ARG, "NULL argument");
  if (!d->has_fields) return fail(d, PFLB_ERR_STATE, "set_fields must run once first");
  if (bytes < state_bytes(d)) return fail(d, PFLB_ERR_ARG, "source too small");
  if (where != PFLB_HOST && where != PFLB_DEVICE) return fail(d, PFLB_ERR_ARG, "bad where");
  CK(d, cudaSetDevice(d->desc.device));
  StateHeader h;
  if (where == PFLB_HOST) std::memcpy(&h, src, sizeof(h));
  else CK(d, cudaMemcpy(&h, src, sizeof(h), cudaMemcpyDeviceToHost));
  if (std::memcmp(h.magic, "PFLBSTv3", 8) != 0 || h.dim != d->dim || h.nx != d->desc.nx ||
      h.ny != d->desc.ny || h.nz != d->desc.nz || h.precision != d->desc.precision ||
      h.K != d->K || h.Ts_field != d->desc.Ts_field || h.N != d->N)
    return fail(d, PFLB_ERR_ARG, "state does not match this domain");
  const char* in = static_cast<const char*>(src);
  const cudaMemcpyKind k = where == PFLB_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(d, cudaMemcpyAsync(d->B.scal, in + sizeof(h), sizeof(DevScalars), k, d->stream));
  d->B.pending = 0;
  int rc = for_each_array(d, [&](size_t off, void* p, size_t b) {
    CK(d, cudaMemcpyAsync(p, in + off, b, k, d->stream));
    return PFLB_OK;
  });
  if (rc != PFLB_OK) return rc;
  // the step count of the restored state (a moving solid's phase field)
  DevScalars sc;
  if (where == PFLB_HOST) std::memcpy(&sc, in + sizeof(h), sizeof(sc));
  else CK(d, cudaMemcpy(&sc, in + sizeof(h), sizeof(sc), cudaMemcpyDeviceToHost));
  if (d->L) CK(d, d->L->set_step(d->B, sc.step, d->stream));
  return PFLB_OK;
}

int pflb_set_wait_limit(pflb_domain* d, long long cycles) {
  if (!d) return fail(d, PFLB_ERR_ARG, "NULL domain");
  if (cycles < 0 || cycles > (1LL << 40)) return fail(d, PFLB_ERR_ARG, "cycles out of range");
  d->wait_limit = cycles;
  if (d->L) d->L->set_wait_limit(cycles);
  return PFLB_OK;
}

int pflb_select_kernel(pflb_domain* d, int kernel) {
  if (!d) return fail(d, PFLB_ERR_ARG, "NULL domain");
  if (!d->L) return fail(d, PFLB_ERR_STATE, "set_fields must come first");
  CK(d, cudaSetDevice(d->desc.device));
  if (!d->L->select_kernel(kernel, d->B, d->cur))
    return fail(d, PFLB_ERR_UNSUPPORTED, "kernel not available for this domain");
  return PFLB_OK;
}

int pflb_autotune(pflb_domain* d, int steps, int* chosen, double* us_per_step) {
  if (!d || !chosen) return fail(d, PFLB_ERR_ARG, "NULL argument");
  if (!d->L) return fail(d, PFLB_ERR_STATE, "set_fields must come first");
  if (steps < 1) return fail(d, PFLB_ERR_ARG, "steps < 1");
  CK(d, cudaSetDevice(d->desc.device));
  // snapshot the state on the device, time each candidate, restore
  size_t nb = state_bytes(d);
  void* snap = nullptr;
  CK(d, cudaMallocAsync(&snap, nb, d->stream));
  int r = pflb_get_state(d, snap, nb, PFLB_DEVICE);
  if (r) { cudaFreeAsync(snap, d->stream); return r; }
  const int prev = d->L->kernel();
  int best = prev;
  double best_us = -1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int k = 0; k < PFLB_KERNELS; ++k) {
    double us = -1;
    if (d->L->select_kernel(k, d->B, d->cur)) {
      cudaError_t e = d->L->step(d->B, d->cur, 1, d->stream);  // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, d->stream);
      if (e == cudaSuccess) e = d->L->step(d->B, d->cur, steps, d->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, d->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0;
      if (e == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
        us = 1e3 * ms / steps;
      if ((r = pflb_set_state(d, snap, nb, PFLB_DEVICE))) break;
      if (us > 0 && (best_us < 0 || us < best_us)) { best_us = us; best = k; }
    }
    if (us_per_step) us_per_step[k] = us;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(snap, d->stream);
  if (r) return r;
  d->L->select_kernel(best >= 0 ? best : prev, d->B, d->cur);
  *chosen = d->L->kernel();
  CK(d, cudaStreamSynchronize(d->stream));
  return PFLB_OK;
}

}  // extern "C"

namespace pflb {
mlp::Net mlp_net(const pflb_mlp* m);
}

extern "C" {

int pflb_set_surrogate(pflb_domain* d, const pflb_mlp* net, const pflb_surrogate* s) {
  if (!d || !net || !s) return fail(d, PFLB_ERR_ARG, "NULL argument");
  if (!d->L) return fail(d, PFLB_ERR_STATE, "set_fields must come first");
  if (d->mech.chem_mode != PFLB_CHEM_SURROGATE || d->K != 6)
    return fail(d, PFLB_ERR_STATE, "mechanism is not in surrogate mode");
  if (s->n_elem < 0 || s->n_elem > 4) return fail(d, PFLB_ERR_ARG, "n_elem");
  if (s->engine != PFLB_MLP_TCGEN05 && s->engine != PFLB_MLP_WARP_MMA)
    return fail(d, PFLB_ERR_ARG, "engine");
  SurrArgs a;
  std::memset(&a, 0, sizeof(a));
  a.net = mlp_net(net);
  for (int f = 0; f < 8; ++f) {
    a.x_mean[f] = float(s->x_mean[f]);
    a.x_istd[f] = s->x_std[f] > 0 ? float(1.0 / s->x_std[f]) : 0.f;
    a.lo[f] = float(s->lo[f]);
    a.hi[f] = float(s->hi[f]);
  }
  for (int k = 0; k < 6; ++k) {
    a.y_mean[k] = float(s->y_mean[k]);
    a.y_std[k] = float(s->y_std[k]);
  }
  a.n_elem = s->n_elem;
  a.engine = s->engine;
  a.tol = s->tol;
  a.theta_s = s->theta_s;
  a.tol_f = float(s->tol);
  a.theta_f = float(s->theta_s);
  // residual weights a_ek M_e / M_k and the orthogonal projection onto
  // {dY : sum_k a_ek dY_k / M_k = 0 for every element}
  double B[4][6] = {};
  for (int e = 0; e < s->n_elem; ++e)
    for (int k = 0; k < 6; ++k) {
      a.E[e][k] = s->elem[e][k] * s->elem_mass[e] / d->mech.M[k];
      a.E_f[e][k] = float(a.E[e][k]);
      B[e][k] = s->elem[e][k] / d->mech.M[k];
    }
  const int ne = s->n_elem;
  double G[4][4] = {}, Gi[4][4] = {};
  for (int i = 0; i < ne; ++i)
    for (int j = 0; j < ne; ++j) {
      for (int k = 0; k < 6; ++k) G[i][j] += B[i][k] * B[j][k];
      Gi[i][j] = i == j ? 1.0 : 0.0;
    }
  for (int c = 0; c < ne; ++c) {  // Gauss-Jordan inverse of the element Gram matrix
    int piv = c;
    for (int r = c + 1; r < ne; ++r)
      if (std::fabs(G[r][c]) > std::fabs(G[piv][c])) piv = r;
    if (G[piv][c] == 0.0) return fail(d, PFLB_ERR_ARG, "element matrix is rank deficient");
    for (int k = 0; k < ne; ++k) {
      std::swap(G[c][k], G[piv][k]);
      std::swap(Gi[c][k], Gi[piv][k]);
    }
    const double inv = 1.0 / G[c][c];
    for (int k = 0; k < ne; ++k) { G[c][k] *= inv; Gi[c][k] *= inv; }
    for (int r = 0; r < ne; ++r) {
      if (r == c) continue;
      const double f = G[r][c];
      for (int k = 0; k < ne; ++k) { G[r][k] -= f * G[c][k]; Gi[r][k] -= f * Gi[c][k]; }
    }
  }
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double v = i == j ? 1.0 : 0.0;
      for (int p = 0; p < ne; ++p)
        for (int q = 0; q < ne; ++q) v -= B[p][i] * Gi[p][q] * B[q][j];
      a.Pj[i][j] = v;
      a.Pj_f[i][j] = float(v);
    }
  // cold tiles may skip the network: with |tanh| <= 1 the output layer bounds
  // |out_k| by sum_j |W_3[j][k]| + |b_3[k]| (the factor 1 + 2^-7 covers the
  // BF16 rounding of the weights and of the activations), the projection by
  // its infinity norm, and exp(-theta_s / T) does the rest
  if (!(s->skip_eps >= 0.0)) return fail(d, PFLB_ERR_ARG, "skip_eps");
  a.T_skip = 0.0;
  if (s->skip_eps > 0.0) {
    if (!(s->theta_s > 0.0)) return fail(d, PFLB_ERR_ARG, "skip_eps needs theta_s > 0");
    std::vector<float> th(mlp::NPARAM);
    const int r = pflb_mlp_get_params(const_cast<pflb_mlp*>(net), th.data());
    CK(d, cudaSetDevice(d->desc.device));
    if (r) return fail(d, r, "reading the network parameters");
    const float* W3 = th.data() + mlp::woff(3);
    const float* b3 = th.data() + mlp::boff(3);
    double bound = 0.0, pinf = 0.0;
    for (int k = 0; k < 6; ++k) {
      double o = std::fabs(b3[k]);
      for (int j = 0; j < 64; ++j) o += 1.0078125 * std::fabs(W3[j * 6 + k]);
      bound = std::max(bound, std::fabs(s->y_mean[k]) + std::fabs(s->y_std[k]) * o);
      double row = 0.0;
      for (int q = 0; q < 6; ++q) row += std::fabs(a.Pj[k][q]);
      pinf = std::max(pinf, row);
    }
    bound *= pinf;
    a.T_skip = bound > s->skip_eps ? s->theta_s / std::log(bound / s->skip_eps)
                                   : std::numeric_limits<double>::infinity();
  }
  a.T_skip_f = float(a.T_skip);
  if (!d->L->set_surrogate(a)) return fail(d, PFLB_ERR_UNSUPPORTED, "surrogate not available");
  return PFLB_OK;
}

int pflb_chem_increments(pflb_domain* d, void* dst, size_t bytes, int dtype, int where) {
  if (!d || !dst) return fail(d, PFLB_ERR_ARG, "NULL argument");
  int r = check_dtype_where(d, dtype, where);
  if (r) return r;
  if (!d->L || d->K == 0 || d->mech.chem_mode < PFLB_CHEM_IMPLICIT)
    return fail(d, PFLB_ERR_STATE, "needs implicit or surrogate chemistry");
  const size_t n = (size_t)d->N * (d->K + 1), esz = dtype == PFLB_DTYPE_F64 ? 8 : 4;
  if (bytes < n * esz) return fail(d, PFLB_ERR_ARG, "destination too small");
  CK(d, cudaSetDevice(d->desc.device));
  double* tmp = nullptr;
  CK(d, cudaMallocAsync((void**)&tmp, n * sizeof(double), d->stream));
  cudaError_t e = d->L->chem_pass(d->B, d->cur, tmp, d->stream);
  void* out = dst;
  void* stage = nullptr;
  if (e == cudaSuccess && where == PFLB_HOST) {
    e = cudaMallocAsync(&stage, n * esz, d->stream);
    out = stage;
  }
  if (e == cudaSuccess)
    e = esz == 8 ? convert<double, double>(tmp, out, n, d->stream)
                 : convert<double, float>(tmp, out, n, d->stream);
  if (e == cudaSuccess && where == PFLB_HOST)
    e = cudaMemcpyAsync(dst, stage, n * esz, cudaMemcpyDeviceToHost, d->stream);
  if (stage) cudaFreeAsync(stage, d->stream);
  cudaFreeAsync(tmp, d->stream);
  CK(d, e);
  CK(d, cudaStreamSynchronize(d->stream));
  return PFLB_OK;
}

int pflb_chem_stats(pflb_domain* d, double* fallback_cells, double* evaluated_cells) {
  if (!d) return fail(d, PFLB_ERR_ARG, "NULL domain");
  double h[2] = {0, 0};
  if (d->B.chem_stats) {
    CK(d, cudaSetDevice(d->desc.device));
    CK(d, cudaMemcpyAsync(h, d->B.chem_stats, sizeof(h), cudaMemcpyDeviceToHost, d->stream));
    CK(d, cudaStreamSynchronize(d->stream));
  }
  if (fallback_cells) *fallback_cells = h[0];
  if (evaluated_cells) *evaluated_cells = h[1];
  return PFLB_OK;
}

int pflb_destroy(pflb_domain* d) {
  if (!d) return PFLB_OK;
  cudaSetDevice(d->desc.device);
  cudaStreamSynchronize(d->stream);
  free_buffers(d);
  for (int b = 0; b < 2; ++b)
    if (d->B.Y[b]) cudaFree(d->B.Y[b]);
  delete d->L;
  delete d;
  return PFLB_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches
struct pflb_batch {
  std::vector<pflb_domain*> doms;
  std::vector<int> cur_expected;  // each domain's input buffer at the next batch step
  Launcher* L0 = nullptr;
  int device = 0;
  cudaStream_t stream = nullptr;  // the batch's own (blocking) stream
  cudaEvent_t ev = nullptr;
  size_t entry_bytes = 0;
  void* entries = nullptr;        // device work list [n][entry_bytes]
  unsigned* tile_ctr = nullptr;   // tile counters, one per launch parity
  std::vector<unsigned char> host_entries;
  int* tile_begin[BATCH_SHAPES] = {};  // device prefix sums per tile shape
  int occ[BATCH_SHAPES] = {};
  int sms = 0;
  int cfg = 0, bps = 0, grid = 0;
  int flip = 0;                   // parity of the next batch step
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // two steps, starting at flip 0 / 1
  std::string err;
};

namespace {

int bfail(pflb_batch* b, int code, const char* msg) {
  if (b) b->err = msg;
  else g_create_err = msg;
  return code;
}

void drop_graphs(pflb_batch* b) {
  for (auto& g : b->graph)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
}

int batch_grid(const pflb_batch* b, int cfg, int bps) {
  const int occ = b->occ[cfg];
  const int per = bps > 0 ? std::min(bps, occ) : occ;
  return std::max(1, per * b->sms);
}

// Rebuild the work list when a domain was stepped on its own since the last
// batch step (its input buffer moved); order the batch after the domains'
// queued work and fold their deferred reductions.
int batch_prepare(pflb_batch* b) {
  bool stale = false;
  for (size_t i = 0; i < b->doms.size(); ++i) {
    pflb_domain* d = b->doms[i];
    if (d->L->finalize(d->B, d->stream) != cudaSuccess)
      return bfail(b, PFLB_ERR_CUDA, "finalize of a member domain failed");
    if ((d->cur ^ b->flip) != b->cur_expected[i]) stale = true;
  }
  if (stale) {
    for (size_t i = 0; i < b->doms.size(); ++i) {
      pflb_domain* d = b->doms[i];
      b->doms[i]->L->batch_entry(b->host_entries.data() + i * b->entry_bytes, d->B,
                                 d->cur ^ b->flip);
      b->cur_expected[i] = d->cur ^ b->flip;
    }
  }
  cudaStream_t last = reinterpret_cast<cudaStream_t>(-1);
  for (pflb_domain* d : b->doms) {
    if (d->stream == last) continue;
    last = d->stream;
    if (cudaEventRecord(b->ev, d->stream) != cudaSuccess ||
        cudaStreamWaitEvent(b->stream, b->ev, 0) != cudaSuccess)
      return bfail(b, PFLB_ERR_CUDA, "stream ordering failed");
  }
  if (stale &&
      cudaMemcpyAsync(b->entries, b->host_entries.data(), b->host_entries.size(),
                      cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
    return bfail(b, PFLB_ERR_CUDA, "work list upload failed");
  if (stale && cudaStreamSynchronize(b->stream) != cudaSuccess)  // host staging reused
    return bfail(b, PFLB_ERR_CUDA, "work list upload failed");
  return PFLB_OK;
}

int batch_finish(pflb_batch* b, int nsteps) {
  if (cudaEventRecord(b->ev, b->stream) != cudaSuccess)
    return bfail(b, PFLB_ERR_CUDA, "stream ordering failed");
  cudaStream_t last = reinterpret_cast<cudaStream_t>(-1);
  for (pflb_domain* d : b->doms) {
    if ((nsteps & 1) != 0) d->cur ^= 1;
    d->B.pending = 0;
    if (d->stream == last) continue;
    last = d->stream;
    if (cudaStreamWaitEvent(d->stream, b->ev, 0) != cudaSuccess)
      return bfail(b, PFLB_ERR_CUDA, "stream ordering failed");
  }
  return PFLB_OK;
}

cudaError_t batch_launch_one(pflb_batch* b, int flip) {
  return b->L0->batch_launch(b->entries, b->tile_begin[b->cfg], (int)b->doms.size(), b->cfg,
                             b->grid, flip, b->tile_ctr, b->stream);
}

cudaError_t batch_capture(pflb_batch* b, int start) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t e1 = batch_launch_one(b, start);
  cudaError_t e2 = batch_launch_one(b, start ^ 1);
  e = cudaStreamEndCapture(b->stream, &g);
  if (e == cudaSuccess && e1 == cudaSuccess && e2 == cudaSuccess)
    e = cudaGraphInstantiate(&b->graph[start], g, 0);
  if (g) cudaGraphDestroy(g);
  if (e == cudaSuccess && e1 != cudaSuccess) e = e1;
  if (e == cudaSuccess && e2 != cudaSuccess) e = e2;
  return e;
}

// nsteps batch steps on the batch stream: graph replays of two steps, one
// plain launch for an odd remainder.
int batch_run(pflb_batch* b, int nsteps) {
  int n = nsteps;
  while (n >= 2) {
    if (!b->graph[b->flip]) {
      cudaError_t e = batch_capture(b, b->flip);
      if (e != cudaSuccess) return bfail(b, PFLB_ERR_CUDA, cudaGetErrorString(e));
    }
    if (cudaGraphLaunch(b->graph[b->flip], b->stream) != cudaSuccess)
      return bfail(b, PFLB_ERR_CUDA, "graph launch failed");
    n -= 2;
  }
  if (n == 1) {
    cudaError_t e = batch_launch_one(b, b->flip);
    if (e != cudaSuccess) return bfail(b, PFLB_ERR_CUDA, cudaGetErrorString(e));
    b->flip ^= 1;
  }
  return PFLB_OK;
}

}  // namespace

extern "C" {

int pflb_create_batch(pflb_domain** domains, int n, pflb_batch** out) {
  if (!domains || !out || n < 1) return bfail(nullptr, PFLB_ERR_ARG, "NULL argument or n < 1");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    pflb_domain* d = domains[i];
    if (!d) return bfail(nullptr, PFLB_ERR_ARG, "NULL domain");
    if (!d->L || !d->has_fields) return bfail(nullptr, PFLB_ERR_STATE, "set_fields must come first");
    if (d->L->batch_entry_bytes() == 0)
      return bfail(nullptr, PFLB_ERR_UNSUPPORTED, "only 2-D domains without species batch");
    if (d->desc.outlet_nscbc)
      return bfail(nullptr, PFLB_ERR_UNSUPPORTED, "the characteristic outlet steps alone");
    if (d->B.phi0)
      return bfail(nullptr, PFLB_ERR_UNSUPPORTED, "a moving solid steps alone");
    if (d->L->batch_key() != domains[0]->L->batch_key())
      return bfail(nullptr, PFLB_ERR_UNSUPPORTED, "domains of a batch share one precision");
    if (d->desc.device != domains[0]->desc.device)
      return bfail(nullptr, PFLB_ERR_UNSUPPORTED, "domains of a batch share one device");
    for (int j = 0; j < i; ++j)
      if (domains[j] == d) return bfail(nullptr, PFLB_ERR_ARG, "a domain appears twice");
  }
  pflb_batch* b = new (std::nothrow) pflb_batch();
  if (!b) return bfail(nullptr, PFLB_ERR_OOM, "host allocation failed");
  b->doms.assign(domains, domains + n);
  b->L0 = domains[0]->L;
  b->device = domains[0]->desc.device;
  b->entry_bytes = b->L0->batch_entry_bytes();
  b->host_entries.resize(b->entry_bytes * n);
  b->cur_expected.assign(n, -1);
  auto bad = [&](int code, const char* msg) {
    pflb_batch_destroy(b);
    return bfail(nullptr, code, msg);
  };
  if (cudaSetDevice(b->device) != cudaSuccess) return bad(PFLB_ERR_CUDA, "cudaSetDevice failed");
  if (cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess)
    return bad(PFLB_ERR_CUDA, "device query failed");
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess)
    return bad(PFLB_ERR_CUDA, "stream creation failed");
  if (cudaMalloc(&b->entries, b->host_entries.size()) != cudaSuccess ||
      cudaMalloc((void**)&b->tile_ctr, 2 * sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(b->tile_ctr, 0, 2 * sizeof(unsigned)) != cudaSuccess)
    return bad(PFLB_ERR_OOM, "device allocation failed");
  for (int cfg = 0; cfg < BATCH_SHAPES; ++cfg) {
    std::vector<int> tb(n + 1, 0);
    for (int i = 0; i < n; ++i) {
      const pflb_domain_desc& D = domains[i]->desc;
      const long long t = (long long)((D.nx + batch_tx(cfg) - 1) / batch_tx(cfg)) *
                          ((D.ny + batch_ty(cfg) - 1) / batch_ty(cfg));
      if (t > domains[i]->B.slots) return bad(PFLB_ERR_STATE, "reduction slots too few");
      if ((long long)tb[i] + t > (1LL << 30)) return bad(PFLB_ERR_ARG, "batch too large");
      tb[i + 1] = tb[i] + (int)t;
    }
    if (cudaMalloc((void**)&b->tile_begin[cfg], (n + 1) * sizeof(int)) != cudaSuccess)
      return bad(PFLB_ERR_OOM, "device allocation failed");
    if (cudaMemcpy(b->tile_begin[cfg], tb.data(), (n + 1) * sizeof(int),
                   cudaMemcpyHostToDevice) != cudaSuccess)
      return bad(PFLB_ERR_CUDA, "upload failed");
    b->occ[cfg] = b->L0->batch_occupancy(cfg);
    if (b->occ[cfg] < 1) return bad(PFLB_ERR_CUDA, "batch kernel has no occupancy");
  }
  b->cfg = 0;
  b->bps = 0;
  b->grid = batch_grid(b, 0, 0);
  *out = b;
  return PFLB_OK;
}

int pflb_batch_step(pflb_batch* b, int nsteps) {
  if (!b) return bfail(b, PFLB_ERR_ARG, "NULL batch");
  if (nsteps < 0) return bfail(b, PFLB_ERR_ARG, "nsteps < 0");
  if (nsteps == 0) return PFLB_OK;
  if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, PFLB_ERR_CUDA, "cudaSetDevice");
  int r = batch_prepare(b);
  if (r) return r;
  if ((r = batch_run(b, nsteps))) return r;
  return batch_finish(b, nsteps);
}

int pflb_batch_set_config(pflb_batch* b, int tile, int blocks_per_sm) {
  if (!b) return bfail(b, PFLB_ERR_ARG, "NULL batch");
  if (tile < 0 || tile >= BATCH_SHAPES || blocks_per_sm < 0)
    return bfail(b, PFLB_ERR_ARG, "bad tile shape or blocks per SM");
  if (blocks_per_sm > b->occ[tile]) return bfail(b, PFLB_ERR_ARG, "blocks per SM above occupancy");
  if (cudaStreamSynchronize(b->stream) != cudaSuccess)
    return bfail(b, PFLB_ERR_CUDA, "synchronise failed");
  drop_graphs(b);
  b->cfg = tile;
  b->bps = blocks_per_sm;
  b->grid = batch_grid(b, tile, blocks_per_sm);
  return PFLB_OK;
}

int pflb_batch_get_config(const pflb_batch* b, int* tile, int* blocks_per_sm, int* grid) {
  if (!b) return PFLB_ERR_ARG;
  if (tile) *tile = b->cfg;
  if (blocks_per_sm) *blocks_per_sm = b->bps > 0 ? std::min(b->bps, b->occ[b->cfg]) : b->occ[b->cfg];
  if (grid) *grid = b->grid;
  return PFLB_OK;
}

int pflb_batch_autotune(pflb_batch* b, int steps, int* tile, int* blocks_per_sm,
                        double* us_per_step) {
  if (!b || !tile || !blocks_per_sm) return bfail(b, PFLB_ERR_ARG, "NULL argument");
  if (steps < 1) return bfail(b, PFLB_ERR_ARG, "steps < 1");
  if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, PFLB_ERR_CUDA, "cudaSetDevice");
  const size_t n = b->doms.size();
  std::vector<void*> snap(n, nullptr);
  std::vector<size_t> nbytes(n, 0);
  int r = PFLB_OK;
  for (size_t i = 0; i < n && !r; ++i) {
    nbytes[i] = state_bytes(b->doms[i]);
    if (cudaMalloc(&snap[i], nbytes[i]) != cudaSuccess) r = bfail(b, PFLB_ERR_OOM, "snapshot");
    else r = pflb_get_state(b->doms[i], snap[i], nbytes[i], PFLB_DEVICE);
  }
  if (us_per_step)
    for (int k = 0; k < BATCH_SHAPES * 8; ++k) us_per_step[k] = 0;
  const int cfg0 = b->cfg, bps0 = b->bps;
  int best_cfg = cfg0, best_bps = bps0;
  double best = -1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int cfg = 0; cfg < BATCH_SHAPES && !r; ++cfg) {
    for (int bps = 1; bps <= std::min(b->occ[cfg], 8) && !r; ++bps) {
      if ((r = pflb_batch_set_config(b, cfg, bps))) break;
      if ((r = pflb_batch_step(b, 2))) break;  // warm-up and graph capture
      if ((r = batch_prepare(b))) break;
      cudaEventRecord(e0, b->stream);
      if ((r = batch_run(b, 2 * steps))) break;
      cudaEventRecord(e1, b->stream);
      if ((r = batch_finish(b, 2 * steps))) break;
      float ms = 0;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        r = bfail(b, PFLB_ERR_CUDA, "timing failed");
        break;
      }
      const double us = 1e3 * ms / (2 * steps);
      if (us_per_step) us_per_step[cfg * 8 + bps - 1] = us;
      if (best < 0 || us < best) { best = us; best_cfg = cfg; best_bps = bps; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (size_t i = 0; i < n; ++i) {
    if (snap[i]) {
      int r2 = pflb_set_state(b->doms[i], snap[i], nbytes[i], PFLB_DEVICE);
      if (!r && r2) r = bfail(b, r2, "restoring a domain failed");
      cudaStreamSynchronize(b->doms[i]->stream);
      cudaFree(snap[i]);
    }
  }
  if (r) {
    pflb_batch_set_config(b, cfg0, bps0);
    return r;
  }
  if ((r = pflb_batch_set_config(b, best_cfg, best_bps))) return r;
  *tile = b->cfg;
  pflb_batch_get_config(b, nullptr, blocks_per_sm, nullptr);
  return PFLB_OK;
}

int pflb_batch_destroy(pflb_batch* b) {
  if (!b) return PFLB_OK;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  for (int* p : b->tile_begin)
    if (p) cudaFree(p);
  if (b->entries) cudaFree(b->entries);
  if (b->tile_ctr) cudaFree(b->tile_ctr);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return PFLB_OK;
}

const char* pflb_batch_last_error(const pflb_batch* b) {
  return b ? b->err.c_str() : g_create_err.c_str();
}

}  // extern "C"
