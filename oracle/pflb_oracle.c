/*
 * pflb_oracle.c -- plain, slow FP64 CPU oracle for one time step of the
 * low-Mach phase-field / lattice-Boltzmann / finite-difference (PF-LB-FD)
 * scheme of Namdar, Norouzi & Varnik (arXiv 2310.17214).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library: the lattice tables, the unit conversions
 * and every formula below are written out here independently.
 *
 * What it computes (paper references are to sections / equations):
 *   - EOS rho = Mw P0 / (R T)                     (Sec. 3.1, eq. rho-in-terms-of-P0-and-T)
 *   - P0 = m R / int(Mw/T dV) over the fluid      (Sec. 3.1, text after the EOS)
 *   - drag F = -A_u mu phi_f phi_s^2/eta^2 u      (Sec. 3.2.1, eq. Fdrag-empirical-law; u_s = 0)
 *   - species transport + omega_k = M_k sum s Q   (Sec. 3.2.2, eqs. volume-averaged-species-equation-5, 8)
 *   - temperature equation with S_I and omega_T   (Sec. 3.3, eqs. diffusion-heat-flux-3,
 *                                                   energy-transport-DI-version, 9)
 *   - pressure-based LB with source Xi, f_eq, g_eq (Sec. 3.3, eqs. pop-g, body-force,
 *                                                   eq-pop-f, eq-pop-g; mu = rho cs^2 (tau-1/2))
 *   - upwind convection, central diffusion, forward Euler (Sec. 3.3, last paragraph)
 *   - Sutherland viscosity and lambda = mu cp / Pr (Sec. 4, eqs. muT, lambdaT)
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   BGK with second-order (half-step) source; P_h = sum g + rho cs^2 D / 2 and
 *   rho u = sum c g / cs^2 + F / 2 with the drag implicit in u; D = div u from
 *   the low-Mach constraint using this step's increments; conservative
 *   phi_f-weighted FD with arithmetic-mean face coefficients; S_I relaxes the
 *   fluid toward the solid temperature; lagged dP0/dt; half-way bounce-back
 *   walls, moving-wall bounce-back inlet, anti-bounce-back P_h = 0 outlet.
 *
 * Layout: cell = x + nx*(y + ny*z); populations g[i*N + cell]; species
 * Y[k*N + cell]; velocity u[a*N + cell].
 *
 * Host threads: within each phase of a step the per-cell updates are
 * independent (every cell reads the previous phase's arrays and writes only
 * its own entries), so those loops carry an OpenMP "parallel for".  No sum is
 * split across threads: the global reductions (I, the boundary fluxes) stay
 * serial in cell order, and the results do not depend on the thread count.
 *
 * Parity pins: tests/test_oracle_pins.py (closed forms, invariants, brute force).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_KMAX 8
#define ORC_JMAX 4
#define ORC_QMAX 19
#define ORC_R 8.314 /* J/(mol K), value printed in Sec. 3.1 */

enum { ORC_BC_PERIODIC = 0, ORC_BC_WALL = 1, ORC_BC_INLET = 2, ORC_BC_OUTLET = 3 };
enum { ORC_P0_FIXED = 0, ORC_P0_CLOSED = 1 };
enum { ORC_CHEM_NONE = 0, ORC_CHEM_EXPLICIT = 1, ORC_CHEM_IMPLICIT = 2 };

typedef struct {
  int dim, nx, ny, nz;
  int bc[6];               /* x-lo, x-hi, y-lo, y-hi, z-lo, z-hi */
  double wall_u[6][3];     /* tangential velocity of each wall face (lattice) */
  double wall_T[6];        /* wall temperature (K) of each wall face, 0 = adiabatic */
  double dx, dt, rho_ref;  /* physical scales (1,1,1 = pure lattice units) */
  /* fluid properties */
  int K;                   /* number of species, 0 = non-reactive single gas */
  double M0, cp0;          /* molar mass / heat capacity when K == 0 */
  double M[ORC_KMAX], cp[ORC_KMAX], hf[ORC_KMAX], Dref[ORC_KMAX];
  double D_Tref, D_exp;    /* D_k = Dref_k (T / D_Tref)^D_exp */
  double mu_ref;           /* dynamic viscosity (physical units) */
  int sutherland;          /* 1: mu(T) Sutherland law */
  double suth_T, suth_S, Pr;
  double A_u, A_T, eta;    /* coupling parameters, interface width (cells) */
  double Fb[3];            /* body force density (lattice) */
  /* inlet */
  int inlet_parabolic;
  double u_in, T_in, Y_in[ORC_KMAX];
  /* thermodynamic pressure */
  int p0_mode;
  /* solid */
  int Ts_field;            /* 0: uniform fixed Ts_uniform, 1: transported field */
  double Ts_uniform, rhocp_s, lambda_s;
  double phi_min;
  /* chemistry */
  int chem_mode, J;
  double A[ORC_JMAX], b[ORC_JMAX], EaR[ORC_JMAX];
  double order[ORC_JMAX][ORC_KMAX], stoich[ORC_JMAX][ORC_KMAX];
  /* reversible reactions: K_c from standard dH, dS (ideal gas, p_ref) */
  int rev[ORC_JMAX];
  double dH[ORC_JMAX], dS[ORC_JMAX], rorder[ORC_JMAX][ORC_KMAX];
  double p_ref;
  /* mixture-averaged transport (Sec. 4.4, eqs. muT_mix, phi_mix, conduct_mix):
   * species viscosities from Sutherland laws mu_k(T) = mu_k (T / Tk)^1.5
   * (Tk + Sk) / (T + Sk), species conductivities from the modified Eucken
   * relation lambda_k = mu_k (1.32 cv_k + 1.77 R / M_k), cv_k = cp_k - R / M_k;
   * 0 = single gas (mu_ref, Pr) */
  int transport_mix;
  double mu_k[ORC_KMAX], suth_Tk[ORC_KMAX], suth_Sk[ORC_KMAX];
  /* inlet mass-flow feedback (Sec. 4.4.1): after each step the inlet speed is
   * set so that the fuel (species fb_k) entering through the inlet equals
   * the fuel the step consumed, u_in = sum phi_f (-omega_F) / (rho_in Y_F,in A),
   * A = sum over the inlet cells of the inlet profile; held in [0, 0.3] */
  int feedback, fb_k;
  /* Partially non-reflecting outlet (Sec. 4.1, the characteristic outlet of
   * Poinsot and Lele): instead of P_h = 0 the anti-bounce-back imposes a
   * boundary pressure P_b that follows the 1-D characteristic relation
   * dP_b/dt = -(L5 + L1)/2 of a plane wave leaving through the outlet, with
   * the outgoing wave L5 = (u + cs) (dP_h/dx + rho cs du/dx) from the face
   * means of the last step's P_h, u_x (one-sided differences over the two
   * outlet columns) and rho of the outlet column, and the incoming wave
   * L1 = K P_b (relaxation to the ambient P_h = 0).  ob (caller-owned, 6 NF
   * doubles, NF = ny nz): P_b, then P_h and u_x of column nx-1, P_h and u_x
   * of column nx-2 and rho of column nx-1, all of the last step. */
  int nscbc;
  double nscbc_K;
  double* ob;
  /* Moving solid (v_I != 0, Sec. 2: the indicator is carried by the
   * interface velocity, d chi/dt = d_t chi + v_I . grad chi = 0): the solid
   * translates rigidly with the uniform velocity u_s (lattice units).  The
   * phase field of step n is the given one (step 0) displaced by n u_s,
   * multilinear interpolation between cells (periodic axes wrap, others
   * clamp); the drag acts on u - u_s; the solid temperature is carried with
   * u_s (upwind, as the FD convection of T). */
  int moving;
  double u_s[3];
} orc_params;

/* ---------------------------------------------------------------- lattices */
static const int C2[9][3] = {{0,0,0},{1,0,0},{0,1,0},{-1,0,0},{0,-1,0},
                             {1,1,0},{-1,1,0},{-1,-1,0},{1,-1,0}};
static const double W2[9] = {4.0/9, 1.0/9, 1.0/9, 1.0/9, 1.0/9,
                             1.0/36, 1.0/36, 1.0/36, 1.0/36};
static const int C3[19][3] = {{0,0,0},
  {1,0,0},{-1,0,0},{0,1,0},{0,-1,0},{0,0,1},{0,0,-1},
  {1,1,0},{-1,-1,0},{1,-1,0},{-1,1,0},
  {1,0,1},{-1,0,-1},{1,0,-1},{-1,0,1},
  {0,1,1},{0,-1,-1},{0,1,-1},{0,-1,1}};
static const double W3[19] = {1.0/3,
  1.0/18,1.0/18,1.0/18,1.0/18,1.0/18,1.0/18,
  1.0/36,1.0/36,1.0/36,1.0/36,1.0/36,1.0/36,
  1.0/36,1.0/36,1.0/36,1.0/36,1.0/36,1.0/36};
static const double CS2 = 1.0 / 3.0;

typedef struct { int Q; const int (*c)[3]; const double* w; } lat_t;
static lat_t lattice_of(int dim) {
  lat_t L;
  if (dim == 2) { L.Q = 9; L.c = C2; L.w = W2; }
  else { L.Q = 19; L.c = C3; L.w = W3; }
  return L;
}
static int opposite(lat_t L, int i) {
  for (int j = 0; j < L.Q; ++j)
    if (L.c[j][0] == -L.c[i][0] && L.c[j][1] == -L.c[i][1] && L.c[j][2] == -L.c[i][2]) return j;
  return -1;
}

/* Exported so that tests can check both sides use the same direction order. */
int orc_lattice(int dim, int* c_out, double* w_out) {
  lat_t L = lattice_of(dim);
  for (int i = 0; i < L.Q; ++i) {
    for (int a = 0; a < 3; ++a) c_out[3 * i + a] = L.c[i][a];
    w_out[i] = L.w[i];
  }
  return L.Q;
}

/* ------------------------------------------------ equilibrium and source */
/* f_eq (Sec. 3.3, eq. eq-pop-f) and g_eq = cs^2 f_eq + w (P_h - rho cs^2)
 * (eq. eq-pop-g), written literally. */
void orc_equilibrium(int dim, double Ph, double rho, const double* u, double* geq) {
  lat_t L = lattice_of(dim);
  double uu = 0;
  for (int a = 0; a < dim; ++a) uu += u[a] * u[a];
  for (int i = 0; i < L.Q; ++i) {
    double cu = 0;
    for (int a = 0; a < dim; ++a) cu += L.c[i][a] * u[a];
    double feq = rho * L.w[i] * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    geq[i] = CS2 * feq + L.w[i] * (Ph - rho * CS2);
  }
}

/* Source Xi (Sec. 3.3, eq. body-force): G = grad(rho cs^2), F = total force
 * density (body force plus drag), D = div u. */
void orc_source(int dim, double rho, const double* G, const double* u, const double* F,
                double D, double* xi) {
  lat_t L = lattice_of(dim);
  double uu = 0;
  for (int a = 0; a < dim; ++a) uu += u[a] * u[a];
  for (int i = 0; i < L.Q; ++i) {
    double cu = 0;
    for (int a = 0; a < dim; ++a) cu += L.c[i][a] * u[a];
    double feq = rho * L.w[i] * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    double s = 0;
    for (int a = 0; a < dim; ++a)
      s += (L.c[i][a] - u[a]) * (G[a] * (feq / rho - L.w[i]) + F[a] * feq / rho);
    xi[i] = s + rho * CS2 * L.w[i] * D;
  }
}

/* ---------------------------------------------------------- thermo, props */
typedef struct { double T, Y[ORC_KMAX], phi, Ts; } cellv;
typedef struct { double Mw, rho, cp, mu, lam, D[ORC_KMAX]; } derv;

static double mixture_Mw(const orc_params* p, const double* Y) {
  if (p->K == 0) return p->M0;
  double s = 0;
  for (int k = 0; k < p->K; ++k) s += Y[k] / p->M[k];
  return 1.0 / s;
}
static double mixture_cp(const orc_params* p, const double* Y) {
  if (p->K == 0) return p->cp0;
  double s = 0;
  for (int k = 0; k < p->K; ++k) s += Y[k] * p->cp[k];
  return s;
}
/* lattice density rho / rho_ref from the EOS */
static double eos_rho(const orc_params* p, double P0, double Mw, double T) {
  return P0 * Mw / (ORC_R * T * p->rho_ref);
}
/* lattice dynamic viscosity: Sutherland (Sec. 4, eq. muT) or constant */
static double visc(const orc_params* p, double T) {
  double mu = p->mu_ref;
  if (p->sutherland)
    mu = p->mu_ref * pow(T / p->suth_T, 1.5) * (p->suth_T + p->suth_S) / (T + p->suth_S);
  return mu * p->dt / (p->rho_ref * p->dx * p->dx);
}

/* Mixture-averaged viscosity and conductivity (physical units) of a gas of
 * composition Y at T (Sec. 4.4): mole fractions X_k = Y_k Mw / M_k;
 * mu = sum_k mu_k X_k / sum_j Phi_kj X_j with
 * Phi_kj = (1 + sqrt(mu_k / mu_j sqrt(M_j / M_k)))^2 / (sqrt(8) sqrt(1 + M_k / M_j))
 * (eqs. muT_mix, phi_mix); lambda = (sum_k X_k lambda_k + 1 / sum_k X_k / lambda_k) / 2
 * (eq. conduct_mix). */
void orc_mixture_transport(const orc_params* p, double T, const double* Y, double* mu_out,
                           double* lam_out) {
  int K = p->K;
  double Mw = mixture_Mw(p, Y);
  double X[ORC_KMAX], mu[ORC_KMAX], lam[ORC_KMAX];
  for (int k = 0; k < K; ++k) {
    X[k] = Y[k] * Mw / p->M[k];
    mu[k] = p->mu_k[k] * pow(T / p->suth_Tk[k], 1.5) * (p->suth_Tk[k] + p->suth_Sk[k]) /
            (T + p->suth_Sk[k]);
    lam[k] = mu[k] * (1.32 * (p->cp[k] - ORC_R / p->M[k]) + 1.77 * ORC_R / p->M[k]);
  }
  double m = 0, l1 = 0, l2 = 0;
  for (int k = 0; k < K; ++k) {
    double den = 0;
    for (int j = 0; j < K; ++j) {
      double a = 1.0 + sqrt(mu[k] / mu[j] * sqrt(p->M[j] / p->M[k]));
      double phi = a * a / (sqrt(8.0) * sqrt(1.0 + p->M[k] / p->M[j]));
      den += phi * X[j];
    }
    m += mu[k] * X[k] / den;
    l1 += X[k] * lam[k];
    l2 += X[k] / lam[k];
  }
  *mu_out = m;
  *lam_out = 0.5 * (l1 + 1.0 / l2);
}

/* lattice viscosity of a gas of composition Y at T */
static double visc_of(const orc_params* p, double T, const double* Y) {
  if (!(p->transport_mix && p->K > 0)) return visc(p, T);
  double mu, lam;
  orc_mixture_transport(p, T, Y, &mu, &lam);
  return mu * p->dt / (p->rho_ref * p->dx * p->dx);
}

static void derive(const orc_params* p, const cellv* v, double P0, derv* d) {
  d->Mw = mixture_Mw(p, v->Y);
  d->rho = eos_rho(p, P0, d->Mw, v->T);
  d->cp = mixture_cp(p, v->Y);
  if (p->transport_mix && p->K > 0) {
    double mu, lam, s = p->dt / (p->rho_ref * p->dx * p->dx);
    orc_mixture_transport(p, v->T, v->Y, &mu, &lam);
    d->mu = mu * s;
    d->lam = lam * s;
  } else {
    d->mu = visc(p, v->T);
    d->lam = d->mu * d->cp / p->Pr; /* Sec. 4, eq. lambdaT (lattice units) */
  }
  for (int k = 0; k < p->K; ++k) {
    double D = p->Dref[k];
    if (p->D_exp != 0.0) D = p->Dref[k] * pow(v->T / p->D_Tref, p->D_exp);
    d->D[k] = D * p->dt / (p->dx * p->dx);
  }
}

/* Rate constants of reaction j at T: forward k_f = A T^b exp(-Ea/RT) and,
 * for a reversible reaction, k_r = k_f / K_c with
 * K_c = exp(dS/R - dH/(R T)) (p_ref/(R T))^(sum_k s_kj)  (mass action, ideal gas). */
static void rate_constants(const orc_params* p, int j, double T, double* kf, double* kr) {
  double k = p->A[j] * exp(-p->EaR[j] / T);
  if (p->b[j] != 0.0) k *= pow(T, p->b[j]);
  *kf = k;
  *kr = 0.0;
  if (p->rev[j]) {
    double dn = 0;
    for (int m = 0; m < p->K; ++m) dn += p->stoich[j][m];
    double Kc = exp(p->dS[j] / ORC_R - p->dH[j] / (ORC_R * T)) * pow(p->p_ref / (ORC_R * T), dn);
    *kr = k / Kc;
  }
}

/* Explicit rates: Q_j = A T^b exp(-Ea/RT) prod C_k^order, C_k = rho Y_k / M_k
 * (mol/m^3); omega_k = M_k sum_j s_kj Q_j (Sec. 3.2.2, eq. 8), omega_T =
 * -sum hf_k omega_k (Sec. 3.3, eq. 9).  Outputs are per lattice step per
 * rho_ref:  omega_k dt / rho_ref (1/step) and omega_T dt / rho_ref (J/kg). */
static double powi_or_pow(double x, double e) {
  if (e == 1.0) return x;
  if (e == 2.0) return x * x;
  if (e == 0.0) return 1.0;
  return pow(x, e);
}
void orc_chem_rates(const orc_params* p, double T, const double* Y, double rho_lat,
                    double* omega, double* omegaT) {
  double rho = rho_lat * p->rho_ref;
  double C[ORC_KMAX];
  for (int k = 0; k < p->K; ++k) C[k] = rho * (Y[k] > 0 ? Y[k] : 0.0) / p->M[k];
  for (int k = 0; k < p->K; ++k) omega[k] = 0;
  for (int j = 0; j < p->J; ++j) {
    double kf, kr;
    rate_constants(p, j, T, &kf, &kr);
    double q = kf;
    for (int k = 0; k < p->K; ++k)
      if (p->order[j][k] != 0.0) q *= powi_or_pow(C[k], p->order[j][k]);
    if (p->rev[j]) {
      double qr = kr;
      for (int k = 0; k < p->K; ++k)
        if (p->rorder[j][k] != 0.0) qr *= powi_or_pow(C[k], p->rorder[j][k]);
      q -= qr;
    }
    for (int k = 0; k < p->K; ++k) omega[k] += p->M[k] * p->stoich[j][k] * q;
  }
  double wt = 0;
  for (int k = 0; k < p->K; ++k) {
    omega[k] = omega[k] * p->dt / p->rho_ref;
    wt -= p->hf[k] * omega[k];
  }
  *omegaT = wt;
}

/* ------------------------------------------------- implicit chemistry
 * Backward Euler over one step for the chemistry alone at frozen density
 * (operator splitting): with z = (Y_1..Y_K, T),
 *   dY_k/dt = omega_k / rho,   dT/dt = omega_T / (rho cp(Y))   (Sec. 3.2.2 eq. 8,
 *   Sec. 3.3 eqs. energy-transport-DI-version and 9, chemistry terms only),
 * solve G(z) = z - z0 - dt F(z) = 0 by Newton with the analytic Jacobian and a
 * dense Gaussian elimination with partial pivoting.  If Newton does not
 * converge (or leaves the physical range) the step is split into 2, 4, ...,
 * 64 equal backward-Euler sub-steps. */
#define ORC_NMAX (ORC_KMAX + 1)

/* physical rates and their Jacobian: w[k] = omega_k (kg/m^3/s), dw[k][m] =
 * d omega_k / d z_m (z = Y..., T) at density rho (kg/m^3) */
static void rates_and_jacobian(const orc_params* p, const double* z, double rho, double* w,
                               double dw[ORC_KMAX][ORC_NMAX]) {
  int K = p->K;
  double T = z[K];
  double C[ORC_KMAX], dC[ORC_KMAX];
  for (int k = 0; k < K; ++k) {
    C[k] = z[k] > 0 ? rho * z[k] / p->M[k] : 0.0;
    dC[k] = z[k] > 0 ? rho / p->M[k] : 0.0;
    w[k] = 0;
    for (int m = 0; m <= K; ++m) dw[k][m] = 0;
  }
  for (int j = 0; j < p->J; ++j) {
    double kf, kr;
    rate_constants(p, j, T, &kf, &kr);
    /* d ln kf / dT and d ln kr / dT */
    double dlkf = p->EaR[j] / (T * T) + p->b[j] / T;
    double dlkr = dlkf;
    if (p->rev[j]) {
      double dn = 0;
      for (int m = 0; m < K; ++m) dn += p->stoich[j][m];
      dlkr = dlkf - (p->dH[j] / (ORC_R * T * T) + dn / T);
    }
    double dq[ORC_NMAX];
    for (int m = 0; m <= K; ++m) dq[m] = 0;
    for (int dir = 0; dir < (p->rev[j] ? 2 : 1); ++dir) {
      const double* ord = dir == 0 ? p->order[j] : p->rorder[j];
      double kk = dir == 0 ? kf : kr, sign = dir == 0 ? 1.0 : -1.0;
      double prod = 1.0;
      for (int k = 0; k < K; ++k)
        if (ord[k] != 0.0) prod *= powi_or_pow(C[k], ord[k]);
      double q = sign * kk * prod;
      for (int k = 0; k < K; ++k) w[k] += p->M[k] * p->stoich[j][k] * q;
      dq[K] += q * (dir == 0 ? dlkf : dlkr);
      for (int m = 0; m < K; ++m) {
        if (ord[m] == 0.0 || dC[m] == 0.0) continue;
        double rest = 1.0;
        for (int k = 0; k < K; ++k)
          if (k != m && ord[k] != 0.0) rest *= powi_or_pow(C[k], ord[k]);
        double dpow = ord[m] == 1.0 ? 1.0 : ord[m] * pow(C[m], ord[m] - 1.0);
        dq[m] += sign * kk * rest * dpow * dC[m];
      }
    }
    for (int k = 0; k < K; ++k)
      for (int m = 0; m <= K; ++m) dw[k][m] += p->M[k] * p->stoich[j][k] * dq[m];
  }
}

static int solve_dense(int n, double A[ORC_NMAX][ORC_NMAX], double* b) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
    if (A[piv][c] == 0.0) return -1;
    if (piv != c) {
      for (int k = 0; k < n; ++k) { double t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
      double t = b[c]; b[c] = b[piv]; b[piv] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      double f = A[r][c] / A[c][c];
      for (int k = c; k < n; ++k) A[r][k] -= f * A[c][k];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s2 = b[r];
    for (int k = r + 1; k < n; ++k) s2 -= A[r][k] * b[k];
    b[r] = s2 / A[r][r];
  }
  return 0;
}

/* one backward-Euler step of length h from z0; returns 0 on convergence */
static int be_newton(const orc_params* p, const double* z0, double rho, double h, double* z) {
  int K = p->K, n = K + 1;
  for (int m = 0; m < n; ++m) z[m] = z0[m];
  for (int it = 0; it < 30; ++it) {
    double w[ORC_KMAX], dw[ORC_KMAX][ORC_NMAX], A[ORC_NMAX][ORC_NMAX], r[ORC_NMAX];
    rates_and_jacobian(p, z, rho, w, dw);
    double cp = mixture_cp(p, z), hw = 0;
    for (int k = 0; k < K; ++k) hw += p->hf[k] * w[k];
    /* F_T = -hw / (rho cp) */
    for (int k = 0; k < K; ++k) {
      r[k] = -(z[k] - z0[k] - h * w[k] / rho);
      for (int m = 0; m < n; ++m) A[k][m] = (k == m ? 1.0 : 0.0) - h * dw[k][m] / rho;
    }
    r[K] = -(z[K] - z0[K] - h * (-hw / (rho * cp)));
    for (int m = 0; m < n; ++m) {
      double dhw = 0;
      for (int k = 0; k < K; ++k) dhw += p->hf[k] * dw[k][m];
      double dFT = -dhw / (rho * cp);
      if (m < K) dFT += hw * p->cp[m] / (rho * cp * cp);
      A[K][m] = (m == K ? 1.0 : 0.0) - h * dFT;
    }
    if (solve_dense(n, A, r)) return -1;
    double big = 0;
    for (int m = 0; m < n; ++m) {
      z[m] += r[m];
      double sc = m < K ? 1.0 : z0[K];
      double e = fabs(r[m]) / sc;
      if (!(e == e)) return -1;
      if (e > big) big = e;
    }
    if (!(z[K] > 0)) return -1;
    if (big < 1e-13) return 0;
  }
  return -1;
}

/* chemistry increments over one lattice step: dY[k], dT (K) */
int orc_chem_implicit(const orc_params* p, double T, const double* Y, double rho_lat, double* dY,
                      double* dT) {
  int K = p->K;
  double rho = rho_lat * p->rho_ref;
  double z0[ORC_NMAX], z[ORC_NMAX], zs[ORC_NMAX];
  for (int k = 0; k < K; ++k) z0[k] = Y[k];
  z0[K] = T;
  int ok = -1;
  for (int nsub = 1; nsub <= 64 && ok; nsub *= 2) {
    for (int m = 0; m <= K; ++m) zs[m] = z0[m];
    ok = 0;
    for (int s2 = 0; s2 < nsub && !ok; ++s2) {
      ok = be_newton(p, zs, rho, p->dt / nsub, z);
      for (int m = 0; m <= K; ++m) zs[m] = z[m];
    }
  }
  for (int k = 0; k < K; ++k) dY[k] = zs[k] - Y[k];
  *dT = zs[K] - T;
  return ok;
}

/* ----------------------------------------------------------- grid helpers */
static int ncell(const orc_params* p) { return p->nx * p->ny * (p->dim == 3 ? p->nz : 1); }
static int extent(const orc_params* p, int a) { return a == 0 ? p->nx : a == 1 ? p->ny : p->nz; }

/* Neighbour value along axis a, side s (-1/+1): periodic wraps; an inlet face
 * gives the inlet state (T_in, Y_in); a wall with a set temperature gives that
 * temperature; other walls and the outlet give the cell's own value (zero
 * normal gradient).  phi, Y at walls and Ts of ghosts are the cell's own. */
static void neighbour(const orc_params* p, const double* phi, const double* T, const double* Y,
                      const double* Ts, int N, const int xyz[3], int a, int s, cellv* out) {
  int q[3] = {xyz[0], xyz[1], xyz[2]};
  q[a] += s;
  int n = extent(p, a);
  int face = 2 * a + (s > 0 ? 1 : 0);
  int c0 = xyz[0] + p->nx * (xyz[1] + p->ny * xyz[2]);
  int ghost = 0;
  if (q[a] < 0 || q[a] >= n) {
    if (p->bc[face] == ORC_BC_PERIODIC) q[a] = (q[a] + n) % n;
    else ghost = 1;
  }
  if (!ghost) {
    int c = q[0] + p->nx * (q[1] + p->ny * q[2]);
    out->T = T[c];
    for (int k = 0; k < p->K; ++k) out->Y[k] = Y[(size_t)k * N + c];
    out->phi = phi[c];
    out->Ts = Ts ? Ts[c] : p->Ts_uniform;
    return;
  }
  out->phi = phi[c0];
  out->Ts = Ts ? Ts[c0] : p->Ts_uniform;
  if (p->bc[face] == ORC_BC_INLET) {
    out->T = p->T_in;
    for (int k = 0; k < p->K; ++k) out->Y[k] = p->Y_in[k];
  } else if (p->bc[face] == ORC_BC_WALL && p->wall_T[face] > 0.0) {
    out->T = p->wall_T[face];
    for (int k = 0; k < p->K; ++k) out->Y[k] = Y[(size_t)k * N + c0];
  } else {
    out->T = T[c0];
    for (int k = 0; k < p->K; ++k) out->Y[k] = Y[(size_t)k * N + c0];
  }
}

static void own(const orc_params* p, const double* phi, const double* T, const double* Y,
                const double* Ts, int N, int c, cellv* out) {
  out->T = T[c];
  for (int k = 0; k < p->K; ++k) out->Y[k] = Y[(size_t)k * N + c];
  out->phi = phi[c];
  out->Ts = Ts ? Ts[c] : p->Ts_uniform;
}

static void coords(const orc_params* p, int c, int xyz[3]) {
  xyz[0] = c % p->nx;
  xyz[1] = (c / p->nx) % p->ny;
  xyz[2] = c / (p->nx * p->ny);
}

/* Inlet velocity at a cell of the x = 0 column: uniform, uniform times the
 * cell's fluid fraction (profile 2: a diffuse-interface channel whose walls
 * are solid layers), or a parabola over each wall-bounded transverse axis
 * (walls half-way outside the domain). */
static double inlet_u(const orc_params* p, const int xyz[3], double phis) {
  double u = p->u_in;
  if (p->inlet_parabolic == 2) return u * (1.0 - phis);
  if (!p->inlet_parabolic) return u;
  for (int a = 1; a < p->dim; ++a) {
    if (p->bc[2 * a] != ORC_BC_WALL) continue;
    double n = extent(p, a), s = xyz[a] + 0.5;
    u *= 4.0 * s * (n - s) / (n * n);
  }
  return u;
}

/* --------------------------------------------------- FD transport (T, Y, Ts)
 * Conservative phi_f-weighted form of eqs. volume-averaged-species-equation-5
 * and energy-transport-DI-version, forward Euler, upwind convection with the
 * cell velocity, central diffusion with arithmetic-mean face coefficients, the
 * species-enthalpy term -(sum cp_k j_k).grad T with central gradients, the
 * lagged dP0/dt, omega_T and S_I = A_T lambda phi_f phi_s^2 / eta^2 (Ts - T).
 * u is the lattice velocity field u[a*N + c]; Tn/Yn/Tsn receive step n+1.
 * DTm (nullable) receives the material increments of the step that the
 * divergence needs, (1/T) DT/Dt + Mw sum_k (1/M_k) DY_k/Dt, each formed as
 * the step's increment plus u.grad of the field with central differences
 * (the gradient the LB source takes of rho); frozen cells: (T^{n+1} - T^n)/T. */
int orc_fd_phase(const orc_params* p, const double* phi, const double* T, const double* Y,
                 const double* Ts, const double* u, double P0, double P0prev,
                 double* Tn, double* Yn, double* Tsn, double* DTm) {
  int N = ncell(p), K = p->K, dim = p->dim;
  double eta2 = p->eta * p->eta;
  double Cs = p->rhocp_s / p->rho_ref;
  double Lams = p->lambda_s * p->dt / (p->rho_ref * p->dx * p->dx);
  #pragma omp parallel for schedule(static)
  for (int c = 0; c < N; ++c) {
    int xyz[3];
    coords(p, c, xyz);
    cellv v0, vm[3], vp[3];
    derv d0, dm[3], dp[3];
    own(p, phi, T, Y, Ts, N, c, &v0);
    derive(p, &v0, P0, &d0);
    for (int a = 0; a < dim; ++a) {
      neighbour(p, phi, T, Y, Ts, N, xyz, a, -1, &vm[a]);
      neighbour(p, phi, T, Y, Ts, N, xyz, a, +1, &vp[a]);
      derive(p, &vm[a], P0, &dm[a]);
      derive(p, &vp[a], P0, &dp[a]);
    }
    double phif = 1.0 - v0.phi, phis = v0.phi;
    int fluid_on = phif >= p->phi_min;
    int solid_on = p->Ts_field ? (phis >= p->phi_min) : 1;
    double SI = 0;
    if (fluid_on && solid_on)
      SI = p->A_T * d0.lam * phif * phis * phis / eta2 * (v0.Ts - v0.T);

    /* species */
    double omega[ORC_KMAX] = {0}, omegaT = 0;
    if (p->chem_mode == ORC_CHEM_EXPLICIT && K > 0 && fluid_on)
      orc_chem_rates(p, v0.T, v0.Y, d0.rho, omega, &omegaT);
    if (p->chem_mode == ORC_CHEM_IMPLICIT && K > 0 && fluid_on) {
      /* the implicit increments enter the FD update as rho dY_k and rho cp dT */
      double dY[ORC_KMAX], dT;
      orc_chem_implicit(p, v0.T, v0.Y, d0.rho, dY, &dT);
      for (int k = 0; k < K; ++k) omega[k] = d0.rho * dY[k];
      omegaT = d0.rho * d0.cp * dT;
    }
    double sYm = 0; /* sum_k (1/M_k) DY_k/Dt dt */
    for (int k = 0; k < K; ++k) {
      if (!fluid_on) { Yn[(size_t)k * N + c] = v0.Y[k]; continue; }
      double adv = 0, dif = 0;
      double kc = phif * d0.rho * d0.D[k];
      for (int a = 0; a < dim; ++a) {
        double ua = u[(size_t)a * N + c];
        if (ua > 0) adv += ua * (v0.Y[k] - vm[a].Y[k]);
        else adv += ua * (vp[a].Y[k] - v0.Y[k]);
        double km = 0.5 * (kc + (1.0 - vm[a].phi) * dm[a].rho * dm[a].D[k]);
        double kp = 0.5 * (kc + (1.0 - vp[a].phi) * dp[a].rho * dp[a].D[k]);
        dif += kp * (vp[a].Y[k] - v0.Y[k]) - km * (v0.Y[k] - vm[a].Y[k]);
      }
      double rhs = -phif * d0.rho * adv + dif + phif * omega[k];
      Yn[(size_t)k * N + c] = v0.Y[k] + rhs / (phif * d0.rho);
      double advc = 0; /* u.grad Y_k, central */
      for (int a = 0; a < dim; ++a) advc += u[(size_t)a * N + c] * 0.5 * (vp[a].Y[k] - vm[a].Y[k]);
      sYm += (Yn[(size_t)k * N + c] - v0.Y[k] + advc) / p->M[k];
    }

    /* temperature */
    if (fluid_on) {
      double adv = 0, dif = 0, cross = 0;
      double kc = phif * d0.lam;
      for (int a = 0; a < dim; ++a) {
        double ua = u[(size_t)a * N + c];
        if (ua > 0) adv += ua * (v0.T - vm[a].T);
        else adv += ua * (vp[a].T - v0.T);
        double km = 0.5 * (kc + (1.0 - vm[a].phi) * dm[a].lam);
        double kp = 0.5 * (kc + (1.0 - vp[a].phi) * dp[a].lam);
        dif += kp * (vp[a].T - v0.T) - km * (v0.T - vm[a].T);
        double gT = 0.5 * (vp[a].T - vm[a].T);
        for (int k = 0; k < K; ++k)
          cross += p->cp[k] * d0.D[k] * 0.5 * (vp[a].Y[k] - vm[a].Y[k]) * gT;
      }
      double rhs = -phif * d0.rho * d0.cp * adv + dif +
                   phif * (d0.rho * cross + (P0 - P0prev) / p->rho_ref + omegaT + SI);
      Tn[c] = v0.T + rhs / (phif * d0.rho * d0.cp);
      double advc = 0; /* u.grad T, central */
      for (int a = 0; a < dim; ++a) advc += u[(size_t)a * N + c] * 0.5 * (vp[a].T - vm[a].T);
      if (DTm) DTm[c] = (Tn[c] - v0.T + advc) / v0.T + d0.Mw * sYm;
    } else {
      Tn[c] = v0.Ts;
      if (DTm) DTm[c] = (v0.Ts - v0.T) / v0.T;
    }

    /* solid temperature (field mode) */
    if (p->Ts_field && Tsn) {
      if (phis >= p->phi_min) {
        double dif = 0;
        for (int a = 0; a < dim; ++a) {
          double km = 0.5 * (phis + vm[a].phi) * Lams;
          double kp = 0.5 * (phis + vp[a].phi) * Lams;
          dif += kp * (vp[a].Ts - v0.Ts) - km * (v0.Ts - vm[a].Ts);
        }
        /* a moving solid carries its temperature with u_s (upwind) */
        double advs = 0;
        for (int a = 0; a < dim; ++a) {
          double us = p->u_s[a];
          if (us > 0) advs += us * (v0.Ts - vm[a].Ts);
          else if (us < 0) advs += us * (vp[a].Ts - v0.Ts);
        }
        Tsn[c] = v0.Ts + (dif - phif * SI) / (phis * Cs) - advs;
      } else {
        Tsn[c] = v0.Ts;
      }
    }
  }
  return 0;
}

/* ------------------------------------------------------------ streaming */
/* The stored P_b advanced by dP_b/dt = -(L5 + L1)/2 over one lattice step
 * from the stored outlet columns (the boundary pressure of the next step). */
static double outlet_pb(const orc_params* p) {
  int NF = p->ny * (p->dim == 3 ? p->nz : 1);
  const double* ob = p->ob;
  /* plane wave: face means of the outlet columns */
  double P1 = 0, u1 = 0, P2 = 0, u2 = 0, r = 0;
  for (int f = 0; f < NF; ++f) {
    P1 += ob[NF + f]; u1 += ob[2 * NF + f]; P2 += ob[3 * NF + f]; u2 += ob[4 * NF + f];
    r += ob[5 * NF + f];
  }
  P1 /= NF; u1 /= NF; P2 /= NF; u2 /= NF; r /= NF;
  double pb = ob[0];
  double cs = sqrt(CS2);
  double L5 = (u1 + cs) * ((P1 - P2) + r * cs * (u1 - u2));
  double L1 = p->nscbc_K * pb;
  return pb - 0.5 * (L5 + L1);
}

/* Pull the populations arriving at cell c from the post-collision field gs,
 * applying the boundary rules; uw is the outlet wall-velocity estimate. */
static void pull(const orc_params* p, lat_t L, const double* gs, int N, int c, const int xyz[3],
                 double rho_c, double rho_in, double phis_c, const double* uw, double* gin) {
  double pb = (p->nscbc && p->bc[1] == ORC_BC_OUTLET && xyz[0] == p->nx - 1) ? p->ob[0] : 0.0;
  for (int i = 0; i < L.Q; ++i) {
    int s[3] = {xyz[0] - L.c[i][0], xyz[1] - L.c[i][1], xyz[2] - L.c[i][2]};
    int out_face[3] = {-1, -1, -1};
    for (int a = 0; a < p->dim; ++a) {
      int n = extent(p, a);
      if (s[a] < 0 || s[a] >= n) {
        int face = 2 * a + (s[a] >= n ? 1 : 0);
        if (p->bc[face] == ORC_BC_PERIODIC) s[a] = (s[a] + n) % n;
        else out_face[a] = face;
      }
    }
    int wall = -1, inlet = 0, outlet = 0;
    for (int a = 0; a < p->dim; ++a) {
      if (out_face[a] < 0) continue;
      int bc = p->bc[out_face[a]];
      if (bc == ORC_BC_WALL && wall < 0) wall = out_face[a];
      if (bc == ORC_BC_INLET) inlet = 1;
      if (bc == ORC_BC_OUTLET) outlet = 1;
    }
    int ib = opposite(L, i);
    if (wall >= 0) {
      double cu = 0;
      for (int a = 0; a < p->dim; ++a) cu += L.c[i][a] * p->wall_u[wall][a];
      gin[i] = gs[(size_t)ib * N + c] + 2.0 * L.w[i] * rho_c * cu;
    } else if (inlet) {
      double cu = L.c[i][0] * inlet_u(p, xyz, phis_c);
      gin[i] = gs[(size_t)ib * N + c] + 2.0 * L.w[i] * rho_in * cu;
    } else if (outlet) {
      double cu = 0, uu = 0;
      for (int a = 0; a < p->dim; ++a) { cu += L.c[i][a] * uw[a]; uu += uw[a] * uw[a]; }
      gin[i] = -gs[(size_t)ib * N + c] + L.w[i] * (2.0 * pb + rho_c * (cu * cu / CS2 - uu));
    } else {
      int sc = s[0] + p->nx * (s[1] + p->ny * s[2]);
      gin[i] = gs[(size_t)i * N + sc];
    }
  }
}

static int is_outlet_cell(const orc_params* p, const int xyz[3]) {
  return p->bc[1] == ORC_BC_OUTLET && xyz[0] == p->nx - 1;
}

/* Phase field of step n of a moving solid: the step-0 field phi0 displaced
 * by s = n u_s, phi_n(x) = phi0(x - s), multilinear interpolation between
 * the cells around x - s (periodic axes wrap, other axes clamp).  Without
 * motion phi0 itself. */
static const double* phase_at(const orc_params* p, const double* phi0, double n, double* buf) {
  if (!p->moving) return phi0;
  int N = ncell(p), dim = p->dim;
  int ish[3] = {0, 0, 0};
  double fr[3] = {0, 0, 0};
  for (int a = 0; a < dim; ++a) {
    double sa = n * p->u_s[a];
    ish[a] = (int)floor(sa);
    fr[a] = sa - ish[a];
  }
  #pragma omp parallel for schedule(static)
  for (int c = 0; c < N; ++c) {
    int xyz[3];
    coords(p, c, xyz);
    double v = 0;
    for (int corner = 0; corner < (1 << dim); ++corner) {
      double w = 1;
      int q[3] = {xyz[0], xyz[1], xyz[2]};
      for (int a = 0; a < dim; ++a) {
        int up = (corner >> a) & 1; /* 0: x - i, 1: x - i - 1 */
        w *= up ? fr[a] : 1.0 - fr[a];
        int n_a = extent(p, a), qa = xyz[a] - ish[a] - up;
        if (p->bc[2 * a] == ORC_BC_PERIODIC) qa = ((qa % n_a) + n_a) % n_a;
        else qa = qa < 0 ? 0 : (qa >= n_a ? n_a - 1 : qa);
        q[a] = qa;
      }
      v += w * phi0[q[0] + p->nx * (q[1] + p->ny * q[2])];
    }
    buf[c] = v;
  }
  return buf;
}

/* Pull + moments for every cell: gin (Q*N), u (dim*N), rho (N), Kd (N). */
static void stream_and_moments(const orc_params* p, lat_t L, const double* phi, const double* gs,
                               const double* T, const double* Y, double P0, double* gin_all,
                               double* u, double* rho, double* Kd, double* mu_out) {
  int N = ncell(p), dim = p->dim;
  double eta2 = p->eta * p->eta;
  double rho_in = eos_rho(p, P0, mixture_Mw(p, p->Y_in), p->T_in);
  #pragma omp parallel for schedule(static)
  for (int c = 0; c < N; ++c) {
    int xyz[3];
    coords(p, c, xyz);
    double Yc[ORC_KMAX];
    for (int k = 0; k < p->K; ++k) Yc[k] = Y[(size_t)k * N + c];
    double r = eos_rho(p, P0, mixture_Mw(p, Yc), T[c]);
    double mu = visc_of(p, T[c], Yc);
    double phis = phi[c], phif = 1.0 - phis;
    double kd = p->A_u * mu * phif * phis * phis / eta2;
    double gin[ORC_QMAX], uw[3] = {0, 0, 0}, uc[3] = {0, 0, 0};
    int passes = is_outlet_cell(p, xyz) ? 2 : 1;
    for (int pass = 0; pass < passes; ++pass) {
      pull(p, L, gs, N, c, xyz, r, rho_in, phis, uw, gin);
      for (int a = 0; a < dim; ++a) {
        double m = 0;
        for (int i = 0; i < L.Q; ++i) m += L.c[i][a] * gin[i];
        m /= CS2;
        /* rho u = m + F/2, F = F_b - K_d (u - u_s), implicit in u */
        uc[a] = (m + 0.5 * p->Fb[a] + 0.5 * kd * p->u_s[a]) / (r + 0.5 * kd);
      }
      for (int a = 0; a < dim; ++a) uw[a] = uc[a];
    }
    for (int i = 0; i < L.Q; ++i) gin_all[(size_t)i * N + c] = gin[i];
    for (int a = 0; a < dim; ++a) u[(size_t)a * N + c] = uc[a];
    rho[c] = r;
    Kd[c] = kd;
    mu_out[c] = mu;
  }
}

/* ----------------------------------------------------------- public API */
/* scal: [0] P0, [1] P0 of the previous step, [2] fluid mass m (lattice),
 * [3] I = sum phi_f Mw / T, [4] inlet mass flux, [5] outlet mass flux,
 * [6] step counter, [7] / [8] inlet / outlet mass flux summed over the steps,
 * [9] inlet peak speed of the next step, [10] fuel consumed in the last step. */
static double reduce_I(const orc_params* p, const double* phi, const double* T, const double* Y) {
  int N = ncell(p);
  double I = 0;
  for (int c = 0; c < N; ++c) {
    double Yc[ORC_KMAX];
    for (int k = 0; k < p->K; ++k) Yc[k] = Y[(size_t)k * N + c];
    I += (1.0 - phi[c]) * mixture_Mw(p, Yc) / T[c];
  }
  return I;
}

/* g = g_eq(P_h, rho, u) from the given T, Y, u (nullable: rest), P_h
 * (nullable: 0) and P0; m = sum phi_f rho = P0 I / (R rho_ref). */
int orc_init(const orc_params* p, const double* phi, double* g, const double* T, const double* Y,
             const double* u, const double* Ph, double P0, double* scal) {
  lat_t L = lattice_of(p->dim);
  int N = ncell(p);
  #pragma omp parallel for schedule(static)
  for (int c = 0; c < N; ++c) {
    double Yc[ORC_KMAX], uc[3] = {0, 0, 0}, geq[ORC_QMAX];
    for (int k = 0; k < p->K; ++k) Yc[k] = Y[(size_t)k * N + c];
    if (u)
      for (int a = 0; a < p->dim; ++a) uc[a] = u[(size_t)a * N + c];
    double r = eos_rho(p, P0, mixture_Mw(p, Yc), T[c]);
    orc_equilibrium(p->dim, Ph ? Ph[c] : 0.0, r, uc, geq);
    for (int i = 0; i < L.Q; ++i) g[(size_t)i * N + c] = geq[i];
  }
  double I = reduce_I(p, phi, T, Y);
  scal[0] = P0;
  scal[1] = P0;
  scal[2] = P0 * I / (ORC_R * p->rho_ref);
  scal[3] = I;
  scal[4] = scal[5] = 0;
  scal[6] = 0;
  scal[7] = scal[8] = 0; /* inlet / outlet mass flux summed over the steps */
  scal[9] = p->u_in;     /* inlet peak speed of the next step */
  scal[10] = 0;          /* fuel consumed in the last step (feedback) */
  return 0;
}

/* Velocity, density and sum-of-populations pressure that the next step will
 * see at every cell (pull + moments of the current state, no collision). */
int orc_moments(const orc_params* p_in, const double* phi0, const double* g, const double* T,
                const double* Y, const double* scal, double* u, double* rho, double* Ph) {
  orc_params pc = *p_in; /* the inlet speed of the next step */
  pc.u_in = scal[9];
  const orc_params* p = &pc;
  double* phibuf = p->moving ? malloc(sizeof(double) * (size_t)ncell(p)) : NULL;
  const double* phi = phase_at(p, phi0, scal[6], phibuf);
  lat_t L = lattice_of(p->dim);
  int N = ncell(p);
  double* gin = malloc(sizeof(double) * (size_t)L.Q * N);
  double* Kd = malloc(sizeof(double) * N);
  double* mu = malloc(sizeof(double) * N);
  stream_and_moments(p, L, phi, g, T, Y, scal[0], gin, u, rho, Kd, mu);
  for (int c = 0; c < N; ++c) {
    double s = 0;
    for (int i = 0; i < L.Q; ++i) s += gin[(size_t)i * N + c];
    Ph[c] = s;
  }
  free(gin); free(Kd); free(mu);
  if (phibuf) free(phibuf);
  return 0;
}

/* One full time step n -> n+1 (in place on g, T, Y, Ts, scal).  diag
 * (nullable) receives u (dim*N), rho (N), P_h (N), D (N) of step n. */
/* Fuel (species fb_k) consumed over one step by the chemistry of the state
 * (T, Y) at pressure P0: sum over fluid cells of phi_f (-omega_F) in lattice
 * units (explicit rates, or the implicit increments times rho). */
static double fuel_consumed(const orc_params* p, const double* phi, const double* T,
                            const double* Y, double P0) {
  int N = ncell(p), K = p->K;
  double s = 0;
  for (int c = 0; c < N; ++c) {
    double phif = 1.0 - phi[c];
    if (!(phif >= p->phi_min)) continue;
    double Yc[ORC_KMAX];
    for (int k = 0; k < K; ++k) Yc[k] = Y[(size_t)k * N + c];
    double rho = eos_rho(p, P0, mixture_Mw(p, Yc), T[c]);
    double om[ORC_KMAX] = {0}, omT = 0;
    if (p->chem_mode == ORC_CHEM_EXPLICIT) {
      orc_chem_rates(p, T[c], Yc, rho, om, &omT);
    } else if (p->chem_mode == ORC_CHEM_IMPLICIT) {
      double dY[ORC_KMAX], dT;
      orc_chem_implicit(p, T[c], Yc, rho, dY, &dT);
      for (int k = 0; k < K; ++k) om[k] = rho * dY[k];
    }
    s += phif * (-om[p->fb_k]);
  }
  return s;
}

/* the inlet profile summed over the inlet face (the area of the feedback) */
static double inlet_area(const orc_params* p) {
  orc_params q = *p;
  q.u_in = 1.0;
  double a = 0;
  int nz = p->dim == 3 ? p->nz : 1;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < p->ny; ++y) {
      int xyz[3] = {0, y, z};
      a += inlet_u(&q, xyz, 0.0);
    }
  return a;
}

int orc_step(const orc_params* p_in, const double* phi0, double* g, double* T, double* Y,
             double* Ts, double* scal, double* diag) {
  /* the inlet speed of this step is scal[9] (the feedback moves it) */
  orc_params pc = *p_in;
  pc.u_in = scal[9];
  const orc_params* p = &pc;
  /* a moving solid: the phase field of this step (scal[6] steps taken) */
  double* phibuf = p->moving ? malloc(sizeof(double) * (size_t)ncell(p)) : NULL;
  const double* phi = phase_at(p, phi0, scal[6], phibuf);
  double fuel = p->feedback ? fuel_consumed(p, phi, T, Y, scal[0]) : 0.0;
  lat_t L = lattice_of(p->dim);
  int N = ncell(p), dim = p->dim, K = p->K;
  double P0 = scal[0], P0prev = scal[1];
  double* gin = malloc(sizeof(double) * (size_t)L.Q * N);
  double* u = malloc(sizeof(double) * (size_t)dim * N);
  double* rho = malloc(sizeof(double) * N);
  double* Kd = malloc(sizeof(double) * N);
  double* mu = malloc(sizeof(double) * N);
  double* Tn = malloc(sizeof(double) * N);
  double* Yn = malloc(sizeof(double) * (size_t)(K > 0 ? K : 1) * N);
  double* Tsn = p->Ts_field ? malloc(sizeof(double) * N) : NULL;

  /* 1-2: EOS, pull streaming with boundary rules, moments, implicit drag */
  stream_and_moments(p, L, phi, g, T, Y, P0, gin, u, rho, Kd, mu);

  /* 3: FD transport of T, Y (and Ts) with u^n, rho^n, explicit chemistry */
  double* DTm = malloc(sizeof(double) * N);
  orc_fd_phase(p, phi, T, Y, p->Ts_field ? Ts : NULL, u, P0, P0prev, Tn, Yn, Tsn, DTm);

  /* 4-5: divergence from the low-Mach constraint, source, collision */
  int NF = p->ny * (dim == 3 ? p->nz : 1);
  double* obnew = (p->nscbc && p->bc[1] == ORC_BC_OUTLET) ? malloc(sizeof(double) * 5 * (size_t)NF) : NULL;
  #pragma omp parallel for schedule(static)
  for (int c = 0; c < N; ++c) {
    int xyz[3];
    coords(p, c, xyz);
    /* D = (1/T) DT/Dt + Mw sum_k (1/M_k) DY_k/Dt - (1/P0) dP0/dt: the
     * continuity equation with the EOS (Sec. 3, eq. rho-in-terms-of-P0-and-T)
     * at uniform P0, with the material increments of this step */
    double D = DTm[c] - (P0 - P0prev) / P0;

    double r = rho[c], uc[3] = {0, 0, 0}, G[3] = {0, 0, 0}, F[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) uc[a] = u[(size_t)a * N + c];
    for (int a = 0; a < dim; ++a) {
      cellv vm, vp;
      neighbour(p, phi, T, Y, p->Ts_field ? Ts : NULL, N, xyz, a, -1, &vm);
      neighbour(p, phi, T, Y, p->Ts_field ? Ts : NULL, N, xyz, a, +1, &vp);
      double rm = eos_rho(p, P0, mixture_Mw(p, vm.Y), vm.T);
      double rp = eos_rho(p, P0, mixture_Mw(p, vp.Y), vp.T);
      G[a] = CS2 * 0.5 * (rp - rm);
      F[a] = p->Fb[a] - Kd[c] * (uc[a] - p->u_s[a]);
    }
    double sg = 0;
    for (int i = 0; i < L.Q; ++i) sg += gin[(size_t)i * N + c];
    /* P_h = sum g + half the zeroth moment of Xi, sum_i Xi_i = u.G + rho cs^2 D,
     * so that each step adds the whole source to sum g */
    double uG = 0;
    for (int a = 0; a < dim; ++a) uG += uc[a] * G[a];
    double Ph = sg + 0.5 * (r * CS2 * D + uG);
    double geq[ORC_QMAX], xi[ORC_QMAX];
    orc_equilibrium(dim, Ph, r, uc, geq);
    orc_source(dim, r, G, uc, F, D, xi);
    double tau = 0.5 + mu[c] / (r * CS2);
    for (int i = 0; i < L.Q; ++i) {
      double gi = gin[(size_t)i * N + c];
      g[(size_t)i * N + c] = gi - (gi - geq[i]) / tau + (1.0 - 1.0 / (2.0 * tau)) * xi[i];
    }
    if (diag) {
      for (int a = 0; a < dim; ++a) diag[(size_t)a * N + c] = uc[a];
      diag[(size_t)dim * N + c] = r;
      diag[(size_t)(dim + 1) * N + c] = Ph;
      diag[(size_t)(dim + 2) * N + c] = D;
    }
    if (obnew && xyz[0] >= p->nx - 2) {
      int col = xyz[0] == p->nx - 1 ? 0 : 1, f = xyz[1] + p->ny * xyz[2];
      obnew[(2 * col) * NF + f] = Ph;
      obnew[(2 * col + 1) * NF + f] = uc[0];
      if (col == 0) obnew[4 * NF + f] = r;
    }
  }
  /* characteristic outlet: keep this step's outlet columns, then advance P_b
   * with them to the boundary pressure of the next step */
  if (obnew) {
    memcpy(p->ob + NF, obnew, sizeof(double) * 5 * (size_t)NF);
    double pb = outlet_pb(p);
    for (int f = 0; f < NF; ++f) p->ob[f] = pb;
    free(obnew);
  }

  /* 6: global FP64 reduction -> P0^{n+1} */
  double fin = 0, fout = 0;
  if (p->bc[0] == ORC_BC_INLET || p->bc[1] == ORC_BC_OUTLET) {
    for (int c = 0; c < N; ++c) {
      int x = c % p->nx;
      double f = (1.0 - phi[c]) * rho[c] * u[c];
      if (x == 0 && p->bc[0] == ORC_BC_INLET) fin += f;
      if (x == p->nx - 1 && p->bc[1] == ORC_BC_OUTLET) fout += f;
    }
  }
  memcpy(T, Tn, sizeof(double) * N);
  if (K > 0) memcpy(Y, Yn, sizeof(double) * (size_t)K * N);
  if (p->Ts_field) memcpy(Ts, Tsn, sizeof(double) * N);
  double I = reduce_I(p, phi, T, Y);
  double m = scal[2];
  double P0n = P0;
  if (p->p0_mode != ORC_P0_FIXED) P0n = m * ORC_R * p->rho_ref / I;
  scal[1] = P0;
  scal[0] = P0n;
  scal[2] = m;
  scal[3] = I;
  scal[4] = fin;
  scal[5] = fout;
  scal[6] += 1;
  scal[7] += fin;
  scal[8] += fout;
  scal[10] = fuel;
  if (p->feedback) {
    /* inflow of fuel rho_in Y_F,in u_in A equals the fuel the step consumed */
    double rho_in = eos_rho(p, P0, mixture_Mw(p, p->Y_in), p->T_in);
    double u = fuel / (rho_in * p->Y_in[p->fb_k] * inlet_area(p));
    scal[9] = u < 0.0 ? 0.0 : (u > 0.3 ? 0.3 : u);
  }

  free(gin); free(u); free(rho); free(Kd); free(mu); free(Tn); free(Yn); free(DTm);
  if (phibuf) free(phibuf);
  if (Tsn) free(Tsn);
  return 0;
}

/* Diagnostics of the current state (what the next step sees), plain sums
 * over the cells, lattice units:
 *   out[0..2] drag: sum K_d u, the force of the fluid on the solid phase
 *             (Sec. 3.2.1, eq. Fdrag-empirical-law with u_s = 0);
 *   out[3]    heat: sum phi_f S_I, the heat flowing from the solid into the
 *             fluid per step (Sec. 3.3, eq. diffusion-heat-flux-3, read as
 *             relaxation toward Ts);
 *   out[4]    fluid mass: sum phi_f rho;
 *   out[5]    sum over the outlet column of rho u_x cp T, and
 *   out[6]    of rho u_x cp: their ratio is the mixing-cup temperature T_m of
 *             Sec. 4.2, eq. Tmean-def (0 / 0 without an outlet). */
int orc_diagnostics(const orc_params* p_in, const double* phi0, const double* g, const double* T,
                    const double* Y, const double* Ts, const double* scal, double* out) {
  orc_params pc = *p_in; /* the inlet speed of the next step */
  pc.u_in = scal[9];
  const orc_params* p = &pc;
  double* phibuf = p->moving ? malloc(sizeof(double) * (size_t)ncell(p)) : NULL;
  const double* phi = phase_at(p, phi0, scal[6], phibuf);
  lat_t L = lattice_of(p->dim);
  int N = ncell(p), dim = p->dim;
  double* gin = malloc(sizeof(double) * (size_t)L.Q * N);
  double* u = malloc(sizeof(double) * (size_t)dim * N);
  double* rho = malloc(sizeof(double) * N);
  double* Kd = malloc(sizeof(double) * N);
  double* mu = malloc(sizeof(double) * N);
  stream_and_moments(p, L, phi, g, T, Y, scal[0], gin, u, rho, Kd, mu);
  for (int k = 0; k < 7; ++k) out[k] = 0;
  double eta2 = p->eta * p->eta;
  for (int c = 0; c < N; ++c) {
    int xyz[3];
    coords(p, c, xyz);
    cellv v;
    derv d;
    own(p, phi, T, Y, p->Ts_field ? Ts : NULL, N, c, &v);
    derive(p, &v, scal[0], &d);
    double phis = v.phi, phif = 1.0 - phis;
    for (int a = 0; a < dim; ++a) out[a] += Kd[c] * (u[(size_t)a * N + c] - p->u_s[a]);
    int fluid_on = phif >= p->phi_min;
    int solid_on = p->Ts_field ? (phis >= p->phi_min) : 1;
    if (fluid_on && solid_on) out[3] += phif * (p->A_T * d.lam * phif * phis * phis / eta2 * (v.Ts - v.T));
    out[4] += phif * rho[c];
    if (p->bc[1] == ORC_BC_OUTLET && xyz[0] == p->nx - 1) {
      out[5] += rho[c] * u[c] * d.cp * v.T;
      out[6] += rho[c] * u[c] * d.cp;
    }
  }
  free(gin); free(u); free(rho); free(Kd); free(mu);
  if (phibuf) free(phibuf);
  return 0;
}

int orc_run(const orc_params* p, const double* phi, double* g, double* T, double* Y, double* Ts,
            double* scal, int nsteps) {
  for (int n = 0; n < nsteps; ++n) orc_step(p, phi, g, T, Y, Ts, scal, NULL);
  return 0;
}

int orc_params_size(void) { return (int)sizeof(orc_params); }

/* The phase field of step n into out (N). */
int orc_phase_at(const orc_params* p, const double* phi0, double n, double* out) {
  const double* ph = phase_at(p, phi0, n, out);
  if (ph != out) memcpy(out, ph, sizeof(double) * (size_t)ncell(p));
  return 0;
}

/* Host threads used by the per-cell loops (n <= 0: all cores); returns the
 * number in effect (1 without OpenMP). */
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n <= 0) n = omp_get_num_procs();
  omp_set_num_threads(n);
  return n;
#else
  (void)n;
  return 1;
#endif
}
