/*
 * pflb.h -- C ABI of the GB300 PF-LB-FD time-step library (libpflb.so).
 *
 * The library advances the low-Mach phase-field / lattice-Boltzmann /
 * finite-difference model of Namdar, Norouzi & Varnik (arXiv 2310.17214) on
 * one NVIDIA GB300 GPU (sm_103a):
 *   (a) pull-scheme D2Q9 / D3Q19 collide-stream of the pressure-based
 *       populations g_i (Sec. 3.3, eqs. pop-g, body-force, eq-pop-f, eq-pop-g)
 *       with the diffuse-interface drag of Sec. 3.2.1 (eq. Fdrag-empirical-law)
 *       and the velocity-divergence source of the low-Mach constraint;
 *   (b) explicit finite-difference transport of T and Y_k (Sec. 3.2.2 eq.
 *       volume-averaged-species-equation-5, Sec. 3.3 eq.
 *       energy-transport-DI-version) with the heat coupling S_I (eq.
 *       diffusion-heat-flux-3);
 *   (c) the per-cell reaction source (Sec. 3.2.2 eq. 8, Sec. 3.3 eq. 9);
 *   (d) the FP64 global reduction for the thermodynamic pressure P0
 *       (Sec. 3.1, closure P0 = m R / int(Mw/T) dV).
 *
 * Conventions for every entry point:
 *   - All functions return an int status (PFLB_OK = 0 or a negative code);
 *     no exception crosses the ABI.  pflb_last_error() gives a message.
 *   - "where" is PFLB_HOST or PFLB_DEVICE for the caller's buffer.  Device
 *     buffers must live on the domain's device.  The library copies what it
 *     needs; the caller keeps ownership of every buffer it passes.
 *   - The library owns all device memory of a domain (allocated at create,
 *     released at destroy).  Work is queued on the domain's CUDA stream
 *     (desc.stream, NULL = the legacy default stream).
 *   - Field layout: cell = x + nx*(y + ny*z) (x fastest); multi-component
 *     fields are component-major (Y[k*N + cell], u[a*N + cell]).
 *   - A handle is not thread-safe; use one stream per domain.
 */
#ifndef PFLB_H
#define PFLB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PFLB_OK 0
#define PFLB_ERR_ARG -1
#define PFLB_ERR_OOM -2
#define PFLB_ERR_CUDA -3
#define PFLB_ERR_STATE -4       /* calls made in the wrong order */
#define PFLB_ERR_UNSTABLE -5    /* tau <= 1/2 or diffusion number too large at create; NaN at run */
#define PFLB_ERR_TIMEOUT -6     /* a bounded device wait ran out */
#define PFLB_ERR_UNSUPPORTED -7

/* precision modes */
#define PFLB_FP64 0             /* FP64 compute and storage */
#define PFLB_FP32 1             /* FP32 compute and storage; P0 / mass reductions in FP64 */
#define PFLB_FP32_FP16STORE 2   /* FP32 compute; populations stored as FP16 residuals from the
                                   cell's first-order equilibrium w_i (P + 3 c_i.j), with the
                                   cell's moments (P, j) in FP32 */

/* boundary kinds per face (x-lo, x-hi, y-lo, y-hi, z-lo, z-hi) */
#define PFLB_BC_PERIODIC 0
#define PFLB_BC_WALL 1          /* half-way bounce-back (optionally moving), T Dirichlet or adiabatic */
#define PFLB_BC_INLET 2         /* x-lo only: moving-wall bounce-back with the inlet velocity, Dirichlet T, Y */
#define PFLB_BC_OUTLET 3        /* x-hi only: anti-bounce-back P_h = 0, zero-gradient T, Y */

/* thermodynamic-pressure closure */
#define PFLB_P0_FIXED 0         /* open domain: P0 stays at its initial (ambient) value */
#define PFLB_P0_CLOSED 1        /* closed domain: P0 = m R / sum(phi_f Mw / T) dV with m fixed */

/* chemistry */
#define PFLB_CHEM_NONE 0
#define PFLB_CHEM_EXPLICIT 1    /* forward-Euler Arrhenius source */
#define PFLB_CHEM_IMPLICIT 2    /* per-cell backward Euler + Newton, FP64 state and residual
                                   (operator split); FP32 domains build and eliminate the
                                   Newton matrix in FP32, the root is the same (update < 1e-13) */
#define PFLB_CHEM_SURROGATE 3   /* learned MLP increments, Newton fallback (six species); the
                                   fallback of FP32 domains is an FP32 backward-Euler step in
                                   increment form, converged to a few ulp of the fields */

#define PFLB_HOST 0
#define PFLB_DEVICE 1

#define PFLB_KMAX 8
#define PFLB_JMAX 4

/* field selectors for set/get */
#define PFLB_FIELD_T 1u         /* temperature (K), N values */
#define PFLB_FIELD_Y 2u         /* mass fractions, K*N values */
#define PFLB_FIELD_TS 4u        /* solid temperature (K), N values */
#define PFLB_FIELD_U 8u         /* velocity (lattice units), dim*N values (get only) */
#define PFLB_FIELD_RHO 16u      /* density / rho_ref, N values (get only) */
#define PFLB_FIELD_PH 32u       /* sum of populations (lattice pressure), N values (get only) */
#define PFLB_FIELD_G 64u        /* post-collision populations, Q*N values (get only) */

#define PFLB_DTYPE_F64 0
#define PFLB_DTYPE_F32 1

typedef struct pflb_domain pflb_domain;

/* Physical description of one domain.  Units are SI except where noted; with
 * dx = dt = 1 and rho_ref = 1 every quantity is read in lattice units. */
typedef struct pflb_domain_desc {
  int dim;                 /* 2 -> D2Q9, 3 -> D3Q19 */
  int nx, ny, nz;          /* nz ignored (1) for dim == 2 */
  int precision;           /* PFLB_FP64 / PFLB_FP32 / PFLB_FP32_FP16STORE */
  int bc[6];
  double wall_u[6][3];     /* wall velocity per face (lattice units) */
  double wall_T[6];        /* wall temperature per face (K); 0 = adiabatic */
  double dx, dt, rho_ref;  /* grid spacing (m), time step (s), reference density (kg/m^3) */
  double M0, cp0;          /* single-gas molar mass (kg/mol), heat capacity (J/kg/K) when K = 0 */
  double mu_ref;           /* dynamic viscosity (Pa s); Sutherland reference value if enabled */
  int sutherland;          /* 1: mu(T) = mu_ref (T/suth_T)^1.5 (suth_T + suth_S)/(T + suth_S) */
  double suth_T, suth_S;
  double Pr;               /* Prandtl number: lambda = mu cp / Pr */
  double A_u, A_T, eta;    /* coupling parameters, interface width (cells) */
  double Fb[3];            /* body-force density (lattice units) */
  int inlet_parabolic;     /* inlet profile: 0 uniform, 1 parabola across wall-bounded axes,
                              2 uniform times the inlet cell's fluid fraction 1 - phi_s (a
                              channel whose walls are diffuse solid layers, Sec. 4.1) */
  double u_in, T_in;       /* inlet peak velocity (lattice units), temperature (K) */
  int p0_mode;             /* PFLB_P0_FIXED / PFLB_P0_CLOSED */
  double P0;               /* initial thermodynamic pressure (Pa) */
  int Ts_field;            /* 0: solid at the uniform Ts_uniform; 1: transported solid temperature */
  double Ts_uniform;       /* K */
  double rhocp_s, lambda_s;/* solid volumetric heat capacity (J/m^3/K), conductivity (W/m/K) */
  double phi_min;          /* phase fraction below which a phase is frozen (e.g. 1e-6) */
  double T_max;            /* hottest temperature the run may reach (K), e.g. the adiabatic
                              flame temperature; 0 = none beyond T_in, Ts_uniform and the
                              wall temperatures.  Only the stability checks read it. */
  int outlet_nscbc;        /* 1: partially non-reflecting outlet (Sec. 4.1, the
                              characteristic outlet of Poinsot and Lele).  The
                              anti-bounce-back imposes a boundary pressure P_b instead of
                              P_h = 0; after every step P_b advances by
                              dP_b/dt = -(L5 + L1)/2 with the outgoing plane wave
                              L5 = (u + cs)(dP_h/dx + rho cs du/dx) from the face means of
                              P_h, u_x (one-sided over the two outlet columns) and rho of
                              the outlet column, and L1 = K P_b, K = nscbc_sigma cs / nx
                              (the Mach-number factor 1 - Ma^2 taken as 1).  Needs an
                              outlet face; pflb_batch_step and pflb_step_noalloc refuse it.
                              0: P_h = 0. */
  double nscbc_sigma;      /* relaxation factor sigma of K (e.g. 0.25) */
  double u_s[3];           /* velocity of a rigidly translating solid (lattice units; Sec. 2,
                              the interface velocity v_I).  Nonzero: the phase field given to
                              pflb_set_phase_field is the one of step 0 and the phase field of
                              step n is it displaced by n u_s (multilinear interpolation between
                              cells; periodic axes wrap, other axes clamp), the drag acts on
                              u - u_s and the solid temperature is carried with u_s (upwind).
                              pflb_batch_step and pflb_step_noalloc refuse it.  Zero: a static
                              solid. */
  void* stream;            /* cudaStream_t (NULL = legacy default stream) */
  int device;              /* CUDA device ordinal */
} pflb_domain_desc;

/* Species thermochemistry and reactions (Sec. 3.2.2 eq. 8, Sec. 3.3 eq. 9).
 * Q_j = A_j T^b_j exp(-EaR_j / T) prod_k C_k^order_jk, C_k = rho Y_k / M_k,
 * minus, for a reversible reaction, Q_j,r = (k_f / K_c) prod_k C_k^rorder_jk with
 * K_c = exp(dS_j/R - dH_j/(R T)) (p_ref/(R T))^(sum_k stoich_jk). */
typedef struct pflb_mechanism {
  int K;                   /* species (0, 5 or 6 are compiled) */
  int J;                   /* reactions, <= PFLB_JMAX */
  int chem_mode;           /* PFLB_CHEM_NONE / _EXPLICIT / _IMPLICIT */
  double M[PFLB_KMAX];     /* kg/mol */
  double cp[PFLB_KMAX];    /* J/kg/K (constant) */
  double hf[PFLB_KMAX];    /* formation enthalpy, J/kg */
  double Dref[PFLB_KMAX];  /* m^2/s at D_Tref */
  double D_Tref, D_exp;    /* D_k = Dref_k (T / D_Tref)^D_exp */
  double Y_in[PFLB_KMAX];  /* inlet composition */
  double A[PFLB_JMAX], b[PFLB_JMAX], EaR[PFLB_JMAX];
  double order[PFLB_JMAX][PFLB_KMAX];
  double stoich[PFLB_JMAX][PFLB_KMAX];
  int rev[PFLB_JMAX];      /* 1: reversible */
  double dH[PFLB_JMAX], dS[PFLB_JMAX];    /* standard reaction enthalpy (J/mol), entropy (J/mol/K) */
  double rorder[PFLB_JMAX][PFLB_KMAX];    /* reverse orders */
  double p_ref;            /* standard pressure of K_c (Pa) */
  /* Transport.  PFLB_TRANSPORT_SINGLE: the description's viscosity law
   * (mu_ref, Sutherland) and lambda = mu cp / Pr for the whole mixture.
   * PFLB_TRANSPORT_MIXTURE: mixture-averaged values (Sec. 4.4, eqs. muT_mix,
   * phi_mix, conduct_mix) -- mu = sum_k mu_k X_k / sum_j Phi_kj X_j with
   * Wilke's Phi_kj, lambda = (sum_k X_k lambda_k + 1 / sum_k X_k / lambda_k) / 2 --
   * from the species' Sutherland laws mu_k(T) = mu_k (T / suth_Tk)^1.5
   * (suth_Tk + suth_Sk) / (T + suth_Sk) and the modified Eucken relation
   * lambda_k = mu_k (1.32 cv_k + 1.77 R / M_k), cv_k = cp_k - R / M_k. */
  int transport;
  double mu_k[PFLB_KMAX], suth_Tk[PFLB_KMAX], suth_Sk[PFLB_KMAX];
  /* Inlet mass-flow feedback (Sec. 4.4.1: a flame held stationary by the
   * inflow).  0: off, the inlet speed is the description's u_in.  k + 1: after
   * every step the inlet peak speed of the next step is set so that species k
   * flows in as fast as that step consumed it,
   *   u_in = sum_cells phi_f (-omega_k) / (rho_in Y_in[k] A),
   * omega_k the step's reaction source of the cells' state at its start (the
   * rates, or the increments of the implicit integrator or surrogate times
   * rho), rho_in the inlet density and A the inlet profile summed over the
   * inlet face at unit peak speed; the result is held in [0, 0.3].  The
   * description's u_in is the speed of the first step.  Needs an inlet face,
   * PFLB_P0_FIXED, Y_in[k] > 0 and an inlet profile other than 2;
   * pflb_batch_step and pflb_step_noalloc
   * refuse such a domain (PFLB_ERR_UNSUPPORTED).  pflb_get_scalars reports
   * the current speed and the consumption it came from. */
  int inlet_feedback;
} pflb_mechanism;

#define PFLB_TRANSPORT_SINGLE 0
#define PFLB_TRANSPORT_MIXTURE 1

typedef struct pflb_scalars {
  double P0;               /* thermodynamic pressure at the current step (Pa) */
  double P0_prev;          /* at the previous step */
  double mass;             /* fluid mass used by the closure (lattice units) */
  double I;                /* sum phi_f Mw / T over the domain */
  double flux_in, flux_out;/* inlet / outlet mass flux of the last step (lattice units) */
  long long step;          /* steps taken */
  int status;              /* latched device status (PFLB_OK or PFLB_ERR_UNSTABLE) */
  double u_in;             /* inlet peak speed of the next step (lattice units) */
  double fuel;             /* with the inlet feedback: sum phi_f (-omega_k) of the last
                              step (lattice units); else 0 */
  double outlet_pb;        /* boundary pressure of the next step at the characteristic
                              outlet (lattice units); else 0 */
} pflb_scalars;

/* Create a domain: validates the description, then allocates every device
 * array (populations double-buffered for the pull scheme).
 *
 * Checks before any CUDA call (so they run without a GPU):
 *   PFLB_ERR_ARG / PFLB_ERR_UNSUPPORTED -- lattice extent, precision, boundary
 *     kinds (periodic faces in pairs, inlet only at x-lo, outlet only at
 *     x-hi), positive and finite dx, dt, rho_ref, Pr, eta, P0, mu_ref, M0, cp0;
 *   PFLB_ERR_UNSTABLE -- the explicit scheme of Sec. 3.3 (BGK collision,
 *     forward-Euler FD) is outside its stability range at one of T_in,
 *     Ts_uniform, the wall temperatures or T_max, with the single gas of the
 *     description (M0): relaxation time tau = 1/2 + nu/cs^2 not above 1/2,
 *     thermal diffusion number lambda dt / (rho cp dx^2) above 1/(2 dim)
 *     (1/4 in 2-D, 1/6 in 3-D), solid diffusion number above the same
 *     limit, interface exchange number A_T lambda dt / (rho cp (eta dx)^2)
 *     not below 2 (the forward-Euler bound of the relaxation toward Ts), or
 *     |u_in| at or above the lattice sound speed 1/sqrt(3).
 *     pflb_set_mechanism repeats the check with the inlet mixture and the
 *     species diffusion numbers D_k(T) dt / dx^2.
 * Other errors: PFLB_ERR_OOM, PFLB_ERR_CUDA.  On error *out is NULL and
 * pflb_last_error(NULL) names the failed check. */
int pflb_create_domain(const pflb_domain_desc* desc, pflb_domain** out);

/* The checks pflb_create_domain makes (and, when mech is not NULL, those of
 * pflb_set_mechanism with that mechanism), without any CUDA call: PFLB_OK or
 * the code create / set_mechanism would return, the reason in
 * pflb_last_error(NULL). */
int pflb_validate(const pflb_domain_desc* desc, const pflb_mechanism* mech);

/* Static solid fraction phi_s in [0, 1] (N values, sum of phase fractions
 * is one, Sec. 2 eq. sum-varphialpha) and, when Ts_field, the initial solid
 * temperature (N values; NULL = Ts_uniform everywhere).  dtype: F64/F32. */
int pflb_set_phase_field(pflb_domain* d, const void* phi_s, const void* Ts, int dtype, int where);

/* Species data and reactions; must precede pflb_set_fields when K > 0.
 * K must be one of the compiled species counts (0, 5, 6).  Returns
 * PFLB_ERR_UNSTABLE when the inlet mixture breaks one of the stability limits
 * listed under pflb_create_domain (gas and species diffusion numbers, tau). */
int pflb_set_mechanism(pflb_domain* d, const pflb_mechanism* m);

/* Initial T (and Y when K > 0; optional velocity u, dim*N values, NULL = rest).
 * Sets g = g_eq(P_h = 0, rho, u), P0 = desc.P0 and the closure mass m.
 * mask selects the fields present in the packed buffer `src` (T, then Y,
 * then u), dtype F64/F32. */
int pflb_set_fields(pflb_domain* d, unsigned mask, const void* src, int dtype, int where);

/* Advance nsteps time steps asynchronously on the domain's stream.  A NaN
 * or an instability latches PFLB_ERR_UNSTABLE in the device status word (a
 * NaN in T, Y, the populations' sum or the velocity of any cell makes the
 * step's FP64 reduction NaN); a bounded device wait that ran out latches
 * PFLB_ERR_TIMEOUT.  The latched code is returned by the next synchronising
 * call (get_fields / get_scalars); the fields are then not to be trusted.
 * A call for 32 steps or more replays pairs of steps from a CUDA graph that
 * it captures on a private stream (not for a moving solid); the graph is
 * launched on the domain's stream, so the call must not run while that
 * stream is being captured. */
int pflb_step(pflb_domain* d, int nsteps);

/* Copy fields out, packed in the order T, Y, Ts, U, RHO, PH, G of the mask
 * bits.  U, RHO and PH are the moments the next step will see (pull and
 * boundary rules applied, no collision).  Synchronises the stream. */
int pflb_get_fields(pflb_domain* d, unsigned mask, void* dst, size_t bytes, int dtype, int where);

/* Host copy of the scalar state; synchronises the stream. */
int pflb_get_scalars(pflb_domain* d, pflb_scalars* out);

/* Diagnostics of the current state (the state the next step sees), FP64 sums
 * over the cells in lattice units (dx = dt = rho_ref = 1):
 *   drag     sum K_d u, the force of the fluid on the solid phase (Sec.
 *            3.2.1, eq. Fdrag-empirical-law with u_s = 0); a drag coefficient
 *            is 2 drag_x / (rho u_ref^2 D);
 *   heat     sum phi_f S_I, the heat passing from the solid into the fluid per
 *            step (Sec. 3.3, eq. diffusion-heat-flux-3, read as relaxation
 *            toward Ts), in lattice units of rho_ref cp T; a Nusselt number of
 *            a particle of diameter D is heat / (pi lambda dT) in 2-D;
 *   mass     sum phi_f rho, the fluid mass;
 *   outlet_Tm  mixing-cup temperature of the outlet column (Sec. 4.2, eq.
 *            Tmean-def), 0 without an outlet or outflow;
 *   flux_in_total, flux_out_total  inlet and outlet mass fluxes summed over
 *            every step since pflb_set_fields (a mass balance is mass(t) -
 *            mass(0) against flux_in_total - flux_out_total).
 * Allocates temporary device memory and synchronises the stream. */
typedef struct pflb_diagnostics {
  double drag[3];
  double heat;
  double mass;
  double outlet_Tm;
  double flux_in_total, flux_out_total;
  long long step;
} pflb_diagnostics;
int pflb_get_diagnostics(pflb_domain* d, pflb_diagnostics* out);

/* Size in bytes of a serialised state of this domain (header, scalars,
 * populations in their storage precision -- with FP16 storage the residuals
 * and then the FP32 cell moments (P, j) -- T, Y, Ts). */
int pflb_state_bytes(const pflb_domain* d, size_t* bytes);

/* Serialise the complete time-step state (checkpoint) into dst (host or
 * device memory of at least pflb_state_bytes).  Restoring it with
 * pflb_set_state and stepping reproduces an uninterrupted run bit for bit
 * (the reductions are deterministic).  Synchronises the stream. */
int pflb_get_state(pflb_domain* d, void* dst, size_t bytes, int where);

/* Restore a state written by pflb_get_state for a domain of the same shape,
 * precision and species count (checked against the header; PFLB_ERR_ARG on
 * mismatch).  Requires set_phase_field and set_fields to have run once.
 * Asynchronous on the domain's stream. */
int pflb_set_state(pflb_domain* d, const void* src, size_t bytes, int where);

/* Step kernels.  PFLB_KERNEL_TILED (default): 32 x 8 tiles staged in shared
 * memory with per-cell properties evaluated once (2.5-D z-marching in 3-D).
 * PFLB_KERNEL_TMA: persistent blocks, the next tile's fields and population
 * windows fetched by the tensor memory accelerator into a double-buffered
 * stage (2-D, FP32 compute, nx a multiple of 4 -- 8 with FP16 storage). */
#define PFLB_KERNEL_TILED 0
#define PFLB_KERNEL_TMA 1
/* PFLB_KERNEL_PERSISTENT(_32x16): 2-D only; one grid of resident blocks walks
 * the 32 x 8 (or 32 x 16, two rows per thread) tiles, handed out by an
 * atomic counter, so no second wave and no idle SMs at the end. */
#define PFLB_KERNEL_PERSISTENT 2
#define PFLB_KERNEL_PERSISTENT_32x16 3
/* PFLB_KERNEL_MARCH(_PREFETCH): 3-D only; a resident grid in which each block
 * marches a contiguous, equal share of the tile-planes along z (ring of three
 * staged planes holding only what neighbours read); _PREFETCH also issues the
 * next plane's pulls into registers before the current plane is updated,
 * periodic faces wrapped in the addresses. */
#define PFLB_KERNEL_MARCH 4
#define PFLB_KERNEL_MARCH_PREFETCH 5
#define PFLB_KERNELS 6

/* Select the step kernel of a domain (after pflb_set_fields).  The default is
 * PFLB_KERNEL_MARCH for 3-D domains with FP32 storage, PFLB_KERNEL_TILED
 * otherwise.  Returns PFLB_ERR_UNSUPPORTED if the kernel cannot run this
 * domain. */
int pflb_select_kernel(pflb_domain* d, int kernel);

/* Bound, in SM clock cycles, of the device-side waits of this domain's
 * kernels (the TMA kernel's wait for each staged tile).  Default 2^31, about
 * a second at 2 GHz; 0 makes each wait a single non-blocking probe.  A wait
 * that runs out latches PFLB_ERR_TIMEOUT and the block stops working on
 * tiles; before it exits it still waits (with the default bound) for the
 * copies it has issued, so no copy lands in a finished block's shared
 * memory.  A small bound is how the timeout path is exercised without a
 * hung GPU.  Errors: PFLB_ERR_ARG (cycles < 0 or > 2^40). */
int pflb_set_wait_limit(pflb_domain* d, long long cycles);

/* Time every step kernel that can run this domain over `steps` steps each
 * and keep the fastest (the domain's state is restored afterwards, so the
 * physics is unchanged).  *chosen receives the kernel, *us_per_step (may be
 * NULL) the time per step of each candidate in kernel order (PFLB_KERNELS
 * values, a negative value for a kernel that cannot run).  Synchronises the
 * stream. */
int pflb_autotune(pflb_domain* d, int steps, int* chosen, double* us_per_step);

/* ------------------------------------------------------------------------
 * Learned chemistry surrogate.  Not in the paper: an added pattern that
 * replaces the per-cell implicit chemistry by a small network where it is
 * trustworthy.  Network: 8 -> 64 -> 64 -> 64 -> 6, tanh hidden layers, BF16
 * weights and FP32 accumulation on tensor cores; inputs the normalised
 * (T, Y_1..Y_6, P0), outputs the normalised species change over one step.
 * Parameters: PFLB_MLP_PARAMS floats, W1 (8x64, input-major), b1, W2, b2,
 * W3, b3, W4 (64x6), b4 with y = x W + b.  All X / Y / out pointers below are
 * device pointers (row-major, 8 / 6 floats per row, normalised values).
 * ------------------------------------------------------------------------ */
#define PFLB_MLP_PARAMS 9286
typedef struct pflb_mlp pflb_mlp;

/* New network on `device`, work queued on `stream`; parameters zero. */
int pflb_mlp_create(int device, void* stream, pflb_mlp** out);
/* Load FP32 parameters from host memory (resets the Adam state); synchronises. */
int pflb_mlp_set_params(pflb_mlp* m, const float* theta);
/* Copy the FP32 master parameters to host memory; synchronises. */
int pflb_mlp_get_params(pflb_mlp* m, float* theta);
/* out[n][6] = network(X[n][8]) (asynchronous); X 16-byte aligned. */
int pflb_mlp_forward(pflb_mlp* m, const float* X, float* out, long long n);
/* Gradient of the mean squared error over the n rows (host grad[PFLB_MLP_PARAMS],
 * may be NULL) and the loss; synchronises. */
int pflb_mlp_gradient(pflb_mlp* m, const float* X, const float* Y, long long n, float* grad,
                      double* loss);
/* `steps` Adam steps (lr, beta 0.9 / 0.999, eps 1e-8) over consecutive mini-batches of
 * `batch` rows (wrapping); *last_loss = loss of the last mini-batch (may be NULL). */
int pflb_mlp_train(pflb_mlp* m, const float* X, const float* Y, long long n, int batch,
                   int steps, float lr, double* last_loss);
int pflb_mlp_destroy(pflb_mlp* m);

/* How a domain uses a trained network (PFLB_CHEM_SURROGATE). */
typedef struct pflb_surrogate {
  double x_mean[8], x_std[8];   /* input normalisation (std 0: feature ignored) */
  double y_mean[6], y_std[6];   /* output normalisation */
  double theta_s;               /* output scale temperature: dY = exp(-theta_s / T) *
                                   (y_mean + y_std * out); 0 for no scaling */
  double lo[8], hi[8];          /* training bounding box of the raw inputs */
  int n_elem;                   /* elements checked (<= 4) */
  double elem[4][PFLB_KMAX];    /* atoms of element e in species k */
  double elem_mass[4];          /* element molar masses (kg/mol) */
  double tol;                   /* element residual tolerance, e.g. 1e-6 */
  int engine;                   /* network kernel: PFLB_MLP_WARP_MMA (0, warp-level
                                   mma.sync, 32 cells per warp; the faster of the two on the
                                   bench's bed) or PFLB_MLP_TCGEN05 (1, tensor-memory
                                   accumulators, 128 cells per MMA); both use the network's
                                   FP32 parameters rounded to BF16 and FP32 accumulation */
  double skip_eps;              /* 0: the network runs on every tile of cells.  > 0: a
                                   tile of cells (32 for the warp engine, 128 for tcgen05)
                                   skips the network when none of its cells needs it, i.e.
                                   each is solid (phi_f < phi_min), outside [lo, hi] (the
                                   fallback takes it anyway) or at T <= T_skip, where the
                                   projected increment the network could give is bounded by
                                   skip_eps in every species: |out_k| <= sum_j |W_3[j][k]|
                                   + |b_3[k]| because |tanh| <= 1, so T_skip = theta_s /
                                   ln(|P|_inf max_k (|y_mean_k| + y_std_k max|out_k|) /
                                   skip_eps).  Such cold cells take a zero increment.
                                   Needs theta_s > 0; negative or NaN: PFLB_ERR_ARG */
} pflb_surrogate;

#define PFLB_MLP_WARP_MMA 0
#define PFLB_MLP_TCGEN05 1

/* Attach a trained network to a domain whose mechanism has chem_mode
 * PFLB_CHEM_SURROGATE and six species.  A cell uses the network when its
 * inputs are inside [lo, hi] and |sum_k elem[e][k] M_e / M_k dY_k| <= tol for
 * every element; the increment is then projected onto the element-conserving
 * subspace.  Other fluid cells take the backward-Euler Newton integrator (FP32
 * in FP32 domains, see PFLB_CHEM_SURROGATE).
 * The network must outlive the domain's use of it. */
int pflb_set_surrogate(pflb_domain* d, const pflb_mlp* m, const pflb_surrogate* s);

/* Chemistry increments over one step of the CURRENT state with the domain's
 * chemistry mode (implicit or surrogate): dst receives (K+1)*N values, dY_k
 * then dT, in dtype; synchronises.  The state is not advanced. */
int pflb_chem_increments(pflb_domain* d, void* dst, size_t bytes, int dtype, int where);

/* Surrogate counters since the mechanism was set: cells that fell back to
 * the integrator and cells the network evaluated.  Synchronises. */
int pflb_chem_stats(pflb_domain* d, double* fallback_cells, double* evaluated_cells);

/* ------------------------------------------------------------------------
 * Batched stepping.  Not in the paper: an added pattern for many independent
 * particle assemblies (2-D, no species).  One persistent kernel per step
 * walks the tiles of every domain of the batch; the steps are replayed from
 * a captured CUDA graph (two steps per graph).  Domains keep their own
 * arrays and stay usable through the single-domain calls; a batch step
 * leaves every domain's scalars current (no deferred reduction).
 * ------------------------------------------------------------------------ */
typedef struct pflb_batch pflb_batch;
#define PFLB_BATCH_TILE_32x8 0
#define PFLB_BATCH_TILE_32x16 1 /* two rows per thread */
#define PFLB_BATCH_TILE_64x4 2
#define PFLB_BATCH_TILES 3

/* A batch over n domains (all 2-D, K = 0, same precision and device, fields
 * set).  The domains must outlive the batch.  PFLB_ERR_UNSUPPORTED when a
 * domain cannot be batched. */
int pflb_create_batch(pflb_domain** domains, int n, pflb_batch** out);
/* Advance every domain of the batch by nsteps (asynchronous; ordered after
 * the work already queued on the domains' streams, and their streams wait
 * for it). */
int pflb_batch_step(pflb_batch* b, int nsteps);
/* Tile shape (PFLB_BATCH_TILE_*) and resident blocks per SM (0: the most
 * the kernel allows) of the persistent grid. */
int pflb_batch_set_config(pflb_batch* b, int tile, int blocks_per_sm);
int pflb_batch_get_config(const pflb_batch* b, int* tile, int* blocks_per_sm, int* grid);
/* Time every (tile shape, blocks per SM) pair over `steps` batch steps,
 * keep the fastest, and put every domain back in its state before the
 * call.  us_per_step (may be NULL) receives PFLB_BATCH_TILES x 8 values,
 * [tile][blocks_per_sm - 1], 0 where not run.  Synchronises. */
int pflb_batch_autotune(pflb_batch* b, int steps, int* tile, int* blocks_per_sm,
                        double* us_per_step);
int pflb_batch_destroy(pflb_batch* b);
const char* pflb_batch_last_error(const pflb_batch* b);

/* Device diagnostic (not in the paper): the measured FP64 FMA rate of
 * `device` in TFLOP/s (2 flops per FMA), the ceiling of the FP64 step and of
 * the Newton chemistry.  Allocates 8 bytes, synchronises the device. */
int pflb_probe_fp64_fma(int device, double* tflops);

/* Largest lattice (cells) that pflb_step_noalloc accepts. */
#define PFLB_NOALLOC_MAX_CELLS (1 << 22)

/* One time step on caller-owned device arrays, allocating nothing.
 *
 * For callers that cannot allocate device memory: plug-ins whose host
 * framework owns all device memory through its own pool, and loops that
 * forbid allocator calls after start-up (cudaMalloc / cudaFree can
 * synchronise the whole device and take unbounded time).  The paper has no
 * counterpart; it is the same fused step as pflb_step.  The caller owns and
 * passes every state array (layout as in pflb_get_fields, in the compute
 * precision: double for PFLB_FP64, float for PFLB_FP32): phi (N),
 * g_in/g_out (Q*N), T_in/T_out (N), Y_in/Y_out (K*N, or NULL when K = 0),
 * Ts_in/Ts_out (N, or NULL unless desc->Ts_field).  `mech` may be NULL for
 * K = 0.  `scalars` (host) carries P0 (> 0), P0_prev, mass, step and status
 * in, and returns the updated values (P0 of the next step, I, fluxes) after
 * the step; the call copies the scalars through host memory and
 * synchronises desc->stream before it returns.
 *
 * The description and mechanism pass the same checks as pflb_create_domain
 * and pflb_set_mechanism (PFLB_ERR_ARG, PFLB_ERR_UNSUPPORTED,
 * PFLB_ERR_UNSTABLE); on any error pflb_last_error(NULL) names the reason.
 *
 * The reduction scratch (per-block partials, arrival counter, scalar block)
 * is a fixed device array inside the library, sized for at most
 * PFLB_NOALLOC_MAX_CELLS cells (about 1 MB); every GPU that loads the
 * library holds it until the process exits.  Larger lattices return
 * PFLB_ERR_ARG.  Supported: D2Q9, K = 0 or 5, PFLB_FP64 or PFLB_FP32 (else
 * PFLB_ERR_UNSUPPORTED).  The first call on a device looks up the array's
 * device address; make that first call before any stream capture.  All calls
 * share the one array: calls that overlap on the GPU (other streams, other
 * host threads) race and corrupt each other's reduction -- serialise them. */
int pflb_step_noalloc(const pflb_domain_desc* desc, const pflb_mechanism* mech,
                      const void* phi, const void* g_in, void* g_out,
                      const void* T_in, void* T_out, const void* Y_in, void* Y_out,
                      const void* Ts_in, void* Ts_out, pflb_scalars* scalars);

/* Number of populations Q and the lattice velocities (3*Q ints) and
 * weights (Q doubles) in the library's storage order. */
int pflb_lattice(int dim, int* c_out, double* w_out);

/* Release every device allocation of the domain. */
int pflb_destroy(pflb_domain* d);

/* Last error message of this domain (or of the last failed create when d is
 * NULL).  The string lives until the next call on the same handle. */
const char* pflb_last_error(const pflb_domain* d);

#ifdef __cplusplus
}
#endif
#endif /* PFLB_H */
