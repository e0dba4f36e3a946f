// pflb_step3d.cuh -- persistent z-marching fused step for 3-D lattices.
//
// The same per-cell update as step_kernel (cell_update), organised for the
// D3Q19 bed:
//   - a resident grid (blocks per SM x SMs) in which block b owns the
//     contiguous run [b T / G, (b + 1) T / G) of the T = tiles x nz
//     tile-planes, z innermost: every block gets the same number of planes
//     (+-1), so no second partial wave leaves SMs idle, and a run restages
//     its halo planes only where it crosses into the next column of tiles;
//   - a ring of three staged planes holding only what neighbours read (T,
//     phi_s, rho, phi_f lambda, Ts, phi_f rho f_D, Y_k and, with FP16
//     storage, the cell moments); the own-cell properties mu and f_D are
//     evaluated in the cell;
//   - optionally (PRE) the 19 pulls of the next plane issued into registers
//     before the current plane is updated, with periodic faces wrapped in
//     the addresses, so only cells on non-periodic faces take the boundary
//     path of the pull.
// The block sums of the whole run are published once into slot blockIdx.x.
#pragma once

#include "pflb_kernels.cuh"

namespace pflb {

// staged fields of the march
enum { G_T = 0, G_PHI, G_RHO, G_KT, G_TS, G_RF, G_Y0 };

__host__ __device__ constexpr int march_field(int f) {
  return f == F_T ? G_T : f == F_PHI ? G_PHI : f == F_RHO ? G_RHO : f == F_KT ? G_KT
       : f == F_TS ? G_TS : f == F_RF ? G_RF : G_Y0 + (f - F_Y0);
}

template <int K, class Store>
__host__ __device__ constexpr int march_nf() { return G_Y0 + K + n_mom<3, Store>(); }

template <int K, class Real, class Store>
constexpr size_t march_smem_bytes() {
  return sizeof(Real) * (3 * march_nf<K, Store>() * Tile<3>::HP + Lattice<3>::Q * BLOCK);
}

// Accessor of cell_update over the march's staged planes; mu and f_D are the
// cell's own values.
template <class Real, int K, bool PRE>
struct MarchAcc {
  using TL = Tile<3>;
  static constexpr int HP = TL::HP;
  static constexpr bool has_pops = PRE;
  static constexpr bool kStash = true;  // pulled populations wait in shared memory
  const Real* __restrict__ cen;
  const Real* __restrict__ zm;
  const Real* __restrict__ zp;
  int h;
  Real mu, fD;
  const Real* pre;
  bool pv;  // pre holds this cell's populations
  Real* st; // stash [Q][BLOCK]
  __device__ __forceinline__ Real c(int f) const {
    if (f == F_MU) return mu;
    if (f == F_FD) return fD;
    return cen[march_field(f) * HP + h];
  }
  __device__ __forceinline__ Real n(int f, int a, int s) const {
    const int g = march_field(f) * HP;
    if (a == 0) return cen[g + h + s];
    if (a == 1) return cen[g + h + s * TL::HX];
    return (s < 0 ? zm : zp)[g + h];
  }
  template <class S_>
  __device__ __forceinline__ Real pop(int i, Real) const { return PRE ? pre[i] : Real(0); }
  __device__ __forceinline__ Real mom(int a, int, int dx, int dy, int dz) const {
    const Real* p = dz < 0 ? zm : (dz > 0 ? zp : cen);
    return p[(G_Y0 + K + a) * HP + h + dx + dy * TL::HX];
  }
};

// Stage plane z (may be -1 or nz: ghost plane) of the tile at (x0, y0) with
// its xy halo into `pl` ([NF][HP]), with the ghost rules of stage_plane.
template <class Real, class Store, int K>
__device__ __forceinline__ void march_stage(const Params<Real, K>& P, const State<Real, Store>& S,
                                            Real* __restrict__ pl, int x0, int y0, int z,
                                            Real P0) {
  using T_ = Tile<3>;
  constexpr int HP = T_::HP;
  constexpr int NM = n_mom<3, Store>();
  const bool inner = x0 >= 1 && y0 >= 1 && x0 + T_::TX < P.nx && y0 + T_::TY < P.ny && z >= 0 &&
                     z < P.nz;
  for (int h = threadIdx.x; h < HP; h += blockDim.x) {
    const int hy = h / T_::HX, hx = h - hy * T_::HX;
    int q[3] = {x0 - 1 + hx, y0 - 1 + hy, z};
    int ghost_face = -1, nout = 0;
    if (!inner) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int n = a == 0 ? P.nx : (a == 1 ? P.ny : P.nz);
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
    pl[G_T * HP + h] = T;
    pl[G_PHI * HP + h] = phis;
    pl[G_RHO * HP + h] = rho;
    pl[G_KT * HP + h] = phif * lam;
    pl[G_TS * HP + h] = Ts;
    pl[G_RF * HP + h] = phif * rho * fD;
#pragma unroll
    for (int k = 0; k < K; ++k) pl[(G_Y0 + k) * HP + h] = Y[k];
    if constexpr (NM > 0) {
#pragma unroll
      for (int a = 0; a < NM; ++a)
        pl[(G_Y0 + K + a) * HP + h] = __ldg(S.M_in + (size_t)a * P.N + c);
    }
  }
}

// The 19 pulls of cell (x, y, z) with periodic faces wrapped; false (and
// nothing loaded) for a cell on a non-periodic face, whose pull needs the
// boundary rules.
template <class Real, class Store, int K>
__device__ __forceinline__ bool march_prefetch(const Params<Real, K>& P,
                                               const State<Real, Store>& S, int x, int y, int z,
                                               Real* __restrict__ out) {
  using L = Lattice<3>;
  const int n[3] = {P.nx, P.ny, P.nz};
  const int xyz[3] = {x, y, z};
  int v[3][3];  // v[a][1 + s]: coordinate a of the neighbour at offset s, wrapped
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int lo = xyz[a] - 1, hi = xyz[a] + 1;
    if ((lo < 0 && P.bc[2 * a] != BC_PERIODIC) || (hi >= n[a] && P.bc[2 * a + 1] != BC_PERIODIC))
      return false;
    v[a][0] = lo < 0 ? lo + n[a] : lo;
    v[a][1] = xyz[a];
    v[a][2] = hi >= n[a] ? hi - n[a] : hi;
  }
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const int src =
        v[0][1 - L::c(i, 0)] + P.nx * (v[1][1 - L::c(i, 1)] + P.ny * v[2][1 - L::c(i, 2)]);
    out[i] = Codec<Store, Real>::raw(S.g_in + (size_t)i * P.N + src);
  }
  return true;
}

// Resident blocks per SM asked of the register allocator: FP32 storage fits
// 80 registers (3 blocks); the FP16 decode needs more (2 blocks, no spills).
template <class Real, class Store, bool PRE> struct MarchBlocks {
  static constexpr int value =
      sizeof(Real) == 8 ? 1 : ((PRE || IsHalf<Store>::value) ? 2 : 3);
};

template <int K, class Real, class Store, bool PRE>
__global__ void __launch_bounds__(BLOCK, (MarchBlocks<Real, Store, PRE>::value))
step3d_march_kernel(const Params<Real, K> P, const State<Real, Store> S, int p0_closed,
                    const double* __restrict__ prev_partials, unsigned prev_nb) {
  using T_ = Tile<3>;
  using L = Lattice<3>;
  constexpr int HP = T_::HP;
  constexpr int NF = march_nf<K, Store>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* planes = reinterpret_cast<Real*>(smem_raw);  // [3][NF][HP]
  __shared__ double red_sh[96];

  if (prev_partials && blockIdx.x == 0 && threadIdx.x < 32)
    combine_partials(prev_partials, prev_nb, S.scal, 0, false, 0.0, P.eos_c, P.inv_rho_ref);

  const Real P0 = scal_P0<Real>(S.scal);
  const Real dlnP0 = scal_dlnP0<Real>(S.scal);
  const Real dP0r = scal_dP0r<Real>(S.scal);

  const int tiles_x = (P.nx + T_::TX - 1) / T_::TX;
  const int tiles = tiles_x * ((P.ny + T_::TY - 1) / T_::TY);
  const long long total = (long long)tiles * P.nz;
  const long long g_end = total * (blockIdx.x + 1) / gridDim.x;
  const int tx = threadIdx.x % T_::TX, ty = threadIdx.x / T_::TX;
  const int h = (ty + 1) * T_::HX + (tx + 1);

  Real accI = 0, accIn = 0, accOut = 0;
  bool flux_block = false;
  for (long long gi = total * blockIdx.x / gridDim.x; gi < g_end;) {
    const int tile = (int)(gi / P.nz);
    const int z_begin = (int)(gi - (long long)tile * P.nz);
    const int z_end = (int)min((long long)P.nz, z_begin + (g_end - gi));
    gi += z_end - z_begin;
    const int x0 = (tile % tiles_x) * T_::TX, y0 = (tile / tiles_x) * T_::TY;
    const int x = x0 + tx, y = y0 + ty;
    const bool in_xy = x < P.nx && y < P.ny;
    flux_block = flux_block || (x0 == 0 && P.bc[0] == BC_INLET) ||
                 (x0 + T_::TX >= P.nx && P.bc[1] == BC_OUTLET);

    __syncthreads();  // the previous column is done with the planes
    march_stage<Real, Store, K>(P, S, planes + ((z_begin + 2) % 3) * NF * HP, x0, y0,
                                z_begin - 1, P0);
    march_stage<Real, Store, K>(P, S, planes + (z_begin % 3) * NF * HP, x0, y0, z_begin, P0);
    Real pre[L::Q], nxt[L::Q];
    bool have = false, have_nxt = false;
    if constexpr (PRE) {
      if (in_xy) have = march_prefetch<Real, Store, K>(P, S, x, y, z_begin, pre);
    }
    for (int z = z_begin; z < z_end; ++z) {
      march_stage<Real, Store, K>(P, S, planes + ((z + 1) % 3) * NF * HP, x0, y0, z + 1, P0);
      if constexpr (PRE) {
        have_nxt = in_xy && z + 1 < z_end &&
                   march_prefetch<Real, Store, K>(P, S, x, y, z + 1, nxt);
      }
      __syncthreads();
      if (in_xy) {
        const int c = x + P.nx * (y + P.ny * z);
        const int xyz[3] = {x, y, z};
        const Real* cen = planes + (z % 3) * NF * HP;
        const Real T0 = cen[G_T * HP + h];
        Real fD = Real(1);
        if constexpr (K > 0) {
          if (P.D_Tdep) fD = fpow(T0 * P.inv_DTref, P.D_exp);
        }
        Real mu0 = viscosity(P, T0);
        if constexpr (K > 0) {
          if (P.mix) {  // mixture-averaged viscosity of the cell's own composition
            Real Yo[K], lam0;
#pragma unroll
            for (int k = 0; k < K; ++k) Yo[k] = cen[(G_Y0 + k) * HP + h];
            transport(P, T0, Yo, mixture_invMw(P, Yo), mixture_cp(P, Yo), mu0, lam0);
          }
        }
        const MarchAcc<Real, K, PRE> A{cen, planes + ((z + 2) % 3) * NF * HP,
                                       planes + ((z + 1) % 3) * NF * HP, h, mu0, fD,
                                       pre, PRE && have, planes + 3 * NF * HP};
        // a cell that prefetched nothing lies on a non-periodic face: the
        // update pulls with the boundary rules there
        Real fi, fo;
        accI += cell_update<3, K, Real, Store>(P, S, A, c, xyz, P0, dlnP0, dP0r, fi, fo);
        accIn += fi;
        accOut += fo;
      }
      __syncthreads();
      if constexpr (PRE) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) pre[i] = nxt[i];
        have = have_nxt;
      }
    }
  }
  double sI, sIn, sOut;
  block_sum3<Real>(accI, accIn, accOut, flux_block, red_sh, sI, sIn, sOut);
  publish_partials(sI, sIn, sOut, S.partials, S.counter, S.scal, p0_closed, false, 0.0, P.eos_c,
                   P.inv_rho_ref);
}

}  // namespace pflb
