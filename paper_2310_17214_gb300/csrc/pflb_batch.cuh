// pflb_batch.cuh -- many 2-D domains advanced by one persistent kernel.
//
// Every domain keeps its own arrays; the batch holds a device work list with
// one entry per domain (its lattice-unit parameters, the two ping-pong views
// of its state, its P0 mode) and, per tile shape, the prefix sums of the
// domains' tile counts.  A launch is a grid-stride loop over the global tile
// index: a block finds the tile's domain by binary search, copies that
// domain's parameters into shared memory when it changes domain, and runs the
// same per-tile code as the single-domain step.  Tiles are handed out by an
// atomic counter (one per launch parity; each launch clears the other one
// for the next launch), so blocks that draw cheap tiles take more of them
// and no SM idles at the end.  Each domain's reduction
// slots are its tile indices, and the last tile of a domain to finish
// combines them at once, so a batch step leaves no deferred work behind and
// every domain's P0 is current for the next launch.
#pragma once

#include "pflb_kernels.cuh"

namespace pflb {

template <int K, class Real, class Store>
struct BatchDom {
  Params<Real, K> P;
  State<Real, Store> S[2];  // S[q]: input state in ping-pong buffer q
  int p0_closed;
  int cur0;                 // buffer holding the input at even batch steps
};

// Tile shapes the batch can run: 32 x 8, 32 x 16 (two rows per thread),
// 64 x 4.
constexpr int BATCH_SHAPES = 3;
template <int CFG> struct BatchShape;
template <> struct BatchShape<0> { using T = Tile<2, 32, 1>; };
template <> struct BatchShape<1> { using T = Tile<2, 32, 2>; };
template <> struct BatchShape<2> { using T = Tile<2, 64, 1>; };

__host__ __device__ constexpr int batch_tx(int cfg) { return cfg == 2 ? 64 : 32; }
__host__ __device__ constexpr int batch_ty(int cfg) { return cfg == 0 ? 8 : (cfg == 1 ? 16 : 4); }

template <class Real, class Store, class T_> struct BatchMinBlocks {
  static constexpr int value = sizeof(Real) == 8 ? 2 : (T_::RPT > 1 ? 3 : 4);
};

template <int K, class Real, class Store, class T_>
__global__ void __launch_bounds__(BLOCK, (BatchMinBlocks<Real, Store, T_>::value))
batch_step_kernel(const BatchDom<K, Real, Store>* __restrict__ doms,
                  const int* __restrict__ tile_begin, int ndom, int flip,
                  unsigned* __restrict__ tile_ctr) {
  using PL = Plane<Real, K, T_::HP, n_mom<2, Store>()>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PL* planes = reinterpret_cast<PL*>(smem_raw);
  __shared__ double red_sh[96];
  __shared__ Params<Real, K> Psh;
  __shared__ State<Real, Store> Ssh;
  __shared__ int p0c_sh;
  __shared__ int next_sh[2];

  const int total = tile_begin[ndom];
  unsigned* ctr = tile_ctr + flip;
  if (threadIdx.x == 0) {
    if (blockIdx.x == 0) tile_ctr[flip ^ 1] = 0u;  // the next launch's counter
    next_sh[0] = (int)atomicAdd(ctr, 1u);
  }
  __syncthreads();
  int cur_dom = -1, par = 0;
  for (int t = next_sh[0]; t < total; t = next_sh[par]) {
    // domain of tile t: the last d with tile_begin[d] <= t
    int lo = 0, hi = ndom - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(tile_begin + mid) <= t) lo = mid;
      else hi = mid - 1;
    }
    if (lo != cur_dom) {
      __syncthreads();  // the previous tile is done with the shared copies
      const BatchDom<K, Real, Store>& D = doms[lo];
      constexpr int PW = sizeof(Params<Real, K>) / 4;
      const uint32_t* src = reinterpret_cast<const uint32_t*>(&D.P);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&Psh);
      for (int i = threadIdx.x; i < PW; i += blockDim.x) dst[i] = __ldg(src + i);
      if (threadIdx.x == 0) {
        Ssh = D.S[D.cur0 ^ flip];
        p0c_sh = D.p0_closed;
      }
      __syncthreads();
      cur_dom = lo;
    }
    // draw the next tile now; the tile's staging barrier publishes it
    par ^= 1;
    if (threadIdx.x == 0) next_sh[par] = (int)atomicAdd(ctr, 1u);
    const int lt = t - tile_begin[lo];
    const int nbx = (Psh.nx + T_::TX - 1) / T_::TX;
    double sI, sIn, sOut;
    step_tile<2, K, Real, Store, T_>(Psh, Ssh, lt % nbx, lt / nbx, 0, planes, red_sh, sI, sIn,
                                     sOut);
    const unsigned nb = (unsigned)(tile_begin[lo + 1] - tile_begin[lo]);
    publish_partials_at(sI, sIn, sOut, Ssh.partials, Ssh.counter, Ssh.scal, p0c_sh, false, 0.0,
                        Psh.eos_c, Psh.inv_rho_ref, (unsigned)lt, nb, true);
  }
}

template <int K, class Real, class Store, class T_>
constexpr size_t batch_smem_bytes() {
  return sizeof(Plane<Real, K, T_::HP, n_mom<2, Store>()>);
}

}  // namespace pflb
