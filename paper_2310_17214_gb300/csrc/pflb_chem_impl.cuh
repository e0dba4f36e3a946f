// pflb_chem_impl.cuh -- definition of chem_pass_launch (see pflb_chem.cuh);
// included by the two translation units that instantiate it.
#pragma once

#include <algorithm>

#include "pflb_chem.cuh"
#include "pflb_surrogate_tc.cuh"

namespace pflb {

template <int K, class Real>
cudaError_t chem_pass_launch(const Params<Real, K>& P, const State<Real, Real>& S, Real* src,
                             const SurrArgs* surr, int* fb_idx, unsigned* fb_count,
                             double* stats, double* out, cudaStream_t st) {
  const int blocks = (P.N + BLOCK - 1) / BLOCK;
  if (P.chem == 2) {
    chem_implicit_kernel<K, Real, Real><<<blocks, BLOCK, 0, st>>>(P, S, src);
  } else if (P.chem == 3) {
    if constexpr (K == 6) {
      if (!surr || !fb_idx) return cudaErrorInvalidValue;
      SurrArgs a = *surr;
      a.fb_idx = fb_idx;
      a.fb_count = fb_count;
      a.stats = stats;
      cudaError_t e = cudaMemsetAsync(fb_count, 0, sizeof(unsigned), st);
      if (e != cudaSuccess) return e;
      int dev = 0, sms = 0;
      e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
      if (a.engine == 1) {
        // tcgen05 network: 128 cells per tile, persistent grid of kTcBlocksPerSm blocks per SM
        constexpr size_t smem = tc_smem_bytes();
        auto kern = chem_surrogate_tc_kernel<K, Real, Real>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        // all of the SM's unified memory as shared memory, so that the blocks
        // of the resident wave fit side by side
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        const int nb = (int)std::min<long long>(((long long)P.N + tc::M - 1) / tc::M,
                                                (long long)sms * kTcBlocksPerSm);
        kern<<<nb, tc::M, smem, st>>>(P, S, src, a, kDefaultWaitCycles);
      } else {
        // warp-level network; one resident wave: each block loads the network once
        auto kern = chem_surrogate_kernel<K, Real, Real>;
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, 0);
        if (e != cudaSuccess) return e;
        occ = std::max(1, occ);
        const int nb = (int)std::min<long long>(((long long)P.N + 255) / 256, (long long)sms * occ);
        kern<<<nb, 256, 0, st>>>(P, S, src, a);
      }
      const int fb_blocks = (int)std::min<long long>(
          ((long long)P.N + FALLBACK_BLOCK - 1) / FALLBACK_BLOCK, (long long)sms * 16);
      chem_fallback_kernel<K, Real, Real><<<fb_blocks, FALLBACK_BLOCK, 0, st>>>(P, S, src,
                                                                                fb_idx, fb_count);
    } else {
      return cudaErrorNotSupported;
    }
  } else {
    return cudaErrorInvalidValue;
  }
  if (out)
    src_to_increments_kernel<K, Real, Real><<<blocks, BLOCK, 0, st>>>(P, S, src, out);
  return cudaGetLastError();
}

}  // namespace pflb
