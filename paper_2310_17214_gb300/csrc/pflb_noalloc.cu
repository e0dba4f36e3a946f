// pflb_noalloc.cu -- pflb_step_noalloc: one time step on caller-owned device
// arrays without any device allocation.
//
// Some callers cannot call cudaMalloc at all: plug-ins living under a host
// framework that owns every device allocation through its own pool, or loops
// that forbid allocator calls after start-up (an allocation or free can
// synchronise the device and take unbounded time).  They own the state
// arrays and pass them in; the only memory this entry point needs
// besides them -- the per-block partial sums of the P0 reduction, the
// arrival counter of the finishing block and the scalar block -- lives in the
// fixed file-scope device array below, sized for at most
// PFLB_NOALLOC_MAX_CELLS cells.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>

#include "../../include/pflb.h"
#include "pflb_launch.cuh"
#include "pflb_validate.cuh"

using namespace pflb;

namespace {

constexpr int kMaxBlocks = PFLB_NOALLOC_MAX_CELLS / BLOCK;
constexpr size_t kPartialDoubles = (size_t)kMaxBlocks * 4 * 2;

// Layout: [DevScalars][counter + pad to 64 bytes][partials: 2 x kMaxBlocks x 4 doubles].
// Every GPU that loads the library holds this array until the process exits.
constexpr size_t kScalarBytes = (sizeof(DevScalars) + 63) / 64 * 64;
constexpr size_t kScratchBytes = kScalarBytes + 64 + kPartialDoubles * sizeof(double);
static __device__ __align__(256) unsigned char noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* scratch_ptr[kMaxDevices] = {nullptr};

// the reason goes where pflb_last_error(NULL) reads it (this host thread)
int err(int code, const std::string& msg) {
  set_global_error(msg);
  return code;
}

}  // namespace

extern "C" int pflb_step_noalloc(const pflb_domain_desc* desc, const pflb_mechanism* mech,
                                 const void* phi, const void* g_in, void* g_out,
                                 const void* T_in, void* T_out, const void* Y_in, void* Y_out,
                                 const void* Ts_in, void* Ts_out, pflb_scalars* scalars) {
  if (!desc || !phi || !g_in || !g_out || !T_in || !T_out || !scalars)
    return err(PFLB_ERR_ARG, "NULL argument");
  const pflb_domain_desc& D = *desc;
  const int K = mech ? mech->K : 0;
  {
    std::string why;
    int rc = validate_desc(D, why);
    if (rc == PFLB_OK && mech) rc = validate_mech(*mech, why);
    if (rc == PFLB_OK) rc = check_stability(D, mech, why);
    if (rc != PFLB_OK) return err(rc, why);
  }
  if (D.dim != 2) return err(PFLB_ERR_UNSUPPORTED, "pflb_step_noalloc supports D2Q9 only");
  if (D.u_s[0] != 0.0 || D.u_s[1] != 0.0 || D.u_s[2] != 0.0)
    return err(PFLB_ERR_UNSUPPORTED, "a moving solid needs a domain (pflb_create_domain)");
  if (D.outlet_nscbc)
    return err(PFLB_ERR_UNSUPPORTED, "the characteristic outlet needs a domain (pflb_create_domain)");
  if (mech && mech->inlet_feedback)
    return err(PFLB_ERR_UNSUPPORTED, "the inlet feedback needs a domain (pflb_create_domain)");
  if (K != 0 && K != 5) return err(PFLB_ERR_UNSUPPORTED, "pflb_step_noalloc supports K = 0 or 5");
  if (D.precision != PFLB_FP64 && D.precision != PFLB_FP32)
    return err(PFLB_ERR_UNSUPPORTED, "pflb_step_noalloc supports FP64 and FP32");
  if (K > 0 && (!Y_in || !Y_out)) return err(PFLB_ERR_ARG, "Y arrays are required when K > 0");
  if (mech && mech->chem_mode > PFLB_CHEM_EXPLICIT)
    return err(PFLB_ERR_UNSUPPORTED, "pflb_step_noalloc supports explicit chemistry only");
  if (D.Ts_field && (!Ts_in || !Ts_out)) return err(PFLB_ERR_ARG, "Ts arrays are required");
  if (!(scalars->P0 > 0) || !std::isfinite(scalars->P0) || !std::isfinite(scalars->P0_prev))
    return err(PFLB_ERR_ARG, "scalars->P0 must be positive and P0, P0_prev finite");
  const long long N = (long long)D.nx * D.ny;
  if (N > PFLB_NOALLOC_MAX_CELLS)
    return err(PFLB_ERR_ARG, "lattice larger than PFLB_NOALLOC_MAX_CELLS cells");
  if (D.device < 0 || D.device >= kMaxDevices) return err(PFLB_ERR_ARG, "bad device ordinal");

  if (cudaSetDevice(D.device) != cudaSuccess) return err(PFLB_ERR_CUDA, "cudaSetDevice failed");
  // once per device, with that device current: the device address of the
  // scratch array (its host-side name is only a stand-in)
  if (!scratch_ptr[D.device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, noalloc_scratch);
    if (e != cudaSuccess || !p) return err(PFLB_ERR_CUDA, "cudaGetSymbolAddress failed");
    scratch_ptr[D.device] = p;
  }
  unsigned char* base = static_cast<unsigned char*>(scratch_ptr[D.device]);
  cudaStream_t st = static_cast<cudaStream_t>(D.stream);

  DevScalars h;
  std::memset(&h, 0, sizeof(h));
  h.P0 = scalars->P0;
  h.P0_prev = scalars->P0_prev;
  h.mass = scalars->mass;
  h.step = scalars->step;
  h.status = scalars->status;
  // per-step constants the cells read (the finishing block refreshes them)
  h.dlnP0 = (h.P0 - h.P0_prev) / h.P0;
  h.dP0r = (h.P0 - h.P0_prev) / D.rho_ref;
  h.P0_f = float(h.P0);
  h.dlnP0_f = float(h.dlnP0);
  h.dP0r_f = float(h.dP0r);
  if (cudaMemcpyAsync(base, &h, sizeof(h), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(base + kScalarBytes, 0, 64, st) != cudaSuccess)
    return err(PFLB_ERR_CUDA, "scratch set-up copy failed");

  Buffers B;
  std::memset(&B, 0, sizeof(B));
  B.g[0] = const_cast<void*>(g_in);
  B.g[1] = g_out;
  B.T[0] = const_cast<void*>(T_in);
  B.T[1] = T_out;
  B.Y[0] = const_cast<void*>(Y_in);
  B.Y[1] = Y_out;
  B.Ts[0] = const_cast<void*>(Ts_in);
  B.Ts[1] = Ts_out;
  B.phi = const_cast<void*>(phi);
  B.scal = reinterpret_cast<DevScalars*>(base);
  B.counter = reinterpret_cast<unsigned*>(base + kScalarBytes);
  B.partials = reinterpret_cast<double*>(base + kScalarBytes + 64);
  B.N = (int)N;
  B.slots = kMaxBlocks;
  B.pending = 0;

  pflb_mechanism none;
  std::memset(&none, 0, sizeof(none));
  const pflb_mechanism& M = mech ? *mech : none;
  int cur = 0;
  cudaError_t e = cudaSuccess;
  long long nblk = 0;
  auto run = [&](auto& L) {
    nblk = L.step_blocks();
    if (nblk <= kMaxBlocks) {
      e = L.step(B, cur, 1, st);
      if (e == cudaSuccess) e = L.finalize(B, st);
    }
  };
  if (D.precision == PFLB_FP64) {
    if (K == 0) { LauncherImpl<2, 0, MODE_FP64> L(D, M); run(L); }
    else { LauncherImpl<2, 5, MODE_FP64> L(D, M); run(L); }
  } else {
    if (K == 0) { LauncherImpl<2, 0, MODE_FP32> L(D, M); run(L); }
    else { LauncherImpl<2, 5, MODE_FP32> L(D, M); run(L); }
  }
  if (nblk > kMaxBlocks) return err(PFLB_ERR_ARG, "tile count exceeds the scratch array");
  if (e != cudaSuccess) return err(PFLB_ERR_CUDA, cudaGetErrorString(e));
  if (cudaMemcpyAsync(&h, base, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return err(PFLB_ERR_CUDA, "scalar read-back failed");
  scalars->P0 = h.P0;
  scalars->P0_prev = h.P0_prev;
  scalars->mass = h.mass;
  scalars->I = h.I;
  scalars->flux_in = h.flux_in;
  scalars->flux_out = h.flux_out;
  scalars->step = h.step;
  scalars->status = h.status;
  scalars->u_in = D.u_in;  // no inlet feedback on this path
  scalars->fuel = 0.0;
  scalars->outlet_pb = 0.0;
  if (h.status != 0) return err(h.status, status_message(h.status));
  return PFLB_OK;
}
