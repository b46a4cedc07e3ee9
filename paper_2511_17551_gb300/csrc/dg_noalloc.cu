// Allocation-free variant of the FP64 Navier-Stokes right-hand side.
//
// Who needs it: code that runs where device allocation is not allowed -- a host
// framework that owns all device memory and hands a library only its inputs and
// outputs (custom-operator and plugin interfaces work this way), or a real-time
// loop that must not call cudaMalloc/cudaFree because they synchronise the device
// and can fail at run time.  dg_init_mesh allocates the context's buffers, so such
// callers cannot use dg_rhs; this entry point takes every input and output from
// the caller and keeps its one piece of scratch (the BR1 gradients of
// (v, p/rho), 12 doubles per node, plus a status word) in a file-scope device
// array that exists once per GPU for the life of the process.
#include <cuda_runtime.h>
#include <string.h>

#include "../../include/dg.h"
#include "dg_internal.h"

namespace {

// [0, 256): device status word; [256, end): gradients [K][3][4][np] FP64
static __device__ __align__(256) unsigned char g_noalloc_scratch[DG_NOALLOC_SCRATCH_BYTES];

struct NoallocSetup {
  int done;
  unsigned char* base;  // device address of g_noalloc_scratch on that device
};
NoallocSetup g_setup[64];

}  // namespace

extern "C" dg_status dg_rhs_ns_noalloc(int N, int64_t K, const int32_t* nbr, const double* Ja,
                                       const double* invJ, double gamma, double mu, double Pr,
                                       int volume_flux, int surface_flux, const double* u,
                                       double* rhs, void* stream) {
  if (!(N == 2 || N == 3 || N == 4 || N == 7) || K < 1 || !nbr || !Ja || !invJ || !u || !rhs ||
      u == rhs)
    return DG_EINVAL;
  if (!(gamma > 1.0) || !(mu > 0.0) || !(Pr > 0.0)) return DG_EINVAL;
  if (volume_flux < 0 || volume_flux > DG_VF_MORINISHI || surface_flux < 0 || surface_flux > DG_SF_HLL) return DG_EINVAL;
  const int np = (N + 1) * (N + 1) * (N + 1);
  const double need = 256.0 + (double)K * np * 12.0 * sizeof(double);
  if (need > (double)DG_NOALLOC_SCRATCH_BYTES) return DG_EINVAL;  // beyond the static scratch
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DG_ECUDA;
  if (!g_setup[dev].done) {
    // one-time set-up on this device (the calling thread's current device)
    void* p = NULL;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == NULL) return DG_ECUDA;
    if (dg_f64_upload_basis() != cudaSuccess) return DG_ECUDA;
    g_setup[dev].base = (unsigned char*)p;
    g_setup[dev].done = 1;
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* status = (unsigned long long*)g_setup[dev].base;
  double* grad = (double*)(g_setup[dev].base + 256);
  if (cudaMemsetAsync(status, 0, sizeof(unsigned long long), st) != cudaSuccess) return DG_ECUDA;

  DgArgs a;
  memset(&a, 0, sizeof(a));
  a.K = K;
  a.dim = 3;
  a.N = N;
  a.nsp = 1;
  a.nv = 5;
  a.np = np;
  a.vf = volume_flux;
  a.sf = surface_flux;
  a.mode = 0;
  a.ns = 1;
  a.gamma = gamma;
  a.mu = mu;
  a.kappa_fac = mu * gamma / ((gamma - 1.0) * Pr);
  a.visc_coef = gamma * mu / Pr;
  a.u = u;
  a.out = rhs;
  a.Ja = Ja;
  a.invJ = invJ;
  a.gradW = grad;  // every entry is written by the gradient kernel before it is read
  a.nbr = nbr;
  a.status = status;
  if (dg_f64_gradients(a, st) != cudaSuccess) return DG_ECUDA;
  if (dg_f64_rhs(a, st) != cudaSuccess) return DG_ECUDA;
  return DG_OK;
}
