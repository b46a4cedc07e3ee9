// Allocation-free variant of the FP64 Navier-Stokes right-hand side.
//
// Who needs it: code that runs where device allocation is not allowed -- a host
// framework that owns all device memory and hands a library only its inputs and
// outputs (custom-operator and plugin interfaces work this way), or a real-time
// loop that must not call cudaMalloc/cudaFree because they synchronise the device
// and can fail at run time.  dg_init_mesh allocates the context's buffers, so such
// callers cannot use dg_rhs; this entry point takes every input and output from
// the caller and keeps its scratch (a status word, a checked copy of the neighbour
// table and the BR1 gradients of (v, p/rho), 12 doubles per node) in a file-scope
// device array that exists once per GPU for the life of the process.
#include <cuda_runtime.h>
#include <string.h>
#include <time.h>

#include <atomic>
#include <mutex>

#include "../../include/dg.h"
#include "dg_internal.h"

namespace {

// [0, 256): device status word; [256, 256 + nbr bytes rounded up to 256): the checked
// neighbour table [K][6] int32; then the gradients [K][3][4][np] FP64
static __device__ __align__(256) unsigned char g_noalloc_scratch[DG_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
struct NoallocSetup {
  std::atomic<int> done;
  unsigned char* base;  // device address of g_noalloc_scratch on that device
};
NoallocSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

size_t nbr_bytes(int64_t K) { return (((size_t)K * 6 * sizeof(int32_t)) + 255) & ~(size_t)255; }

// Copies the caller's neighbour table into the scratch.  An entry outside [0, K) (a
// boundary face, which this periodic-only entry point does not support, or a corrupt
// index) is replaced by the element's own index, so that no kernel reads outside the
// state, and latches (DG_EINVAL << 56) | element in the status word.
__global__ void check_nbr_kernel(const int32_t* nbr, int64_t K, int32_t* out, unsigned long long* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < K * 6; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t nb = nbr[i];
    const int64_t e = i / 6;
    if (nb >= 0 && nb < K) {
      out[i] = nb;
    } else {
      out[i] = (int32_t)e;
      atomicCAS(status, 0ull, ((unsigned long long)DG_EINVAL << 56) | (unsigned long long)e);
    }
  }
}

// device address of the scratch on the current device, looked up once per device
// (thread-safe: concurrent first calls serialise on a mutex)
dg_status scratch_base(unsigned char** base) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DG_ECUDA;
  NoallocSetup& s = g_setup[dev];
  if (!s.done.load(std::memory_order_acquire)) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!s.done.load(std::memory_order_relaxed)) {
      void* p = NULL;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == NULL) return DG_ECUDA;
      if (dg_f64_upload_basis() != cudaSuccess) return DG_ECUDA;
      s.base = (unsigned char*)p;
      s.done.store(1, std::memory_order_release);
    }
  }
  *base = s.base;
  return DG_OK;
}

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
  const double need = 256.0 + (double)nbr_bytes(K) + (double)K * np * 12.0 * sizeof(double);
  if (need > (double)DG_NOALLOC_SCRATCH_BYTES) return DG_EINVAL;  // beyond the static scratch
  unsigned char* base = NULL;
  const dg_status sb = scratch_base(&base);
  if (sb != DG_OK) return sb;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* status = (unsigned long long*)base;
  int32_t* nbr_ok = (int32_t*)(base + 256);
  double* grad = (double*)(base + 256 + nbr_bytes(K));
  if (cudaMemsetAsync(status, 0, sizeof(unsigned long long), st) != cudaSuccess) return DG_ECUDA;
  int64_t g = (K * 6 + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  check_nbr_kernel<<<(unsigned)g, 256, 0, st>>>(nbr, K, nbr_ok, status);
  if (cudaGetLastError() != cudaSuccess) return DG_ECUDA;

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
  a.nbr = nbr_ok;  // every entry in [0, K): no boundary table is needed
  a.status = status;
  if (dg_f64_gradients(a, st) != cudaSuccess) return DG_ECUDA;
  if (dg_f64_rhs(a, st) != cudaSuccess) return DG_ECUDA;
  return DG_OK;
}

extern "C" dg_status dg_noalloc_status(void* stream, uint64_t* status_out) {
  if (!status_out) return DG_EINVAL;
  unsigned char* base = NULL;
  const dg_status sb = scratch_base(&base);
  if (sb != DG_OK) return sb;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long word = 0;
  if (cudaMemcpyAsync(&word, base, sizeof(word), cudaMemcpyDeviceToHost, st) != cudaSuccess) return DG_ECUDA;
  // bounded wait for the copy (600 s of wall time, 20 us sleeps after the first 2 ms)
  struct timespec t0, t1;
  clock_gettime(CLOCK_MONOTONIC, &t0);
  for (;;) {
    const cudaError_t q = cudaStreamQuery(st);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return DG_ECUDA;
    clock_gettime(CLOCK_MONOTONIC, &t1);
    const double el = (double)(t1.tv_sec - t0.tv_sec) + 1e-9 * (double)(t1.tv_nsec - t0.tv_nsec);
    if (el > 600.0) return DG_ETIMEOUT;
    if (el > 2e-3) {
      struct timespec ts = {0, 20000};
      nanosleep(&ts, NULL);
    }
  }
  *status_out = word;
  if (word == 0) return DG_OK;
  const unsigned long long code = word >> 56;
  return code == DG_EINVAL ? DG_EINVAL : (code == DG_ST_TIMEOUT ? DG_ETIMEOUT : DG_ENONPHYS);
}
