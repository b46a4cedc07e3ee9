// Mixture thermodynamics kernels (filled in with the multi-species form).
#include "dg_thermo.h"
cudaError_t dg_thermo_upload_basis() { return cudaSuccess; }
cudaError_t dg_thermo_init(DgThermo*, int64_t, int, int, const double*, int, int, unsigned long long*) {
  return cudaErrorNotSupported;
}
void dg_thermo_free(DgThermo*) {}
cudaError_t dg_thermo_reset(DgThermo*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t dg_thermo_update(DgThermo*, const void*, int, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t dg_thermo_boundary(DgThermo*, const double*, int, void*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t dg_thermo_prim2cons(DgThermo*, const double*, void*, cudaStream_t) { return cudaErrorNotSupported; }
