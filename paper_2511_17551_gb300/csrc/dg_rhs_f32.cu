// Mixed form: FP32 two-point fluxes, volume sums and accumulation (the caller keeps
// FP64 for the time-step reduction and the domain integrals).
#define DG_REAL float
#define DG_PREFIX dg_f32
#include <string.h>
#include "dg_rhs_impl.cuh"
