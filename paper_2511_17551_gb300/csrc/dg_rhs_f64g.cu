// FP64 form, right-hand-side kernels with the runtime choice of volume and surface flux.
#define DG_REAL double
#define DG_PREFIX dg_f64g
#define DG_GENERIC_ONLY 1
#include <string.h>
#include "dg_rhs_impl.cuh"
