// FP64 form of the right-hand-side kernels.
#define DG_REAL double
#define DG_PREFIX dg_f64
#include <string.h>
#include "dg_rhs_impl.cuh"
