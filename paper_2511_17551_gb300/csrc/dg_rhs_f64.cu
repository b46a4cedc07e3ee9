// FP64 form of the right-hand-side kernels (production flux pair; the other pairs live
// in dg_rhs_f64g.cu).
#define DG_REAL double
#define DG_PREFIX dg_f64
#define DG_GENERIC_RHS dg_f64g_rhs
#define DG_GENERIC_UPLOAD dg_f64g_upload_basis
#include <string.h>
#include "dg_rhs_impl.cuh"
