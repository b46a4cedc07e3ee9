// Mixed form: FP32 two-point fluxes, volume sums and accumulation (the caller keeps
// FP64 for the time-step reduction and the domain integrals).  Production flux pair;
// the compile-time split forms live in dg_rhs_f32s.cu, the other pairs in dg_rhs_f32g.cu.
#define DG_REAL float
#define DG_PREFIX dg_f32
#define DG_GENERIC_RHS dg_f32g_rhs
#define DG_GENERIC_UPLOAD dg_f32g_upload_basis
#define DG_SPLIT_RHS dg_f32s_rhs
#define DG_SPLIT_UPLOAD dg_f32s_upload_basis
#include <string.h>
#include "dg_rhs_impl.cuh"
