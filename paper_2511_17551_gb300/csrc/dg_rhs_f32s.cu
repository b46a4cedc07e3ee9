// Mixed form, right-hand-side kernels with a compile-time one-gas split form other than
// the production one (Ducros, standard DG, Kennedy-Gruber, Pirozzoli, Morinishi) and LLF
// interfaces, 3D at N = 3.
#define DG_REAL float
#define DG_PREFIX dg_f32s
#define DG_GENERIC_ONLY 1
#define DG_SPLIT_ONLY 1
#include <string.h>
#include "dg_rhs_impl.cuh"
