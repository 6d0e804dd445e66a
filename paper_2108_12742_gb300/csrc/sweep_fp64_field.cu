// Sweep kernels with per-field splitting constants, FP64.
#define ENOAO_FIELD_R double
#define ENOAO_FIELD_NAME(x) sweep_##x##_fp64_field
#include "sweep_field.cuh"
