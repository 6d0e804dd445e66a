// Sweep kernels with per-field splitting constants, FP32 bulk.
#define ENOAO_FIELD_R float
#define ENOAO_FIELD_NAME(x) sweep_##x##_fp32_field
#include "sweep_field.cuh"
