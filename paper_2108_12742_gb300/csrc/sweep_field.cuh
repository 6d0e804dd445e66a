// Instantiations of the sweep kernel with per-field splitting constants
// (Euler systems only; scalar advection has one field), for the bulk type
// ENOAO_FIELD_R; included by sweep_fp32_field.cu and sweep_fp64_field.cu.
#include "sweep.cuh"

#include <cstring>

namespace enoao {
namespace {

using FR = ENOAO_FIELD_R;

template <int NV, int ORDER>
cudaError_t launch_field(const SweepArgs& a, int grid, int block, size_t smem, cudaStream_t s) {
  CUtensorMap none;  // direct loads: the map is not read
  memset(&none, 0, sizeof none);
  sweep_kernel<NV, ORDER, FR, false, true><<<grid, block, smem, s>>>(a, none);
  return cudaGetLastError();
}

template <int NV, int ORDER>
cudaError_t configure_field(size_t smem) {
  return raise_smem_limit(sweep_kernel<NV, ORDER, FR, false, true>, smem);
}

template <int NV, int ORDER>
cudaError_t occupancy_field(int block, size_t smem, int* per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      per_sm, sweep_kernel<NV, ORDER, FR, false, true>, block, smem);
}

}  // namespace

#define ENOAO_FIELD_DISPATCH(FN, ...)    \
  switch (nv * 10 + order) {             \
    case 35: return FN<3, 5>(__VA_ARGS__); \
    case 37: return FN<3, 7>(__VA_ARGS__); \
    case 45: return FN<4, 5>(__VA_ARGS__); \
    case 47: return FN<4, 7>(__VA_ARGS__); \
    case 55: return FN<5, 5>(__VA_ARGS__); \
    case 57: return FN<5, 7>(__VA_ARGS__); \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t ENOAO_FIELD_NAME(launch)(int nv, int order, const SweepArgs& a, int grid, int block,
                                     size_t smem, cudaStream_t s) {
  ENOAO_FIELD_DISPATCH(launch_field, a, grid, block, smem, s)
}

cudaError_t ENOAO_FIELD_NAME(configure)(int nv, int order, size_t smem) {
  ENOAO_FIELD_DISPATCH(configure_field, smem)
}

cudaError_t ENOAO_FIELD_NAME(occupancy)(int nv, int order, int block, size_t smem, int* per_sm) {
  ENOAO_FIELD_DISPATCH(occupancy_field, block, smem, per_sm)
}

}  // namespace enoao
