// Instantiations of the fused sweep kernel with the bulk arithmetic in
// FP64 (every step of the path in double precision).
#include "sweep.cuh"

#include <cstring>

namespace enoao {

template <int NV, int ORDER>
static cudaError_t launch_one(const SweepArgs& a, int grid, int block, size_t smem,
                              cudaStream_t s) {
  CUtensorMap none;  // direct loads: the map is not read
  memset(&none, 0, sizeof none);
  sweep_kernel<NV, ORDER, double><<<grid, block, smem, s>>>(a, none);
  return cudaGetLastError();
}

template <int NV, int ORDER>
static cudaError_t configure_one(size_t smem) {
  return raise_smem_limit(sweep_kernel<NV, ORDER, double>, smem);
}

template <int NV, int ORDER>
static cudaError_t occupancy_one(int block, size_t smem, int* per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, sweep_kernel<NV, ORDER, double>,
                                                       block, smem);
}

#define ENOAO_DISPATCH(FN, ...)                                 \
  switch (nv * 10 + order) {                                    \
    case 15: return FN<1, 5>(__VA_ARGS__);                      \
    case 17: return FN<1, 7>(__VA_ARGS__);                      \
    case 35: return FN<3, 5>(__VA_ARGS__);                      \
    case 37: return FN<3, 7>(__VA_ARGS__);                      \
    case 45: return FN<4, 5>(__VA_ARGS__);                      \
    case 47: return FN<4, 7>(__VA_ARGS__);                      \
    case 55: return FN<5, 5>(__VA_ARGS__);                      \
    case 57: return FN<5, 7>(__VA_ARGS__);                      \
    default: return cudaErrorInvalidValue;                      \
  }

cudaError_t sweep_launch_fp64(int nv, int order, const SweepArgs& a, int grid, int block,
                              size_t smem, cudaStream_t s) {
  ENOAO_DISPATCH(launch_one, a, grid, block, smem, s)
}

cudaError_t sweep_configure_fp64(int nv, int order, size_t smem) {
  ENOAO_DISPATCH(configure_one, smem)
}

cudaError_t sweep_occupancy_fp64(int nv, int order, int block, size_t smem, int* per_sm) {
  ENOAO_DISPATCH(occupancy_one, block, smem, per_sm)
}

}  // namespace enoao
