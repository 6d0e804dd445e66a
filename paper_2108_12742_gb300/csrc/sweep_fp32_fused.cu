// Instantiations of the fused 2D stage kernel (both axes of one Runge-Kutta
// stage in one launch), FP32 bulk, for the 2D systems (scalar advection and
// Euler, nv = 1 and 4).
#include "sweep.cuh"

namespace enoao {

template <int NV, int ORDER, bool LEAN>
static auto fused_kernel() {
  return fused2d_kernel<NV, ORDER, LEAN && ORDER == 5>;
}

template <int NV, int ORDER>
static cudaError_t fused_launch_one(const SweepArgs& ax, const SweepArgs& ay, int grid, int block,
                                    size_t smem, cudaStream_t s, int lean) {
  if (lean)
    fused_kernel<NV, ORDER, true>()<<<grid, block, smem, s>>>(ax, ay);
  else
    fused_kernel<NV, ORDER, false>()<<<grid, block, smem, s>>>(ax, ay);
  return cudaGetLastError();
}

template <int NV, int ORDER>
static cudaError_t fused_configure_one(size_t smem, int lean) {
  return lean ? raise_smem_limit(fused_kernel<NV, ORDER, true>(), smem)
              : raise_smem_limit(fused_kernel<NV, ORDER, false>(), smem);
}

template <int NV, int ORDER>
static cudaError_t fused_occupancy_one(int block, size_t smem, int* per_sm, int lean) {
  return lean ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fused_kernel<NV, ORDER, true>(),
                                                              block, smem)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    per_sm, fused_kernel<NV, ORDER, false>(), block, smem);
}

#define ENOAO_FUSED_DISPATCH(FN, ...)       \
  switch (nv * 10 + order) {                \
    case 15: return FN<1, 5>(__VA_ARGS__);  \
    case 17: return FN<1, 7>(__VA_ARGS__);  \
    case 45: return FN<4, 5>(__VA_ARGS__);  \
    case 47: return FN<4, 7>(__VA_ARGS__);  \
    default: return cudaErrorInvalidValue;  \
  }

cudaError_t fused2d_launch_fp32(int nv, int order, const SweepArgs& ax, const SweepArgs& ay,
                                int grid, int block, size_t smem, cudaStream_t s, int lean) {
  ENOAO_FUSED_DISPATCH(fused_launch_one, ax, ay, grid, block, smem, s, lean)
}

cudaError_t fused2d_configure_fp32(int nv, int order, size_t smem, int lean) {
  ENOAO_FUSED_DISPATCH(fused_configure_one, smem, lean)
}

cudaError_t fused2d_occupancy_fp32(int nv, int order, int block, size_t smem, int* per_sm,
                                   int lean) {
  ENOAO_FUSED_DISPATCH(fused_occupancy_one, block, smem, per_sm, lean)
}

}  // namespace enoao
