// Instantiations of the fused sweep kernel with the bulk arithmetic in
// FP32 (state and Runge-Kutta combine in FP64).
#include "sweep.cuh"

#include <cstring>

namespace enoao {

// Two variants per system and order: the sweep that re-decides its near-ties
// itself, and the one that lists them for the grid-wide pass (a.redo set).
// Three variants per system and order: the sweep that re-decides its
// near-ties itself (raw tiles loaded directly, or staged by TMA when tmap is
// given), and the one that lists them for the grid-wide pass (a.redo set).
// The LEAN kernel (ENO-AO5 only): re-decisions out of line, seven blocks.
template <int NV, int ORDER>
static auto lean_kernel() {
  return sweep_kernel<NV, ORDER, float, false, false, false, ORDER == 5>;
}

template <int NV, int ORDER>
static cudaError_t launch_one(const SweepArgs& a, int grid, int block, size_t smem,
                              cudaStream_t s, const CUtensorMap* tmap) {
  CUtensorMap none;
  memset(&none, 0, sizeof none);
  if (a.redo)
    sweep_kernel<NV, ORDER, float, true><<<grid, block, smem, s>>>(a, none);
  else if (tmap)
    sweep_kernel<NV, ORDER, float, false, false, true><<<grid, block, smem, s>>>(a, *tmap);
  else if (a.lean && ORDER == 5)
    lean_kernel<NV, ORDER>()<<<grid, block, smem, s>>>(a, none);
  else
    sweep_kernel<NV, ORDER, float, false><<<grid, block, smem, s>>>(a, none);
  return cudaGetLastError();
}

template <int NV, int ORDER>
static cudaError_t configure_one(size_t smem, int variant) {
  if (variant == 1) return raise_smem_limit(sweep_kernel<NV, ORDER, float, false, false, true>, smem);
  if (variant == 2) return raise_smem_limit(lean_kernel<NV, ORDER>(), smem);
  cudaError_t e = raise_smem_limit(sweep_kernel<NV, ORDER, float, false>, smem);
  if (e == cudaSuccess) e = raise_smem_limit(sweep_kernel<NV, ORDER, float, true>, smem);
  return e;
}

// Resident blocks per SM: the TMA or LEAN variant, or the smaller of the
// other two.
template <int NV, int ORDER>
static cudaError_t occupancy_one(int block, size_t smem, int* per_sm, int variant) {
  if (variant == 1)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        per_sm, sweep_kernel<NV, ORDER, float, false, false, true>, block, smem);
  if (variant == 2)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, lean_kernel<NV, ORDER>(), block,
                                                         smem);
  int p0 = 0, p1 = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &p0, sweep_kernel<NV, ORDER, float, false>, block, smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p1, sweep_kernel<NV, ORDER, float, true>,
                                                      block, smem);
  *per_sm = p0 < p1 ? p0 : p1;
  return e;
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

cudaError_t sweep_launch_fp32(int nv, int order, const SweepArgs& a, int grid, int block,
                              size_t smem, cudaStream_t s, const CUtensorMap* tmap) {
  ENOAO_DISPATCH(launch_one, a, grid, block, smem, s, tmap)
}

template <int NV, int ORDER>
static cudaError_t redo_one(const SweepArgs& a, int grid, cudaStream_t s) {
  redo_kernel<NV, ORDER><<<grid, 128, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  redo_apply_kernel<NV><<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

// The grid-wide FP64 re-decision pass of a sweep launched with a.redo set (two
// kernels, stream-ordered after the sweep).
cudaError_t redo_launch_fp32(int nv, int order, const SweepArgs& a, int grid, cudaStream_t s) {
  ENOAO_DISPATCH(redo_one, a, grid, s)
}

cudaError_t sweep_configure_fp32(int nv, int order, size_t smem, int variant) {
  ENOAO_DISPATCH(configure_one, smem, variant)
}

cudaError_t sweep_occupancy_fp32(int nv, int order, int block, size_t smem, int* per_sm,
                                 int variant) {
  ENOAO_DISPATCH(occupancy_one, block, smem, per_sm, variant)
}

}  // namespace enoao
