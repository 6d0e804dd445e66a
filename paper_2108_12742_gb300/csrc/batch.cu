// Batched independent 1D problems of uneven lengths, all advanced by one
// persistent launch.  Each block takes whole problems from a work queue in
// longest-first order and runs every step of its problem -- alpha and dt of
// that problem (Sec. 2: alpha is the maximum of |f'(u)| over the problem's
// mesh), the three Runge-Kutta stages with the fused ENO-AO sweep of
// sweep.cuh, and the block reduction for the next alpha -- so no block ever
// waits for another.  A problem's three state buffers (<= 1.2 MB for 16k
// cells of the Euler equations) stay in L2 while its block works on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "enoao.h"
#include "enoao_internal.h"
#include "sweep.cuh"

namespace enoao {

struct BatchArgs {
  double* U[3];            // U^n, U1, U2; [nv][total]
  long long total;         // cells of all problems (component stride)
  int nprob;
  int nsteps;
  double cfl;
  const int* order;        // problem indices, largest first
  const long long* off;    // first cell of each problem
  const int* n;            // cells of each problem
  const double* dx;        // grid spacing of each problem
  double* t;               // time reached per problem
  double* alpha;           // alpha of the last step per problem
  double* dt;              // last step size per problem
  int* queue;              // next queue position (reset to 0 before a launch)
  StepState* st;           // error word and FP64 re-decision count
  int ts;                  // cells per tile
  int bc;
  double gamma, adv_speed, delta, tie_rel;
};

// Block-wide maximum of v (all threads get the result).
__device__ __forceinline__ double block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  double r = 0.0;
  for (int w = 0; w < nw; ++w) r = fmax(r, red[w]);
  return r;
}

template <int NV, int ORDER, typename R>
__global__ void __launch_bounds__(256) batch_kernel(const BatchArgs B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_q;
  __shared__ double s_red[32];
  unsigned long long nfall = 0;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_q = atomicAdd(B.queue, 1);
    __syncthreads();
    const int q = s_q;
    if (q >= B.nprob) break;
    const int p = B.order[q];
    const long long off = B.off[p];
    const int n = B.n[p];
    const double dx = B.dx[p];

    SweepArgs A;
    memset(&A, 0, sizeof A);
    A.st = B.st;
    A.n[0] = n;
    A.n[1] = A.n[2] = 1;
    A.ncell = n;
    A.cstride = B.total;
    A.ndim = 1;
    A.dir = 0;
    A.bc = B.bc;
    A.ta = 1;
    A.ts = B.ts;
    A.tiles_s = (n + B.ts - 1) / B.ts;
    A.tiles_a = A.tiles_b = 1;
    A.ntiles = A.tiles_s;
    A.inv_dx = 1.0 / dx;
    A.gamma = B.gamma;
    A.adv_speed = B.adv_speed;
    A.delta = B.delta;
    A.tie_rel = B.tie_rel;

    // alpha of the initial state of this launch
    double alpha;
    if constexpr (NV > 1) {
      double a = 0.0;
      const double* U = B.U[0] + off;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double rho = __ldcg(U + i), m = __ldcg(U + B.total + i), E = __ldcg(U + 2 * B.total + i);
        const double pr = (B.gamma - 1.0) * (E - 0.5 * m * m / rho);
        if (!(rho > 0.0) || !(pr > 0.0) || !isfinite(pr)) {
          atomicOr(&B.st->err, kErrNonPhys);
          atomicMin(&B.st->err_cell, off + i);
          continue;
        }
        a = fmax(a, fabs(m / rho) + sqrt(B.gamma * pr / rho));
      }
      alpha = block_max(a, s_red);
    } else {
      alpha = fabs(B.adv_speed);
    }
    double t = B.t[p], dt = 0.0;
    for (int step = 0; step < B.nsteps; ++step) {
      dt = B.cfl / (alpha / dx);
      double amax[3] = {0.0, 0.0, 0.0};
      for (int stage = 0; stage < 3; ++stage) {
        A.u_in = B.U[stage] + off;
        A.u0 = B.U[0] + off;
        A.u_out = B.U[stage == 2 ? 0 : stage + 1] + off;
        A.stage = stage;
        A.mode = kModeCombine | (stage == 2 ? kModeAlpha : 0);
        for (long long tile = 0; tile < A.ntiles; ++tile)
          sweep_tile<NV, ORDER, R, true>(A, tile_geo(A, tile), smem_raw, alpha, dt, amax, nfall);
      }
      t += dt;
      if constexpr (NV > 1) alpha = block_max(amax[0], s_red);
    }
    if (threadIdx.x == 0) {
      B.t[p] = t;
      B.alpha[p] = alpha;
      B.dt[p] = dt;
    }
  }
  if constexpr (sizeof(R) == 4) {
    if (nfall) atomicAdd(&B.st->fallbacks, nfall);
  }
}

struct BatchState {
  int nprob = 0;
  long long total = 0;
  int nv = 1;
  int* order = nullptr;
  long long* off = nullptr;
  int* n = nullptr;
  double* dx = nullptr;
  double* t = nullptr;
  double* alpha = nullptr;
  double* dt = nullptr;
  int* queue = nullptr;
  double* U[3] = {nullptr, nullptr, nullptr};
  int ts = 256, block = 256;
  long long steps = 0;
  std::vector<long long> off_h;
};

namespace {

template <int NV, int ORDER, typename R>
cudaError_t launch_batch_t(const BatchArgs& b, int block, size_t smem, int sms, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(batch_kernel<NV, ORDER, R>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<NV, ORDER, R>, block, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = std::min(b.nprob, sms * per_sm);
  e = cudaMemsetAsync(b.queue, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  batch_kernel<NV, ORDER, R><<<grid, block, smem, s>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_batch(int nv, int order, int fp32, const BatchArgs& b, int block, size_t smem,
                         int sms, cudaStream_t s) {
  const int key = nv * 100 + order * 10 + fp32;
  switch (key) {
    case 150: return launch_batch_t<1, 5, double>(b, block, smem, sms, s);
    case 170: return launch_batch_t<1, 7, double>(b, block, smem, sms, s);
    case 151: return launch_batch_t<1, 5, float>(b, block, smem, sms, s);
    case 171: return launch_batch_t<1, 7, float>(b, block, smem, sms, s);
    case 350: return launch_batch_t<3, 5, double>(b, block, smem, sms, s);
    case 370: return launch_batch_t<3, 7, double>(b, block, smem, sms, s);
    case 351: return launch_batch_t<3, 5, float>(b, block, smem, sms, s);
    case 371: return launch_batch_t<3, 7, float>(b, block, smem, sms, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// ---- entry points used by enoao_api.cu (the context owns the stream,
// the step state and the error string).
struct BatchHooks {
  static enoao_ctx* ctx;
};

}  // namespace enoao
