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
#include "enoao_ctx.h"
#include "enoao_internal.h"
#include "sweep.cuh"

namespace enoao {

struct BatchArgs {
  double* U[3];            // U^n, U1, U2; [nv][total]
  float* inc[2];           // FP32 bulk: stage increments I0, I1; [nv][total]
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
  int per_stage_alpha;     // 1: each stage splits with the alpha of its input state
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

// Resident 256-thread blocks per SM asked of the compiler: FP32 bulk four
// (64 registers, some spilled), FP64 three (80).  4096 uneven problems,
// against the unbounded 116 registers and two blocks: FP32 bulk 1.52e10 ->
// 1.68e10 (three) -> 1.73e10 (four) cell-stage/s; FP64 1.37e9 at three,
// 1.30e9 at four.
template <typename R>
constexpr int batch_min_blocks() {
  return sizeof(R) == 4 ? 4 : 3;
}

template <int NV, int ORDER, typename R>
__global__ void __launch_bounds__(256, batch_min_blocks<R>()) batch_kernel(const BatchArgs B) {
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
    A.nfaces = n + 1;
    A.cstride = B.total;
    A.ndim = 1;
    A.dir = 0;
    A.bc = B.bc;
    A.ta = 1;
    A.ts = B.ts;
    A.se = B.ts + 2 * Geo<ORDER>::G;  // sweep_row_pitch of a one-line x tile
    A.tiles_s = (n + B.ts - 1) / B.ts;
    A.tiles_a = A.tiles_b = 1;
    A.ntiles = A.tiles_s;
    A.inv_dx = 1.0 / dx;
    A.gamma = B.gamma;
    A.adv_speed = B.adv_speed;
    A.delta = B.delta;
    A.tie_rel = B.tie_rel;
    set_derived_constants(A);
    A.redo_passes = 64 * NV;

    // alpha of the initial state of this launch
    double alpha;
    if constexpr (NV > 1) {
      double a = 0.0;
      const double* U = B.U[0] + off;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        // the speeds as a step's last stage takes them (FP32 bulk: speeds32),
        // so that launches split anywhere give the same run
        double u[NV], sp[3];
#pragma unroll
        for (int c = 0; c < NV; ++c) u[c] = __ldcg(U + c * B.total + i);
        const bool ok = sizeof(R) == 4 ? speeds32<NV, false>(u, B.gamma, sp)
                                       : speeds64<NV, false>(u, B.gamma, sp);
        if (!ok) {
          atomicOr(&B.st->err, kErrNonPhys);
          atomicMin(&B.st->err_cell, off + i);
          continue;
        }
        a = fmax(a, sp[0]);
      }
      alpha = block_max(a, s_red);
    } else {
      alpha = fabs(B.adv_speed);
    }
    double t = B.t[p], dt = 0.0;
    const bool per_stage = NV > 1 && B.per_stage_alpha;
    double alpha_step = alpha;  // alpha the last step split with
    for (int step = 0; step < B.nsteps; ++step) {
      alpha_step = alpha;
      dt = B.cfl / (alpha / dx);
      double a_stage = alpha;  // splitting constant of the current stage
      for (int stage = 0; stage < 3; ++stage) {
        double amax[3] = {0.0, 0.0, 0.0};
        A.u_in = B.U[stage] + off;
        A.u0 = B.U[0] + off;
        A.u_out = B.U[stage == 2 ? 0 : stage + 1] + off;
        A.inc_in = stage == 0 ? nullptr : B.inc[stage - 1] + off;
        A.inc_out = stage == 2 ? nullptr : B.inc[stage] + off;
        A.stage = stage;
        A.mode = kModeCombine | (stage == 2 || per_stage ? kModeAlpha : 0);
        for (long long tile = 0; tile < A.ntiles; ++tile)
          sweep_tile<NV, ORDER, R, true>(A, tile_geo(A, tile), smem_raw, a_stage, dt, amax, nfall);
        if constexpr (NV > 1) {
          if (stage == 2)
            alpha = block_max(amax[0], s_red);
          else if (per_stage)
            a_stage = block_max(amax[0], s_red);
        }
      }
      t += dt;
    }
    if (threadIdx.x == 0) {
      B.t[p] = t;
      B.alpha[p] = alpha_step;
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
  float* inc[2] = {nullptr, nullptr};
  int ts = 256, block = 256;
  long long steps = 0;
  std::vector<long long> off_h;
  cudaGraphExec_t graph = nullptr;
  long long graph_steps = 0;
  double graph_cfl = 0.0;
};

namespace {

template <int NV, int ORDER, typename R>
cudaError_t launch_batch_t(const BatchArgs& b, int block, size_t smem, int sms, cudaStream_t s) {
  cudaError_t e = raise_smem_limit(batch_kernel<NV, ORDER, R>, smem);
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

// ---------------------------------------------------------------- host side

namespace {

enoao_status bfail(enoao_ctx* c, enoao_status st, const std::string& msg) {
  c->err = msg;
  return st;
}

#define BCU(c, call)                                                                    \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return bfail((c), ENOAO_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

__global__ void batch_reset_kernel(StepState* st) {
  st->err = 0;
  st->err_cell = 0x7fffffffffffffffll;
  st->fallbacks = 0;
  st->skip = 0;
}

// rho > 0 and p > 0 of every cell of the concatenated 1D Euler states.
__global__ void batch_check_kernel(const double* U, long long total, double gamma, StepState* st) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const double rho = U[i], m = U[total + i], E = U[2 * total + i];
    const double p = (gamma - 1.0) * (E - 0.5 * m * m / rho);
    if (!(rho > 0.0) || !(p > 0.0) || !isfinite(p)) {
      atomicOr(&st->err, kErrNonPhys);
      atomicMin(&st->err_cell, i);
    }
  }
}

BatchArgs make_args(enoao_ctx* c, int nsteps, double cfl) {
  BatchState* b = c->batch;
  BatchArgs a;
  memset(&a, 0, sizeof a);
  for (int k = 0; k < 3; ++k) a.U[k] = b->U[k];
  for (int k = 0; k < 2; ++k) a.inc[k] = b->inc[k];
  a.total = b->total;
  a.nprob = b->nprob;
  a.nsteps = nsteps;
  a.cfl = cfl;
  a.order = b->order;
  a.off = b->off;
  a.n = b->n;
  a.dx = b->dx;
  a.t = b->t;
  a.alpha = b->alpha;
  a.dt = b->dt;
  a.queue = b->queue;
  a.st = c->st;
  a.ts = b->ts;
  a.bc = c->cfg.bc[0];
  a.gamma = c->cfg.gamma;
  a.adv_speed = c->cfg.adv_speed;
  a.delta = c->cfg.delta;
  a.tie_rel = c->cfg.tie_rel;
  a.per_stage_alpha = c->cfg.alpha_mode == ENOAO_ALPHA_PER_STAGE;
  return a;
}

enoao_status enqueue_batch(enoao_ctx* c, int nsteps, double cfl) {
  BatchState* b = c->batch;
  const int f32 = c->cfg.precision == ENOAO_FP32_BULK;
  const size_t smem = sweep_smem_bytes(b->nv, c->cfg.order, f32, 1, b->ts,
                                       sweep_row_pitch(b->nv, c->cfg.order, f32, 0, 1, b->ts));
  cudaError_t e = launch_batch(b->nv, c->cfg.order, f32, make_args(c, nsteps, cfl), b->block, smem,
                               c->sms, c->s);
  if (e != cudaSuccess)
    return bfail(c, ENOAO_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
  return ENOAO_OK;
}

enoao_status stream_enter(enoao_ctx* c) {
  BCU(c, cudaSetDevice(c->device));
  BCU(c, cudaEventRecord(c->ev_a, c->user));
  BCU(c, cudaStreamWaitEvent(c->s, c->ev_a, 0));
  return ENOAO_OK;
}

enoao_status stream_leave(enoao_ctx* c) {
  BCU(c, cudaEventRecord(c->ev_b, c->s));
  BCU(c, cudaStreamWaitEvent(c->user, c->ev_b, 0));
  return ENOAO_OK;
}

enoao_status read_err(enoao_ctx* c) {
  BCU(c, cudaMemcpyAsync(c->st_host, c->st, sizeof(StepState), cudaMemcpyDeviceToHost, c->s));
  BCU(c, cudaStreamSynchronize(c->s));
  if (c->st_host->err & kErrNonPhys)
    return bfail(c, ENOAO_ENONPHYS,
                 "non-physical state (rho <= 0, p <= 0 or NaN) at cell " +
                     std::to_string((long long)c->st_host->err_cell));
  return ENOAO_OK;
}

}  // namespace

void batch_destroy(BatchState* b) {
  if (!b) return;
  for (int k = 0; k < 3; ++k) cudaFree(b->U[k]);
  for (int k = 0; k < 2; ++k) cudaFree(b->inc[k]);
  cudaFree(b->order);
  cudaFree(b->off);
  cudaFree(b->n);
  cudaFree(b->dx);
  cudaFree(b->t);
  cudaFree(b->alpha);
  cudaFree(b->dt);
  cudaFree(b->queue);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  delete b;
}

enoao_status batch_create(enoao_ctx* c, const enoao_config* proto, int nprob, const int64_t* n,
                          const double* lo, const double* hi) {
  const int G = proto->order / 2 + 2;
  std::vector<long long> off(nprob);
  std::vector<int> nn(nprob), order(nprob);
  std::vector<double> dx(nprob);
  long long total = 0;
  for (int i = 0; i < nprob; ++i) {
    if (n[i] < 2 * G + 1 || n[i] > (1 << 30))
      return bfail(c, ENOAO_EINVAL, "problem " + std::to_string(i) + " has " +
                                        std::to_string((long long)n[i]) + " cells; at least " +
                                        std::to_string(2 * G + 1) + " are needed");
    if (!(hi[i] > lo[i])) return bfail(c, ENOAO_EINVAL, "problem " + std::to_string(i) + ": hi <= lo");
    off[i] = total;
    nn[i] = (int)n[i];
    dx[i] = (hi[i] - lo[i]) / (double)n[i];
    total += n[i];
  }
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return nn[a] > nn[b]; });
  BatchState* b = new BatchState;
  c->batch = b;
  b->nprob = nprob;
  b->total = total;
  b->nv = proto->system == ENOAO_EULER ? 3 : 1;
  b->off_h = off;
  b->ts = 256;
  b->block = 256;
  c->ncell = total;
  const size_t sb = (size_t)b->nv * total * sizeof(double);
  for (int k = 0; k < 3; ++k) BCU(c, cudaMalloc(&b->U[k], sb));
  if (proto->precision == ENOAO_FP32_BULK)
    for (int k = 0; k < 2; ++k) BCU(c, cudaMalloc(&b->inc[k], (size_t)b->nv * total * sizeof(float)));
  BCU(c, cudaMalloc(&b->order, nprob * sizeof(int)));
  BCU(c, cudaMalloc(&b->off, nprob * sizeof(long long)));
  BCU(c, cudaMalloc(&b->n, nprob * sizeof(int)));
  BCU(c, cudaMalloc(&b->dx, nprob * sizeof(double)));
  BCU(c, cudaMalloc(&b->t, nprob * sizeof(double)));
  BCU(c, cudaMalloc(&b->alpha, nprob * sizeof(double)));
  BCU(c, cudaMalloc(&b->dt, nprob * sizeof(double)));
  BCU(c, cudaMalloc(&b->queue, sizeof(int)));
  BCU(c, cudaMemcpy(b->order, order.data(), nprob * sizeof(int), cudaMemcpyHostToDevice));
  BCU(c, cudaMemcpy(b->off, off.data(), nprob * sizeof(long long), cudaMemcpyHostToDevice));
  BCU(c, cudaMemcpy(b->n, nn.data(), nprob * sizeof(int), cudaMemcpyHostToDevice));
  BCU(c, cudaMemcpy(b->dx, dx.data(), nprob * sizeof(double), cudaMemcpyHostToDevice));
  BCU(c, cudaMemset(b->t, 0, nprob * sizeof(double)));
  BCU(c, cudaMemset(b->alpha, 0, nprob * sizeof(double)));
  BCU(c, cudaMemset(b->dt, 0, nprob * sizeof(double)));
  return ENOAO_OK;
}

enoao_status batch_init_state(enoao_ctx* c, const double* U, int on_device) {
  BatchState* b = c->batch;
  enoao_status r = stream_enter(c);
  if (r != ENOAO_OK) return r;
  BCU(c, cudaMemcpyAsync(b->U[0], U, (size_t)b->nv * b->total * sizeof(double),
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->s));
  BCU(c, cudaMemsetAsync(b->t, 0, b->nprob * sizeof(double), c->s));
  batch_reset_kernel<<<1, 1, 0, c->s>>>(c->st);
  if (b->nv == 3)
    batch_check_kernel<<<std::max(1, std::min<int>((int)((b->total + 255) / 256), c->sms * 8)), 256,
                         0, c->s>>>(b->U[0], b->total, c->cfg.gamma, c->st);
  BCU(c, cudaGetLastError());
  b->steps = 0;
  r = stream_leave(c);
  if (r != ENOAO_OK) return r;
  return read_err(c);
}

enoao_status batch_get_state(enoao_ctx* c, double* U, int on_device) {
  BatchState* b = c->batch;
  enoao_status r = stream_enter(c);
  if (r != ENOAO_OK) return r;
  BCU(c, cudaMemcpyAsync(U, b->U[0], (size_t)b->nv * b->total * sizeof(double),
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->s));
  r = stream_leave(c);
  if (r != ENOAO_OK) return r;
  BCU(c, cudaStreamSynchronize(c->s));
  return ENOAO_OK;
}

// One CUDA graph holds the queue reset and the persistent launch for a given
// (nsteps, cfl); replays reuse it.
enoao_status batch_advance(enoao_ctx* c, int64_t nsteps, double cfl, bool sync) {
  BatchState* b = c->batch;
  if (nsteps > (1 << 30)) return bfail(c, ENOAO_EINVAL, "nsteps too large");
  enoao_status r = stream_enter(c);
  if (r != ENOAO_OK) return r;
  if (!b->graph || b->graph_steps != nsteps || b->graph_cfl != cfl) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    cudaGraph_t g;
    BCU(c, cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal));
    r = enqueue_batch(c, (int)nsteps, cfl);
    cudaError_t e = cudaStreamEndCapture(c->s, &g);
    if (r != ENOAO_OK) return r;
    if (e != cudaSuccess) return bfail(c, ENOAO_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(c, ENOAO_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    b->graph_steps = nsteps;
    b->graph_cfl = cfl;
  }
  BCU(c, cudaGraphLaunch(b->graph, c->s));
  b->steps += nsteps;
  r = stream_leave(c);
  if (r != ENOAO_OK) return r;
  if (!sync) return ENOAO_OK;
  return read_err(c);
}

enoao_status batch_stats(enoao_ctx* c, enoao_stats* out) {
  BatchState* b = c->batch;
  enoao_status r = read_err(c);
  if (r != ENOAO_OK && r != ENOAO_ENONPHYS) return r;
  double t0 = 0.0, a0 = 0.0, d0 = 0.0;
  BCU(c, cudaMemcpy(&t0, b->t, sizeof(double), cudaMemcpyDeviceToHost));
  BCU(c, cudaMemcpy(&a0, b->alpha, sizeof(double), cudaMemcpyDeviceToHost));
  BCU(c, cudaMemcpy(&d0, b->dt, sizeof(double), cudaMemcpyDeviceToHost));
  memset(out, 0, sizeof *out);
  out->t = t0;
  out->steps = b->steps;
  out->alpha[0] = a0;
  out->dt = d0;
  out->fp64_fallbacks = c->st_host->fallbacks;
  return ENOAO_OK;
}

}  // namespace enoao

extern "C" enoao_status enoao_batch_problem_stats(enoao_ctx* c, int p, double* t, double* alpha,
                                                  double* dt) {
  using namespace enoao;
  if (!c) return ENOAO_EINVAL;
  if (!c->batch) {
    c->err = "not a batched context";
    return ENOAO_EINVAL;
  }
  BatchState* b = c->batch;
  if (p < 0 || p >= b->nprob) {
    c->err = "problem index out of range";
    return ENOAO_EINVAL;
  }
  enoao_status r = read_err(c);
  if (r != ENOAO_OK && r != ENOAO_ENONPHYS) return r;
  double v[3] = {0.0, 0.0, 0.0};
  BCU(c, cudaMemcpy(&v[0], b->t + p, sizeof(double), cudaMemcpyDeviceToHost));
  BCU(c, cudaMemcpy(&v[1], b->alpha + p, sizeof(double), cudaMemcpyDeviceToHost));
  BCU(c, cudaMemcpy(&v[2], b->dt + p, sizeof(double), cudaMemcpyDeviceToHost));
  if (t) *t = v[0];
  if (alpha) *alpha = v[1];
  if (dt) *dt = v[2];
  return ENOAO_OK;
}

namespace enoao {

// Times one step of the whole batch for each (tile, block) candidate on a
// saved copy of the state and keeps the fastest.
enoao_status batch_autotune(enoao_ctx* c) {
  BatchState* b = c->batch;
  const size_t sb = (size_t)b->nv * b->total * sizeof(double);
  double* save = nullptr;
  double* tsave = nullptr;
  BCU(c, cudaMalloc(&save, sb));
  cudaError_t e0 = cudaMalloc(&tsave, b->nprob * sizeof(double));
  if (e0 != cudaSuccess) {
    cudaFree(save);
    return bfail(c, ENOAO_ENOMEM, "autotune scratch");
  }
  enoao_status r = stream_enter(c);
  const int cands[][2] = {{128, 128}, {256, 128}, {256, 256}, {512, 256}};
  float best = 1e30f;
  int bts = b->ts, bblk = b->block;
  if (r == ENOAO_OK) {
    cudaMemcpyAsync(save, b->U[0], sb, cudaMemcpyDeviceToDevice, c->s);
    cudaMemcpyAsync(tsave, b->t, b->nprob * sizeof(double), cudaMemcpyDeviceToDevice, c->s);
    for (auto& cd : cands) {
      b->ts = cd[0];
      b->block = cd[1];
      cudaEventRecord(c->t0, c->s);
      enoao_status rr = enqueue_batch(c, 1, 0.5);
      cudaEventRecord(c->t1, c->s);
      cudaMemcpyAsync(b->U[0], save, sb, cudaMemcpyDeviceToDevice, c->s);
      if (rr != ENOAO_OK || cudaEventSynchronize(c->t1) != cudaSuccess) continue;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, c->t0, c->t1);
      if (ms < best) {
        best = ms;
        bts = cd[0];
        bblk = cd[1];
      }
    }
    cudaMemcpyAsync(b->t, tsave, b->nprob * sizeof(double), cudaMemcpyDeviceToDevice, c->s);
    cudaStreamSynchronize(c->s);
    c->err.clear();
  }
  b->ts = bts;
  b->block = bblk;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaFree(save);
  cudaFree(tsave);
  if (r != ENOAO_OK) return r;
  r = stream_leave(c);
  if (r != ENOAO_OK) return r;
  return read_err(c);
}

}  // namespace enoao
