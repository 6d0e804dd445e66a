// Host runtime of the ENO-AO library: the C interface of include/enoao.h,
// device buffers, the step kernels that keep alpha and dt on the device, CUDA
// graph capture of whole steps, and the tile autotuner.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "enoao.h"
#include "enoao_ctx.h"
#include "enoao_internal.h"
#include "state_speed.cuh"

using namespace enoao;

namespace {

thread_local std::string g_create_error;

// Batched-problem state (defined with the batch kernels).
}  // namespace

namespace enoao {
// Message returned by enoao_last_error(NULL) on this host thread (used by
// entry points that have no context).
void set_thread_error(const char* msg) { g_create_error = msg; }
}  // namespace enoao

namespace {

enoao_status fail(enoao_ctx* c, enoao_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c)
    c->err = buf;
  else
    g_create_error = buf;
  return st;
}

#define CU(ctx, call)                                                                 \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail((ctx), ENOAO_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

constexpr double kInf = std::numeric_limits<double>::infinity();

// ---------------------------------------------------------------- small kernels

// alpha of the current state (Sec. 2: max of |f'(u)| over the mesh; for the
// Euler equations |u_d| + c per axis) into alpha_acc[slot] (and the per-field
// maxima into alpha_acc_f[slot] with FIELD), plus the non-physical check.
// BULK takes the speeds with the FP32 bulk arithmetic of a step's last stage
// (speeds32), so that a step from a state set here takes the same alpha as
// the uninterrupted run did.
template <int NV, bool BULK, bool FIELD>
__global__ void alpha_kernel(const double* __restrict__ U, long long ncell, long long cstride,
                             double gamma, StepState* st, int slot) {
  constexpr int ND = NV - 2;
  double amax[3] = {0, 0, 0};
  double af[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell;
       i += (long long)gridDim.x * blockDim.x) {
    double u[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) u[c] = U[c * cstride + i];
    double s[3];
    const bool ok = BULK ? speeds32<NV, false>(u, gamma, s) : speeds64<NV, false>(u, gamma, s);
    if (!ok) {
      atomicOr(&st->err, kErrNonPhys);
      atomicMin(&st->err_cell, i);
      continue;
    }
#pragma unroll
    for (int d = 0; d < ND; ++d) amax[d] = fmax(amax[d], s[d]);
    if constexpr (FIELD) {
      double sf[9];
      if (BULK ? speeds32<NV, true>(u, gamma, sf) : speeds64<NV, true>(u, gamma, sf)) {
#pragma unroll
        for (int k = 0; k < 3 * ND; ++k) af[k] = fmax(af[k], sf[k]);
      }
    }
  }
  if constexpr (FIELD) {  // rare option: one atomic per thread and value
#pragma unroll
    for (int k = 0; k < 3 * ND; ++k)
      if (af[k] > 0.0)
        atomicMax(&st->alpha_acc_f[slot][k / 3][k % 3], (unsigned long long)__double_as_longlong(af[k]));
  }
  __shared__ double red[3][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int d = 0; d < 3; ++d) {
    double v = amax[d];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[d][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int d = 0; d < 3; ++d) {
      double v = threadIdx.x < nw ? red[d][threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
      if (threadIdx.x == 0 && d < ND && v > 0.0)
        atomicMax(&st->alpha_acc[slot][d], (unsigned long long)__double_as_longlong(v));
    }
  }
}

template <int NV>
void launch_alpha_nv(const double* U, long long ncell, long long cstride, double gamma,
                     StepState* st, int slot, bool bulk, bool field, int blocks, cudaStream_t s) {
  if (bulk) {
    if (field)
      alpha_kernel<NV, true, true><<<blocks, 256, 0, s>>>(U, ncell, cstride, gamma, st, slot);
    else
      alpha_kernel<NV, true, false><<<blocks, 256, 0, s>>>(U, ncell, cstride, gamma, st, slot);
  } else {
    if (field)
      alpha_kernel<NV, false, true><<<blocks, 256, 0, s>>>(U, ncell, cstride, gamma, st, slot);
    else
      alpha_kernel<NV, false, false><<<blocks, 256, 0, s>>>(U, ncell, cstride, gamma, st, slot);
  }
}

// Launches alpha_kernel for an Euler state of nv = 3, 4 or 5 variables: ncell
// cells from U on, conserved components cstride apart.
void launch_alpha(int nv, const double* U, long long ncell, long long cstride, double gamma,
                  StepState* st, int slot, bool bulk, bool field, int blocks, cudaStream_t s) {
  if (nv == 3) launch_alpha_nv<3>(U, ncell, cstride, gamma, st, slot, bulk, field, blocks, s);
  if (nv == 4) launch_alpha_nv<4>(U, ncell, cstride, gamma, st, slot, bulk, field, blocks, s);
  if (nv == 5) launch_alpha_nv<5>(U, ncell, cstride, gamma, st, slot, bulk, field, blocks, s);
}

struct StepConsts {
  int system, ndim;
  int field;  // per-field splitting constants (Euler)
  double adv_speed;
  double dx[3];
};

__device__ void finalize_pending(StepState* st) {
  if (st->pending) {
    st->t = st->last ? st->t_end : st->t + st->dt;
    st->steps += 1;
    if (st->last) st->done = 1;
    st->pending = 0;
  }
}

// Per-field constants of the step from the running maxima of slot cur (the
// one-alpha value, for dt, is the largest of them); clear: the other slot too.
// alpha of axis d for the CFL rule (Euler): |u_d| + c of slot cur, which per
// field is the larger of max |u_d - c| and max |u_d + c| (the last stage then
// accumulates only the per-field maxima).
__device__ double step_alpha(const StepState* st, const StepConsts& k, int cur, int d) {
  if (k.field)
    return fmax(__longlong_as_double((long long)st->alpha_acc_f[cur][d][0]),
                __longlong_as_double((long long)st->alpha_acc_f[cur][d][2]));
  return __longlong_as_double((long long)st->alpha_acc[cur][d]);
}

__device__ void load_field_alpha(StepState* st, const StepConsts& k, int cur, bool clear) {
  if (!k.field) return;
  for (int d = 0; d < 3; ++d)
    for (int f = 0; f < 3; ++f) {
      st->alpha_f[d][f] = d < k.ndim ? __longlong_as_double((long long)st->alpha_acc_f[cur][d][f]) : 0.0;
      if (clear) st->alpha_acc_f[cur ^ 1][d][f] = 0ull;
    }
}

// Start of a step: finalise the previous one, fix alpha from U^n and dt from
// the CFL rule (or the fixed step), shortened to land on t_end.
__global__ void step_begin_kernel(StepState* st, StepConsts k) {
  finalize_pending(st);
  if (st->done || (st->max_steps > 0 && st->steps >= st->max_steps) || st->err) {
    st->skip = 1;
    return;
  }
  st->skip = 0;
  const int cur = (int)(st->steps & 1);
  double s = 0.0;
  for (int d = 0; d < k.ndim; ++d) {
    const double a = k.system == ENOAO_EULER
                         ? step_alpha(st, k, cur, d)
                         : fabs(k.adv_speed);
    st->alpha[d] = a;
    s += a / k.dx[d];
  }
  st->par = cur ^ 1;
  for (int d = 0; d < 3; ++d) st->alpha_acc[cur ^ 1][d] = st->alpha_stage[d] = 0ull;
  load_field_alpha(st, k, cur, true);
  double dt = st->dt_fixed > 0.0 ? st->dt_fixed : st->cfl / s;
  st->last = 0;
  if (st->t + dt >= st->t_end) {
    dt = st->t_end - st->t;
    st->last = 1;
  }
  st->dt = dt;
  st->pending = 1;
}

__global__ void finalize_kernel(StepState* st) { finalize_pending(st); }


// Per-stage alpha: the next stage splits with the alpha of the state the
// previous stage wrote (accumulated by that stage's last sweep).
__global__ void stage_alpha_kernel(StepState* st, StepConsts k) {
  if (st->skip) return;
  for (int d = 0; d < k.ndim; ++d) {
    st->alpha[d] = __longlong_as_double((long long)st->alpha_stage[d]);
    st->alpha_stage[d] = 0ull;
  }
}

// Manual stages (enoao_rk_stage): stage 0 begins a step with the caller's dt.
__global__ void manual_stage_kernel(StepState* st, StepConsts k, int stage, double dt) {
  if (stage == 0) {
    finalize_pending(st);
    st->skip = 0;
    const int cur = (int)(st->steps & 1);
    for (int d = 0; d < k.ndim; ++d)
      st->alpha[d] = k.system == ENOAO_EULER
                         ? step_alpha(st, k, cur, d)
                         : fabs(k.adv_speed);
    st->par = cur ^ 1;
    for (int d = 0; d < 3; ++d) st->alpha_acc[cur ^ 1][d] = st->alpha_stage[d] = 0ull;
    load_field_alpha(st, k, cur, true);
    st->last = 0;
    st->pending = 0;
  }
  st->dt = dt;
  if (stage == 2) st->pending = 1;  // finalised by the next step start / finalize
}

// For reconstruct_fluxes: alpha of the current state without starting a step.
__global__ void alpha_current_kernel(StepState* st, StepConsts k) {
  finalize_pending(st);
  const int cur = (int)(st->steps & 1);
  for (int d = 0; d < k.ndim; ++d)
    st->alpha[d] = k.system == ENOAO_EULER
                       ? step_alpha(st, k, cur, d)
                       : fabs(k.adv_speed);
  load_field_alpha(st, k, cur, false);
  st->skip = 0;
}

__global__ void reset_state_kernel(StepState* st) {
  StepState z;
  memset(&z, 0, sizeof z);
  z.t_end = __longlong_as_double(0x7ff0000000000000ll);  // +inf
  z.err_cell = 0x7fffffffffffffffll;
  *st = z;
}

__global__ void set_run_kernel(StepState* st, double t_end, double cfl, double dt_fixed,
                               long long max_steps) {
  st->t_end = t_end;
  st->cfl = cfl;
  st->dt_fixed = dt_fixed;
  st->max_steps = max_steps;
  st->done = st->t >= t_end ? 1 : 0;
  st->skip = 0;
}

// ---------------------------------------------------------------- helpers

StepConsts consts(const enoao_ctx* c) {
  StepConsts k;
  k.system = c->cfg.system;
  k.ndim = c->cfg.ndim;
  k.field = c->cfg.system == ENOAO_EULER && c->cfg.alpha_mode == ENOAO_ALPHA_PER_FIELD;
  k.adv_speed = c->cfg.adv_speed;
  for (int d = 0; d < 3; ++d) k.dx[d] = c->dx[d];
  return k;
}

bool fp32(const enoao_ctx* c) { return c->cfg.precision == ENOAO_FP32_BULK; }

int halo(int order) { return order / 2 + 2; }

// Tile lengths are 2^k - 1 cells so that the 2^k faces of a line fill whole
// warps in the per-face phase.
void default_tiles(enoao_ctx* c) {
  const bool f32 = fp32(c);
  for (int d = 0; d < c->cfg.ndim; ++d) {
    // FP32 2D ENO-AO5: 2 x 191 (x) and 8 x 31 (y) tiles take the LEAN kernel
    // at eight blocks per SM (measured fastest on 4096^2 Euler data)
    const bool lean2d = f32 && c->cfg.ndim == 2 && c->cfg.order == 5;
    if (d == 0) {
      c->ta[d] = c->cfg.ndim == 1 ? 1 : (lean2d ? 2 : 4);
      c->ts[d] = lean2d ? 191 : 63;
    } else {
      c->ta[d] = f32 ? 8 : 32;
      c->ts[d] = f32 ? (lean2d ? 31 : 47) : 15;
    }
    c->block[d] = 128;
  }
}

enoao_status check_tiles(enoao_ctx* c, int d, int ta, int ts) {
  if (ta < 1 || ts < 1 || ta * ts > 8192)
    return fail(c, ENOAO_EINVAL, "tile %dx%d out of range", ta, ts);
  if (d > 0 && ta != 8 && ta != 16 && ta != 32 && ta != 64)
    return fail(c, ENOAO_EINVAL, "axis %d needs 8, 16, 32 or 64 lines per tile", d);
  if (d == 0 && ta != 1 && ta != 2 && ta != 4 && ta != 8)
    return fail(c, ENOAO_EINVAL, "axis 0 needs 1, 2, 4 or 8 lines per tile");
  size_t smem = sweep_smem_bytes(c->nv, c->cfg.order, fp32(c), ta, ts,
                                 sweep_row_pitch(c->nv, c->cfg.order, fp32(c), d, ta, ts));
  if (smem > 200 * 1024)
    return fail(c, ENOAO_EINVAL, "tile %dx%d needs %zu bytes of shared memory", ta, ts, smem);
  return ENOAO_OK;
}

// FP32 bulk stepping: whether near-tie choices go to the grid-wide FP64
// re-decision pass after each sweep instead of being re-decided inside the
// sweep's tiles (enoao_set_redecide; AUTO currently re-decides in the sweep).
bool use_list(const enoao_ctx* c) {
  if (!fp32(c) || c->batch || c->sub || c->redecide != ENOAO_REDECIDE_GRID) return false;
  if (consts(c).field) return false;  // per-field splitting re-decides in the sweep
  long long faces = 0;
  for (int d = 0; d < c->cfg.ndim; ++d)
    faces = std::max(faces, c->ncell / c->cfg.n[d] * (c->cfg.n[d] + 1));
  return faces < (1ll << 32);  // list slots are counted in 32 bits
}

// Allocates the re-decision list when the context uses it: a slot per face of
// the axis with the most faces (a sweep lists each face at most once).
enoao_status ensure_list(enoao_ctx* c) {
  if (!use_list(c) || c->redo) return ENOAO_OK;
  long long cap = 0;
  for (int d = 0; d < c->cfg.ndim; ++d)
    cap = std::max(cap, c->ncell / c->cfg.n[d] * (c->cfg.n[d] + 1));
  cudaError_t e = cudaMalloc(&c->redo, (size_t)cap * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&c->redo_dc, (size_t)cap * c->nv * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&c->redo_mark, (size_t)cap * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->redo_mark, 0, (size_t)cap * sizeof(unsigned), c->s);
  if (e != cudaSuccess) {
    cudaFree(c->redo);
    cudaFree(c->redo_dc);
    cudaFree(c->redo_mark);
    c->redo = nullptr;
    c->redo_dc = nullptr;
    c->redo_mark = nullptr;
    return fail(c, e == cudaErrorMemoryAllocation ? ENOAO_ENOMEM : ENOAO_ECUDA,
                "re-decision list of %lld faces: %s", cap, cudaGetErrorString(e));
  }
  c->redo_cap = cap;
  return ENOAO_OK;
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link
// dependency on the driver library); NULL where it is not available.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// TMA staging of a sweep's raw tiles (the FP32-bulk sweep that re-decides its
// near-ties itself): the stencil source u_in as a tensor of FP64 values --
// (x, lines, components) for x sweeps, (x, y, z, components) otherwise -- and
// the box of one tile, every component at once.  Returns false (direct loads)
// where TMA cannot address the tiles: strides not a multiple of 16 bytes, box
// edges beyond 256 cells, sub-domains, the per-field and listing variants.
bool encode_tile_map(enoao_ctx* c, int d, bool list, const double* u_in, SweepArgs& a,
                     CUtensorMap* map) {
  if (!c->tma || !fp32(c) || list || consts(c).field || c->sub) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const int G = halo(c->cfg.order), nv = c->nv;
  const unsigned long long n0 = c->cfg.n[0], n1 = c->cfg.n[1], n2 = c->cfg.n[2];
  const unsigned long long cs = (unsigned long long)c->carr * 8ull;
  cuuint64_t dims[4], strides[3];
  cuuint32_t box[4], es[4] = {1, 1, 1, 1};
  int rank;
  if (d == 0) {
    int bx = a.ts + 2 * G + 1;  // one cell of slack: the box starts on an even x
    bx += bx & 1;               // whole 16-byte rows
    if (bx > 256) return false;
    rank = 3;
    dims[0] = n0, dims[1] = n1 * n2, dims[2] = nv;
    strides[0] = n0 * 8ull, strides[1] = cs;
    box[0] = bx, box[1] = a.ta, box[2] = nv;
    a.tma_box = bx;
  } else {
    const int sb = a.ts + 2 * G;
    if (sb > 256 || (a.ta & 1)) return false;
    rank = 4;
    dims[0] = n0, dims[1] = n1, dims[2] = n2, dims[3] = nv;
    strides[0] = n0 * 8ull, strides[1] = n0 * n1 * 8ull, strides[2] = cs;
    box[0] = a.ta, box[1] = d == 1 ? sb : 1, box[2] = d == 1 ? 1 : sb, box[3] = nv;
    a.tma_box = sb;
  }
  for (int k = 0; k < rank - 1; ++k)
    if (strides[k] % 16 != 0) return false;
  if (reinterpret_cast<uintptr_t>(u_in) % 16 != 0) return false;
  unsigned long long bytes = 8;
  for (int k = 0; k < rank; ++k) bytes *= box[k];
  a.tma_bytes = (unsigned)bytes;
  a.tma_raw_bytes = (int)((bytes + 127) / 128 * 128);
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, rank, const_cast<double*>(u_in), dims,
                         strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    a.tma_box = 0, a.tma_bytes = 0, a.tma_raw_bytes = 0;
    return false;
  }
  return true;
}

// list: a stepping sweep (stage 0..2) of a context that uses the re-decision
// list; the pass is launched right after the sweep (after recording
// after_sweep, when given).
// The arguments of a sweep of axis d with tiles of ta lines x ts cells.
enoao_status fill_sweep_args(enoao_ctx* c, int d, int stage, int mode, const double* u_in,
                             double* u_out, double* fhat, int8_t* idx, bool list, int ta, int ts,
                             SweepArgs& a) {
  memset(&a, 0, sizeof a);
  if (list) {
    a.redo = c->redo;
    a.redo_dc = c->redo_dc;
    a.redo_mark = c->redo_mark;
    a.redo_cap = c->redo_cap;
    a.redo_coef = stage == 0 ? 1.0 : (stage == 1 ? 0.25 : 2.0 / 3.0);
  }
  a.u_in = u_in;
  a.u0 = c->U[0];
  a.u_out = u_out;
  a.rhs = c->rhs;
  // FP32 bulk: stage 0 writes I0, stage 1 reads I0 and writes I1, stage 2 reads I1
  a.inc_in = stage == 0 ? nullptr : c->inc[stage - 1];
  a.inc_out = stage == 2 ? nullptr : c->inc[stage];
  a.fhat = fhat;
  a.idx_out = idx;
  a.st = c->st;
  for (int k = 0; k < 3; ++k) {
    a.n[k] = c->cfg.n[k];
    a.dx_all[k] = c->dx[k];
  }
  a.ncell = c->ncell;
  a.cstride = c->carr;
  a.org = c->org;
  a.ndim = c->cfg.ndim;
  a.dir = d;
  a.bc = c->sub && d == c->cfg.ndim - 1 ? kBcHalo : c->cfg.bc[d];
  a.mode = mode;
  a.stage = stage;
  a.ta = ta;
  a.ts = ts;
  a.se = sweep_row_pitch(c->nv, c->cfg.order, fp32(c), d, a.ta, a.ts);
  const long long nd = c->cfg.n[d];
  a.nfaces = c->ncell / nd * (nd + 1);
  a.tiles_s = (nd + a.ts - 1) / a.ts;
  if (d == 0) {
    const long long rows = c->cfg.n[1] * c->cfg.n[2];
    a.tiles_a = (rows + a.ta - 1) / a.ta;
    a.tiles_b = 1;
  } else {
    a.tiles_a = (c->cfg.n[0] + a.ta - 1) / a.ta;
    a.tiles_b = d == 1 ? c->cfg.n[2] : c->cfg.n[1];
  }
  a.ntiles = a.tiles_s * a.tiles_a * a.tiles_b;
  if (a.ntiles >= (1ll << 31)) return fail(c, ENOAO_EINVAL, "too many tiles for axis %d", d);
  a.inv_dx = 1.0 / c->dx[d];
  a.gamma = c->cfg.gamma;
  a.adv_speed = c->cfg.adv_speed;
  a.delta = c->cfg.delta;
  a.tie_rel = c->cfg.tie_rel;
  set_derived_constants(a);
  a.redo_passes = c->redo_passes >= 0 ? c->redo_passes : 64 * c->nv;
  return ENOAO_OK;
}

enoao_status launch_sweep(enoao_ctx* c, int d, int stage, int mode, const double* u_in,
                          double* u_out, double* fhat, int8_t* idx, bool list = false,
                          cudaEvent_t after_sweep = nullptr) {
  SweepArgs a;
  enoao_status r0 = fill_sweep_args(c, d, stage, mode, u_in, u_out, fhat, idx, list, c->ta[d],
                                    c->ts[d], a);
  if (r0 != ENOAO_OK) return r0;
  CUtensorMap tmap;
  const size_t smem0 = sweep_smem_bytes(c->nv, c->cfg.order, fp32(c), a.ta, a.ts, a.se);
  bool tma = encode_tile_map(c, d, list, u_in, a, &tmap);
  if (tma && smem0 + (size_t)a.tma_raw_bytes > 200 * 1024) tma = false;  // no room for the box
  const size_t smem = smem0 + (tma ? (size_t)a.tma_raw_bytes : 0);
  const int block = c->block[d];
  int per_sm = 1;
  cudaError_t e;
  const int nv = c->nv, order = c->cfg.order;
  a.field = consts(c).field;
  if (fp32(c)) {
    // ENO-AO5 tiles that let seven (or eight) blocks share an SM take the
    // LEAN kernel (re-decisions out of line, 64 registers); measured faster there
    if (!a.field && !list && !tma && order == 5 && smem * 7 <= 220 * 1024) {
      int lean_per_sm = 0;
      if (sweep_configure_fp32(nv, order, smem, 2) == cudaSuccess &&
          sweep_occupancy_fp32(nv, order, block, smem, &lean_per_sm, 2) == cudaSuccess &&
          lean_per_sm >= 7)
        a.lean = 1;
      cudaGetLastError();
    }
    const int variant = tma ? 1 : (a.lean ? 2 : 0);
    e = a.field ? sweep_configure_fp32_field(nv, order, smem)
                : sweep_configure_fp32(nv, order, smem, variant);
    if (e == cudaSuccess)
      e = a.field ? sweep_occupancy_fp32_field(nv, order, block, smem, &per_sm)
                  : sweep_occupancy_fp32(nv, order, block, smem, &per_sm, variant);
  } else {
    e = a.field ? sweep_configure_fp64_field(nv, order, smem) : sweep_configure_fp64(nv, order, smem);
    if (e == cudaSuccess)
      e = a.field ? sweep_occupancy_fp64_field(nv, order, block, smem, &per_sm)
                  : sweep_occupancy_fp64(nv, order, block, smem, &per_sm);
  }
  if (e != cudaSuccess) return fail(c, ENOAO_ECUDA, "sweep setup: %s", cudaGetErrorString(e));
  if (per_sm < 1) return fail(c, ENOAO_EINVAL, "sweep tile does not fit on an SM");
  long long grid = std::min<long long>(a.ntiles, (long long)c->sms * per_sm);
  if (grid < 1) grid = 1;
  if (a.field)
    e = fp32(c) ? sweep_launch_fp32_field(nv, order, a, (int)grid, block, smem, c->s)
                : sweep_launch_fp64_field(nv, order, a, (int)grid, block, smem, c->s);
  else
    e = fp32(c) ? sweep_launch_fp32(nv, order, a, (int)grid, block, smem, c->s,
                                    tma ? &tmap : nullptr)
                : sweep_launch_fp64(nv, order, a, (int)grid, block, smem, c->s);
  if (e != cudaSuccess) return fail(c, ENOAO_ECUDA, "sweep launch: %s", cudaGetErrorString(e));
  if (after_sweep) CU(c, cudaEventRecord(after_sweep, c->s));
  if (list) {
    e = redo_launch_fp32(c->nv, c->cfg.order, a, c->sms * 8, c->s);
    if (e != cudaSuccess) return fail(c, ENOAO_ECUDA, "re-decision pass: %s", cudaGetErrorString(e));
  }
  return ENOAO_OK;
}

// One Runge-Kutta stage: every axis, the last one combining.
bool per_stage_alpha(const enoao_ctx* c) {
  return c->cfg.system == ENOAO_EULER && c->cfg.alpha_mode == ENOAO_ALPHA_PER_STAGE;
}

// Whether a stage of this context runs as one fused 2D launch: asked for,
// 2D, FP32 bulk, one alpha, in-sweep re-decisions, no TMA staging, a whole
// grid (not a sub-domain), and a system the fused kernel is built for.
bool fused_stage(const enoao_ctx* c) {
  return c->fused && c->cfg.ndim == 2 && fp32(c) && !use_list(c) && !consts(c).field && !c->tma &&
         !c->sub && (c->nv == 1 || c->nv == 4) && (c->cfg.order == 5 || c->cfg.order == 7);
}

// One stage as one launch of fused2d_kernel: the x part with tiles of
// fused_tiles[0] rows x fused_tiles[1] cells, the y part with tiles of
// fused_tiles[2] columns x fused_tiles[3] cells, on 2D tiles of
// fused_tiles[1] x fused_tiles[3] cells.
enoao_status launch_fused_stage(enoao_ctx* c, int stage, const double* in, double* out,
                                bool want_alpha) {
  const int* ft = c->fused_tiles;
  SweepArgs ax, ay;
  enoao_status r = fill_sweep_args(c, 0, stage, kModeRhsStore, in, out, nullptr, nullptr, false,
                                   ft[0], ft[1], ax);
  if (r != ENOAO_OK) return r;
  r = fill_sweep_args(c, 1, stage, kModeCombine | kModeRhsAdd | (want_alpha ? kModeAlpha : 0), in,
                      out, nullptr, nullptr, false, ft[2], ft[3], ay);
  if (r != ENOAO_OK) return r;
  const int nv = c->nv, order = c->cfg.order, block = 128;
  const size_t sx = sweep_smem_bytes(nv, order, true, ax.ta, ax.ts, ax.se);
  const size_t sy = sweep_smem_bytes(nv, order, true, ay.ta, ay.ts, ay.se);
  const size_t smem = sx > sy ? sx : sy;
  int lean = 0, per_sm = 0;
  if (order == 5 && smem * 7 <= 220 * 1024) {
    int p = 0;
    if (fused2d_configure_fp32(nv, order, smem, 1) == cudaSuccess &&
        fused2d_occupancy_fp32(nv, order, block, smem, &p, 1) == cudaSuccess && p >= 7)
      lean = 1;
    cudaGetLastError();
  }
  cudaError_t e = fused2d_configure_fp32(nv, order, smem, lean);
  if (e == cudaSuccess) e = fused2d_occupancy_fp32(nv, order, block, smem, &per_sm, lean);
  if (e != cudaSuccess) return fail(c, ENOAO_ECUDA, "fused stage setup: %s", cudaGetErrorString(e));
  if (per_sm < 1) return fail(c, ENOAO_EINVAL, "fused stage tiles do not fit on an SM");
  const long long tiles = ax.tiles_s * ay.tiles_s;
  long long grid = std::min<long long>(tiles, (long long)c->sms * per_sm);
  if (grid < 1) grid = 1;
  e = fused2d_launch_fp32(nv, order, ax, ay, (int)grid, block, smem, c->s, lean);
  if (e != cudaSuccess) return fail(c, ENOAO_ECUDA, "fused stage launch: %s", cudaGetErrorString(e));
  return ENOAO_OK;
}

enoao_status enqueue_stage(enoao_ctx* c, int stage) {
  const double* in = c->U[stage];                 // U^n, U1, U2
  double* out = c->U[stage == 2 ? 0 : stage + 1];  // U1, U2, U^{n+1}
  const int nd = c->cfg.ndim;
  if (stage > 0 && per_stage_alpha(c)) {
    stage_alpha_kernel<<<1, 1, 0, c->s>>>(c->st, consts(c));
    CU(c, cudaGetLastError());
  }
  // alpha of the written state: for the next step (stage 2), or for the next
  // stage when each stage takes its own
  const bool want_alpha = stage == 2 || per_stage_alpha(c);
  if (fused_stage(c)) return launch_fused_stage(c, stage, in, out, want_alpha);
  const bool list = use_list(c);
  if (list && !c->redo) return fail(c, ENOAO_ENOMEM, "re-decision list not allocated");
  for (int d = 0; d < nd; ++d) {
    int mode;
    if (d < nd - 1)
      mode = kModeRhsStore | (d > 0 ? kModeRhsAdd : 0);
    else
      mode = kModeCombine | (nd > 1 ? kModeRhsAdd : 0) | (want_alpha ? kModeAlpha : 0);
    enoao_status r = launch_sweep(c, d, stage, mode, in, out, nullptr, nullptr, list);
    if (r != ENOAO_OK) return r;
  }
  return ENOAO_OK;
}

enoao_status enqueue_step(enoao_ctx* c) {
  step_begin_kernel<<<1, 1, 0, c->s>>>(c->st, consts(c));
  CU(c, cudaGetLastError());
  for (int s = 0; s < 3; ++s) {
    enoao_status r = enqueue_stage(c, s);
    if (r != ENOAO_OK) return r;
  }
  return ENOAO_OK;
}

// Stream ordering against the caller's stream.
enoao_status enter(enoao_ctx* c) {
  CU(c, cudaSetDevice(c->device));
  CU(c, cudaEventRecord(c->ev_a, c->user));
  CU(c, cudaStreamWaitEvent(c->s, c->ev_a, 0));
  return ENOAO_OK;
}
enoao_status leave(enoao_ctx* c) {
  CU(c, cudaEventRecord(c->ev_b, c->s));
  CU(c, cudaStreamWaitEvent(c->user, c->ev_b, 0));
  return ENOAO_OK;
}

enoao_status build_graph(enoao_ctx* c, int steps) {
  if (c->graph && c->graph_steps == steps) return ENOAO_OK;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  cudaGraph_t g;
  CU(c, cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal));
  enoao_status r = ENOAO_OK;
  for (int k = 0; k < steps && r == ENOAO_OK; ++k) r = enqueue_step(c);
  if (r == ENOAO_OK) {
    finalize_kernel<<<1, 1, 0, c->s>>>(c->st);
  }
  cudaError_t e = cudaStreamEndCapture(c->s, &g);
  if (r != ENOAO_OK) return r;
  if (e != cudaSuccess) return fail(c, ENOAO_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(c, ENOAO_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  c->graph_steps = steps;
  return ENOAO_OK;
}

int steps_per_graph(const enoao_ctx* c) {
  // small problems are launch-bound: replay many steps per graph
  return c->ncell < (1ll << 16) ? 32 : (c->ncell < (1ll << 22) ? 8 : 4);
}

enoao_status read_host_state(enoao_ctx* c) {
  CU(c, cudaMemcpyAsync(c->st_host, c->st, sizeof(StepState), cudaMemcpyDeviceToHost, c->s));
  CU(c, cudaStreamSynchronize(c->s));
  return ENOAO_OK;
}

enoao_status check_err(enoao_ctx* c) {
  if (c->st_host->err & kErrNonPhys)
    return fail(c, ENOAO_ENONPHYS, "non-physical state (rho <= 0, p <= 0 or NaN) at cell %lld",
                (long long)c->st_host->err_cell);
  if (c->st_host->err & kErrTimeout) return fail(c, ENOAO_ETIMEOUT, "device wait timed out");
  if (c->st_host->err & kErrRedoFull)
    return fail(c, ENOAO_ECUDA, "internal error: re-decision list overflow");
  return ENOAO_OK;
}

// Copies the interior of a state array from (in) or to the caller's buffer
// ([nv][ncell], contiguous): one 2D copy, component rows carr apart in the array.
enoao_status copy_interior(enoao_ctx* c, double* arr, const double* user_in, int on_device, bool in) {
  const size_t w = (size_t)c->ncell * sizeof(double), pitch = (size_t)c->carr * sizeof(double);
  double* user = const_cast<double*>(user_in);
  if (in)
    CU(c, cudaMemcpy2DAsync(arr + c->org, pitch, user, w, w, c->nv,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->s));
  else
    CU(c, cudaMemcpy2DAsync(user, w, arr + c->org, pitch, w, c->nv,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->s));
  return ENOAO_OK;
}


}  // namespace

// ====================================================================== C ABI

extern "C" {

void enoao_config_default(enoao_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof *cfg);
  cfg->ndim = 1;
  cfg->system = ENOAO_EULER;
  cfg->order = 5;
  cfg->precision = ENOAO_FP64;
  for (int d = 0; d < 3; ++d) {
    cfg->n[d] = 1;
    cfg->lo[d] = 0.0;
    cfg->hi[d] = 1.0;
    cfg->bc[d] = ENOAO_PERIODIC;
  }
  cfg->adv_speed = 1.0;
  cfg->gamma = 1.4;
  cfg->delta = 1e-5;
  cfg->tie_rel = 1e-3;
}

const char* enoao_last_error(const enoao_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

static enoao_status validate(const enoao_config* cfg, bool batched) {
  if (!cfg) return fail(nullptr, ENOAO_EINVAL, "config is NULL");
  if (cfg->ndim < 1 || cfg->ndim > 3) return fail(nullptr, ENOAO_EINVAL, "ndim must be 1, 2 or 3");
  if (cfg->system != ENOAO_EULER && cfg->system != ENOAO_SCALAR_ADVECTION)
    return fail(nullptr, ENOAO_EINVAL, "unknown system %d", cfg->system);
  if (cfg->order != 5 && cfg->order != 7) return fail(nullptr, ENOAO_EINVAL, "order must be 5 or 7");
  if (cfg->precision != ENOAO_FP64 && cfg->precision != ENOAO_FP32_BULK)
    return fail(nullptr, ENOAO_EINVAL, "unknown precision %d", cfg->precision);
  if (batched && cfg->ndim != 1)
    return fail(nullptr, ENOAO_EINVAL, "batched problems must be one-dimensional");
  for (int d = 0; d < 3; ++d) {
    if (d < cfg->ndim) {
      if (!batched && cfg->n[d] < 2 * halo(cfg->order) + 1)
        return fail(nullptr, ENOAO_EINVAL, "axis %d has %lld cells; at least %d are needed", d,
                    (long long)cfg->n[d], 2 * halo(cfg->order) + 1);
      if (!batched && !(cfg->hi[d] > cfg->lo[d]))
        return fail(nullptr, ENOAO_EINVAL, "axis %d: hi must exceed lo", d);
      if (cfg->bc[d] != ENOAO_PERIODIC && cfg->bc[d] != ENOAO_TRANSMISSIVE)
        return fail(nullptr, ENOAO_EINVAL, "axis %d: unknown boundary condition", d);
    } else if (cfg->n[d] != 1) {
      return fail(nullptr, ENOAO_EINVAL, "unused axis %d must have n = 1", d);
    }
  }
  if (cfg->system == ENOAO_EULER && !(cfg->gamma > 1.0))
    return fail(nullptr, ENOAO_EINVAL, "gamma must exceed 1");
  if (!(cfg->delta >= 0.0)) return fail(nullptr, ENOAO_EINVAL, "delta must be >= 0");
  if (!(cfg->tie_rel >= 0.0)) return fail(nullptr, ENOAO_EINVAL, "tie_rel must be >= 0");
  if (cfg->alpha_mode != ENOAO_ALPHA_PER_STEP && cfg->alpha_mode != ENOAO_ALPHA_PER_STAGE &&
      cfg->alpha_mode != ENOAO_ALPHA_PER_FIELD)
    return fail(nullptr, ENOAO_EINVAL,
                "alpha_mode must be ENOAO_ALPHA_PER_STEP, _PER_STAGE or _PER_FIELD");
  if (batched && cfg->alpha_mode == ENOAO_ALPHA_PER_FIELD)
    return fail(nullptr, ENOAO_EINVAL, "per-field alpha is not available for batched contexts");
  return ENOAO_OK;
}

static enoao_status create_common(const enoao_config* cfg, void* stream, enoao_ctx** out,
                                  bool batched, long long ghost_layer_cells = 0) {
  enoao_ctx* c = new (std::nothrow) enoao_ctx;
  if (!c) return fail(nullptr, ENOAO_ENOMEM, "host allocation failed");
  c->cfg = *cfg;
  c->nv = cfg->system == ENOAO_EULER ? cfg->ndim + 2 : 1;
  c->user = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_a, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_b, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&c->t0);
  if (e == cudaSuccess) e = cudaEventCreate(&c->t1);
  if (e == cudaSuccess) e = cudaMalloc(&c->st, sizeof(StepState));
  if (e == cudaSuccess) e = cudaMallocHost(&c->st_host, sizeof(StepState));
  if (e != cudaSuccess) {
    enoao_status r = fail(nullptr, ENOAO_ECUDA, "context setup: %s", cudaGetErrorString(e));
    enoao_destroy(c);
    return r;
  }
  if (!batched) {
    c->ncell = cfg->n[0] * cfg->n[1] * cfg->n[2];
    // ghost layers of a sub-domain: halo() layers on each side of the split axis
    c->org = ghost_layer_cells;
    c->carr = c->ncell + 2 * ghost_layer_cells;
    for (int d = 0; d < 3; ++d) c->dx[d] = d < cfg->ndim ? (cfg->hi[d] - cfg->lo[d]) / cfg->n[d] : 1.0;
    const size_t bytes = (size_t)c->nv * c->carr * sizeof(double);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaMalloc(&c->U[k], bytes);
    if (e == cudaSuccess && cfg->ndim > 1)
      e = cudaMalloc(&c->rhs, (size_t)c->nv * c->carr * (fp32(c) ? 4 : 8));
    for (int k = 0; k < 2 && e == cudaSuccess && fp32(c); ++k)
      e = cudaMalloc(&c->inc[k], (size_t)c->nv * c->carr * sizeof(float));
    if (e != cudaSuccess) {
      enoao_status r = fail(nullptr, e == cudaErrorMemoryAllocation ? ENOAO_ENOMEM : ENOAO_ECUDA,
                            "device allocation of %zu bytes per state failed: %s", bytes,
                            cudaGetErrorString(e));
      enoao_destroy(c);
      return r;
    }
    default_tiles(c);
    enoao_status r = ensure_list(c);
    if (r != ENOAO_OK) {
      g_create_error = c->err;
      enoao_destroy(c);
      return r;
    }
  }
  reset_state_kernel<<<1, 1, 0, c->s>>>(c->st);
  e = cudaStreamSynchronize(c->s);
  if (e != cudaSuccess) {
    enoao_status r = fail(nullptr, ENOAO_ECUDA, "context setup: %s", cudaGetErrorString(e));
    enoao_destroy(c);
    return r;
  }
  *out = c;
  return ENOAO_OK;
}

enoao_status enoao_create(const enoao_config* cfg, void* cuda_stream, enoao_ctx** out) {
  if (!out) return fail(nullptr, ENOAO_EINVAL, "out is NULL");
  *out = nullptr;
  enoao_status r = validate(cfg, false);
  if (r != ENOAO_OK) return r;
  return create_common(cfg, cuda_stream, out, false);
}

enoao_status enoao_create_subdomain(const enoao_config* global, int64_t offset, int64_t n_local,
                                    void* cuda_stream, enoao_ctx** out) {
  if (!out) return fail(nullptr, ENOAO_EINVAL, "out is NULL");
  *out = nullptr;
  enoao_status r = validate(global, false);
  if (r != ENOAO_OK) return r;
  if (global->ndim < 2)
    return fail(nullptr, ENOAO_EINVAL, "sub-domains split 2D or 3D grids along their last axis");
  if (global->alpha_mode != ENOAO_ALPHA_PER_STEP)
    return fail(nullptr, ENOAO_EINVAL, "sub-domains take one alpha per step (ENOAO_ALPHA_PER_STEP)");
  const int last = global->ndim - 1, G = halo(global->order);
  if (offset < 0 || n_local < G || offset + n_local > global->n[last])
    return fail(nullptr, ENOAO_EINVAL,
                "layers [%lld, %lld) are not a sub-domain of %lld layers with at least %d of its own",
                (long long)offset, (long long)(offset + n_local), (long long)global->n[last], G);
  enoao_config local = *global;
  local.n[last] = n_local;
  long long plane = 1;
  for (int d = 0; d < last; ++d) plane *= global->n[d];
  enoao_ctx* c = nullptr;
  r = create_common(&local, cuda_stream, &c, false, G * plane);
  if (r != ENOAO_OK) return r;
  c->sub = 1;
  c->plane = plane;
  c->sub_off = offset;
  c->sub_bc = global->bc[last];
  for (int d = 0; d < global->ndim; ++d)  // the global spacing, bit for bit
    c->dx[d] = (global->hi[d] - global->lo[d]) / global->n[d];
  *out = c;
  return ENOAO_OK;
}

// Halo layers of a sub-domain: the caller's buffer holds [nv][G][plane]
// (layers in increasing index order).  Export takes the G interior layers
// next to side (0: low, 1: high) of stage state k; import writes the G ghost
// layers beyond that side.
static enoao_status halo_copy(enoao_ctx* c, int k, int side, double* buf, int on_device, bool out) {
  if (!c) return fail(c, ENOAO_EINVAL, "NULL context");
  if (!c->sub) return fail(c, ENOAO_EINVAL, "not a sub-domain context");
  if (k < 0 || k > 2 || (side != 0 && side != 1) || !buf)
    return fail(c, ENOAO_EINVAL, "stage state k must be 0..2, side 0 or 1, buffer non-NULL");
  const int G = halo(c->cfg.order);
  const long long nl = c->cfg.n[c->cfg.ndim - 1];
  long long at;  // first array cell of the G layers
  if (out)
    at = c->org + (side == 0 ? 0 : (nl - G) * c->plane);
  else
    at = side == 0 ? 0 : c->org + nl * c->plane;
  const size_t w = (size_t)G * c->plane * sizeof(double), pitch = (size_t)c->carr * sizeof(double);
  enoao_status r = enter(c);
  if (r != ENOAO_OK) return r;
  if (out)
    CU(c, cudaMemcpy2DAsync(buf, w, c->U[k] + at, pitch, w, c->nv,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->s));
  else
    CU(c, cudaMemcpy2DAsync(c->U[k] + at, pitch, buf, w, w, c->nv,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->s));
  r = leave(c);
  if (r != ENOAO_OK) return r;
  CU(c, cudaStreamSynchronize(c->s));
  return ENOAO_OK;
}

enoao_status enoao_halo_export(enoao_ctx* c, int k, int side, double* buf, int on_device) {
  return halo_copy(c, k, side, buf, on_device, true);
}

enoao_status enoao_halo_import(enoao_ctx* c, int k, int side, const double* buf, int on_device) {
  return halo_copy(c, k, side, const_cast<double*>(buf), on_device, false);
}

enoao_status enoao_halo_fill_transmissive(enoao_ctx* c, int k, int side) {
  if (!c) return fail(c, ENOAO_EINVAL, "NULL context");
  if (!c->sub) return fail(c, ENOAO_EINVAL, "not a sub-domain context");
  if (k < 0 || k > 2 || (side != 0 && side != 1))
    return fail(c, ENOAO_EINVAL, "stage state k must be 0..2 and side 0 or 1");
  const int G = halo(c->cfg.order);
  const long long nl = c->cfg.n[c->cfg.ndim - 1];
  // zero-gradient ghosts: every ghost layer is a copy of the edge layer
  const long long edge = c->org + (side == 0 ? 0 : (nl - 1) * c->plane);
  const size_t w = (size_t)c->plane * sizeof(double), pitch = (size_t)c->carr * sizeof(double);
  enoao_status r = enter(c);
  if (r != ENOAO_OK) return r;
  for (int g = 0; g < G; ++g) {
    const long long at = side == 0 ? g * c->plane : c->org + (nl + g) * c->plane;
    CU(c, cudaMemcpy2DAsync(c->U[k] + at, pitch, c->U[k] + edge, pitch, w, c->nv,
                            cudaMemcpyDeviceToDevice, c->s));
  }
  r = leave(c);
  if (r != ENOAO_OK) return r;
  CU(c, cudaStreamSynchronize(c->s));
  return ENOAO_OK;
}

enoao_status enoao_local_alpha(enoao_ctx* c, double* alpha) {
  if (!c || !alpha) return fail(c, ENOAO_EINVAL, "NULL argument");
  if (c->batch) return fail(c, ENOAO_EINVAL, "not available for batched contexts");
  enoao_status r = read_host_state(c);
  if (r != ENOAO_OK) return r;
  r = check_err(c);
  if (r != ENOAO_OK) return r;
  const int cur = (int)(c->st_host->steps & 1);
  for (int d = 0; d < 3; ++d)
    alpha[d] = d < c->cfg.ndim && c->cfg.system == ENOAO_EULER
                   ? __builtin_bit_cast(double, c->st_host->alpha_acc[cur][d])
                   : (d < c->cfg.ndim ? std::fabs(c->cfg.adv_speed) : 0.0);
  return ENOAO_OK;
}

enoao_status enoao_set_step_alpha(enoao_ctx* c, const double* alpha) {
  if (!c || !alpha) return fail(c, ENOAO_EINVAL, "NULL argument");
  if (c->batch) return fail(c, ENOAO_EINVAL, "not available for batched contexts");
  if (c->cfg.alpha_mode != ENOAO_ALPHA_PER_STEP)
    return fail(c, ENOAO_EINVAL, "a step alpha can be set with ENOAO_ALPHA_PER_STEP only");
  for (int d = 0; d < c->cfg.ndim; ++d)
    if (!(alpha[d] >= 0.0) || !std::isfinite(alpha[d]))
      return fail(c, ENOAO_EINVAL, "alpha must be finite and >= 0");
  enoao_status r = read_host_state(c);
  if (r != ENOAO_OK) return r;
  const int cur = (int)(c->st_host->steps & 1);
  unsigned long long bits[3] = {0ull, 0ull, 0ull};
  for (int d = 0; d < c->cfg.ndim; ++d) bits[d] = __builtin_bit_cast(unsigned long long, alpha[d]);
  r = enter(c);
  if (r != ENOAO_OK) return r;
  std::memcpy(c->st_host->alpha_acc[cur], bits, sizeof bits);  // pinned staging
  CU(c, cudaMemcpyAsync(&c->st->alpha_acc[cur][0], c->st_host->alpha_acc[cur], sizeof bits,
                        cudaMemcpyHostToDevice, c->s));
  r = leave(c);
  if (r != ENOAO_OK) return r;
  CU(c, cudaStreamSynchronize(c->s));
  return ENOAO_OK;
}

enoao_status enoao_batch_create(const enoao_config* proto, int nprob, const int64_t* n,
                                const double* lo, const double* hi, void* cuda_stream,
                                enoao_ctx** out) {
  if (!out) return fail(nullptr, ENOAO_EINVAL, "out is NULL");
  *out = nullptr;
  enoao_status r = validate(proto, true);
  if (r != ENOAO_OK) return r;
  if (nprob < 1 || !n || !lo || !hi) return fail(nullptr, ENOAO_EINVAL, "empty batch");
  enoao_ctx* c = nullptr;
  r = create_common(proto, cuda_stream, &c, true);
  if (r != ENOAO_OK) return r;
  r = batch_create(c, proto, nprob, n, lo, hi);
  if (r != ENOAO_OK) {
    g_create_error = c->err;
    enoao_destroy(c);
    return r;
  }
  *out = c;
  return ENOAO_OK;
}

void enoao_destroy(enoao_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->s) cudaStreamSynchronize(c->s);
  if (c->batch) batch_destroy(c->batch);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (int k = 0; k < 3; ++k) cudaFree(c->U[k]);
  cudaFree(c->rhs);
  for (int k = 0; k < 2; ++k) cudaFree(c->inc[k]);
  cudaFree(c->flux_scratch);
  cudaFree(c->idx_scratch);
  cudaFree(c->redo);
  cudaFree(c->redo_dc);
  cudaFree(c->redo_mark);
  cudaFree(c->st);
  if (c->st_host) cudaFreeHost(c->st_host);
  if (c->ev_a) cudaEventDestroy(c->ev_a);
  if (c->ev_b) cudaEventDestroy(c->ev_b);
  if (c->t0) cudaEventDestroy(c->t0);
  if (c->t1) cudaEventDestroy(c->t1);
  if (c->s) cudaStreamDestroy(c->s);
  delete c;
}

enoao_status enoao_init_state(enoao_ctx* c, const double* U, int on_device) {
  if (!c || !U) return fail(c, ENOAO_EINVAL, "NULL argument");
  if (c->batch) return batch_init_state(c, U, on_device);
  enoao_status r = enter(c);
  if (r != ENOAO_OK) return r;
  r = copy_interior(c, c->U[0], U, on_device, true);
  if (r != ENOAO_OK) return r;
  reset_state_kernel<<<1, 1, 0, c->s>>>(c->st);
  if (c->cfg.system == ENOAO_EULER) {
    const int blocks = std::max(1, std::min<int>((int)((c->ncell + 255) / 256), c->sms * 8));
    launch_alpha(c->nv, c->U[0] + c->org, c->ncell, c->carr, c->cfg.gamma, c->st, 0, fp32(c),
                 consts(c).field != 0, blocks, c->s);
  }
  CU(c, cudaGetLastError());
  r = leave(c);
  if (r != ENOAO_OK) return r;
  r = read_host_state(c);
  if (r != ENOAO_OK) return r;
  return check_err(c);
}

enoao_status enoao_get_state(enoao_ctx* c, double* U, int on_device) {
  if (!c || !U) return fail(c, ENOAO_EINVAL, "NULL argument");
  if (c->batch) return batch_get_state(c, U, on_device);
  enoao_status r = enter(c);
  if (r != ENOAO_OK) return r;
  r = copy_interior(c, c->U[0], U, on_device, false);
  if (r != ENOAO_OK) return r;
  r = leave(c);
  if (r != ENOAO_OK) return r;
  CU(c, cudaStreamSynchronize(c->s));
  return ENOAO_OK;
}

enoao_status enoao_get_stage_state(enoao_ctx* c, int k, double* U, int on_device) {
  if (!c || !U) return fail(c, ENOAO_EINVAL, "NULL argument");
  if (c->batch) return fail(c, ENOAO_EINVAL, "not available for batched contexts");
  if (k < 0 || k > 2) return fail(c, ENOAO_EINVAL, "stage state k must be 0, 1 or 2");
  enoao_status r = enter(c);
  if (r != ENOAO_OK) return r;
  r = copy_interior(c, c->U[k], U, on_device, false);
  if (r != ENOAO_OK) return r;
  r = leave(c);
  if (r != ENOAO_OK) return r;
  CU(c, cudaStreamSynchronize(c->s));
  return ENOAO_OK;
}

enoao_status enoao_reconstruct_fluxes(enoao_ctx* c, int dir, double* Fhat, int8_t* idx,
                                      int on_device) {
  if (!c || !Fhat) return fail(c, ENOAO_EINVAL, "NULL argument");
  if (c->batch) return fail(c, ENOAO_EINVAL, "not available for batched contexts");
  if (dir < 0 || dir >= c->cfg.ndim) return fail(c, ENOAO_EINVAL, "dir out of range");
  const long long nf = c->ncell / c->cfg.n[dir] * (c->cfg.n[dir] + 1);
  const size_t fbytes = (size_t)c->nv * nf * sizeof(double);
  const size_t ibytes = (size_t)c->nv * 2 * nf;
  double* dF = Fhat;
  int8_t* dI = idx;
  if (!on_device) {
    // device scratch kept in the context: allocated by the first call that
    // needs it (or more of it), freed by enoao_destroy
    if (c->flux_scratch_bytes < fbytes) {
      cudaFree(c->flux_scratch);
      c->flux_scratch = nullptr;
      c->flux_scratch_bytes = 0;
      if (cudaMalloc(&c->flux_scratch, fbytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, ENOAO_ENOMEM, "flux scratch allocation of %zu bytes failed", fbytes);
      }
      c->flux_scratch_bytes = fbytes;
    }
    if (idx && c->idx_scratch_bytes < ibytes) {
      cudaFree(c->idx_scratch);
      c->idx_scratch = nullptr;
      c->idx_scratch_bytes = 0;
      if (cudaMalloc(&c->idx_scratch, ibytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, ENOAO_ENOMEM, "choice scratch allocation of %zu bytes failed", ibytes);
      }
      c->idx_scratch_bytes = ibytes;
    }
    dF = c->flux_scratch;
    dI = idx ? c->idx_scratch : nullptr;
  }
  enoao_status r = enter(c);
  if (r == ENOAO_OK) {
    alpha_current_kernel<<<1, 1, 0, c->s>>>(c->st, consts(c));
    r = launch_sweep(c, dir, 0, kModeFlux, c->U[0], nullptr, dF, dI);
  }
  if (r == ENOAO_OK && !on_device) {
    cudaError_t e = cudaMemcpyAsync(Fhat, dF, fbytes, cudaMemcpyDeviceToHost, c->s);
    if (e == cudaSuccess && idx) e = cudaMemcpyAsync(idx, dI, ibytes, cudaMemcpyDeviceToHost, c->s);
    if (e != cudaSuccess) r = fail(c, ENOAO_ECUDA, "copy out: %s", cudaGetErrorString(e));
  }
  if (r == ENOAO_OK) r = leave(c);
  cudaError_t e = cudaStreamSynchronize(c->s);
  if (r != ENOAO_OK) return r;
  if (e != cudaSuccess) return fail(c, ENOAO_ECUDA, "reconstruct_fluxes: %s", cudaGetErrorString(e));
  return ENOAO_OK;
}

enoao_status enoao_rk_stage(enoao_ctx* c, int stage, double dt) {
  if (!c) return fail(c, ENOAO_EINVAL, "NULL context");
  if (c->batch) return fail(c, ENOAO_EINVAL, "not available for batched contexts");
  if (stage < 0 || stage > 2) return fail(c, ENOAO_EINVAL, "stage must be 0, 1 or 2");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, ENOAO_EINVAL, "dt must be positive");
  enoao_status r = enter(c);
  if (r != ENOAO_OK) return r;
  manual_stage_kernel<<<1, 1, 0, c->s>>>(c->st, consts(c), stage, dt);
  CU(c, cudaGetLastError());
  r = enqueue_stage(c, stage);
  if (r != ENOAO_OK) return r;
  if (stage == 2) finalize_kernel<<<1, 1, 0, c->s>>>(c->st);
  r = leave(c);
  if (r != ENOAO_OK) return r;
  if (stage == 2) {
    r = read_host_state(c);
    if (r != ENOAO_OK) return r;
    return check_err(c);
  }
  return ENOAO_OK;
}

static enoao_status run_graph_steps(enoao_ctx* c, double t_end, double cfl, double dt_fixed,
                                    long long max_steps, bool until_time, bool sync) {
  if (c->sub)
    return fail(c, ENOAO_EINVAL,
                "a sub-domain steps stage by stage (enoao_rk_stage) between halo exchanges");
  enoao_status r = enter(c);
  if (r != ENOAO_OK) return r;
  r = build_graph(c, steps_per_graph(c));
  if (r != ENOAO_OK) return r;
  CU(c, cudaMemcpyAsync(c->st_host, c->st, sizeof(StepState), cudaMemcpyDeviceToHost, c->s));
  CU(c, cudaStreamSynchronize(c->s));
  const long long start = c->st_host->steps;
  const long long limit = max_steps > 0 ? start + max_steps : 0;
  set_run_kernel<<<1, 1, 0, c->s>>>(c->st, t_end, cfl, dt_fixed, limit);
  CU(c, cudaGetLastError());
  if (!until_time) {
    const long long reps = (max_steps + c->graph_steps - 1) / c->graph_steps;
    for (long long k = 0; k < reps; ++k) CU(c, cudaGraphLaunch(c->graph, c->s));
  } else {
    for (;;) {
      for (int k = 0; k < 4; ++k) CU(c, cudaGraphLaunch(c->graph, c->s));
      r = read_host_state(c);
      if (r != ENOAO_OK) return r;
      if (c->st_host->done || c->st_host->err) break;
      if (limit > 0 && c->st_host->steps >= limit) break;
    }
  }
  r = leave(c);
  if (r != ENOAO_OK) return r;
  if (!sync) return ENOAO_OK;
  r = read_host_state(c);
  if (r != ENOAO_OK) return r;
  return check_err(c);
}

enoao_status enoao_advance(enoao_ctx* c, double t_end, double cfl, double dt_fixed,
                           int64_t max_steps, double* t_out, int64_t* steps_out) {
  if (!c) return fail(c, ENOAO_EINVAL, "NULL context");
  if (c->batch) return fail(c, ENOAO_EINVAL, "use enoao_advance_steps for batched contexts");
  if (!(dt_fixed > 0.0) && !(cfl > 0.0)) return fail(c, ENOAO_EINVAL, "cfl must be positive");
  if (!(t_end >= 0.0)) return fail(c, ENOAO_EINVAL, "t_end must be >= 0");
  enoao_status r = run_graph_steps(c, t_end, cfl, dt_fixed, max_steps, true, true);
  if (t_out) *t_out = c->st_host->t;
  if (steps_out) *steps_out = c->st_host->steps;
  return r;
}

enoao_status enoao_advance_steps_async(enoao_ctx* c, int64_t nsteps, double cfl) {
  if (!c) return fail(c, ENOAO_EINVAL, "NULL context");
  if (!(cfl > 0.0)) return fail(c, ENOAO_EINVAL, "cfl must be positive");
  if (nsteps < 0) return fail(c, ENOAO_EINVAL, "nsteps must be >= 0");
  if (nsteps == 0) return ENOAO_OK;
  if (c->batch) return batch_advance(c, nsteps, cfl, false);
  return run_graph_steps(c, kInf, cfl, 0.0, nsteps, false, false);
}

enoao_status enoao_advance_steps(enoao_ctx* c, int64_t nsteps, double cfl) {
  enoao_status r = enoao_advance_steps_async(c, nsteps, cfl);
  if (r != ENOAO_OK) return r;
  return enoao_sync(c);
}

enoao_status enoao_sync(enoao_ctx* c) {
  if (!c) return fail(c, ENOAO_EINVAL, "NULL context");
  enoao_status r = read_host_state(c);
  if (r != ENOAO_OK) return r;
  return check_err(c);
}

enoao_status enoao_get_stats(enoao_ctx* c, enoao_stats* out) {
  if (!c || !out) return fail(c, ENOAO_EINVAL, "NULL argument");
  if (c->batch) return batch_stats(c, out);
  enoao_status r = read_host_state(c);
  if (r != ENOAO_OK) return r;
  const StepState& h = *c->st_host;
  out->t = h.pending ? (h.last ? h.t_end : h.t + h.dt) : h.t;
  out->steps = h.steps + (h.pending ? 1 : 0);
  for (int d = 0; d < 3; ++d) out->alpha[d] = h.alpha[d];
  out->dt = h.dt;
  out->fp64_fallbacks = h.fallbacks;
  out->decisions = h.decisions;
  return ENOAO_OK;
}

int enoao_launches_per_step(const enoao_ctx* c) {
  if (!c) return 0;
  if (c->batch) return 0;  // one persistent launch covers every step
  return 1 + 3 * c->cfg.ndim * (use_list(c) ? 3 : 1) + (per_stage_alpha(c) ? 2 : 0);
}

enoao_status enoao_set_redecide(enoao_ctx* c, int mode) {
  if (!c) return fail(c, ENOAO_EINVAL, "NULL context");
  if (mode != ENOAO_REDECIDE_AUTO && mode != ENOAO_REDECIDE_IN_SWEEP && mode != ENOAO_REDECIDE_GRID)
    return fail(c, ENOAO_EINVAL, "re-decision mode must be AUTO, IN_SWEEP or GRID");
  if (c->batch && mode == ENOAO_REDECIDE_GRID)
    return fail(c, ENOAO_EINVAL, "batched contexts re-decide inside the sweep");
  const int prev = c->redecide;
  c->redecide = mode;
  enoao_status r = ensure_list(c);
  if (r != ENOAO_OK) {
    c->redecide = prev;
    return r;
  }
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return ENOAO_OK;
}

int enoao_uses_grid_redecide(const enoao_ctx* c) { return c && use_list(c) ? 1 : 0; }

enoao_status enoao_set_tma(enoao_ctx* c, int on) {
  if (!c) return fail(c, ENOAO_EINVAL, "NULL context");
  c->tma = on ? 1 : 0;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return ENOAO_OK;
}

enoao_status enoao_set_fused_stage(enoao_ctx* c, int on, int x_lines, int x_cells, int y_lines,
                                   int y_cells) {
  if (!c) return fail(c, ENOAO_EINVAL, "NULL context");
  if (c->batch) return fail(c, ENOAO_EINVAL, "not available for batched contexts");
  if (on != 0 && on != 1) return fail(c, ENOAO_EINVAL, "on must be 0 or 1");
  if (on) {
    if (c->cfg.ndim != 2) return fail(c, ENOAO_EINVAL, "the fused stage is for 2D problems");
    if (x_lines == 0 && x_cells == 0 && y_lines == 0 && y_cells == 0) {
      x_lines = c->fused_tiles[0], x_cells = c->fused_tiles[1];
      y_lines = c->fused_tiles[2], y_cells = c->fused_tiles[3];
    }
    enoao_status r = check_tiles(c, 0, x_lines, x_cells);
    if (r != ENOAO_OK) return r;
    r = check_tiles(c, 1, y_lines, y_cells);
    if (r != ENOAO_OK) return r;
    if (y_cells % x_lines != 0 || x_cells % y_lines != 0)
      return fail(c, ENOAO_EINVAL,
                  "fused tiles: y cells (%d) must be a multiple of x lines (%d) and x cells (%d) "
                  "of y lines (%d)",
                  y_cells, x_lines, x_cells, y_lines);
    c->fused_tiles[0] = x_lines, c->fused_tiles[1] = x_cells;
    c->fused_tiles[2] = y_lines, c->fused_tiles[3] = y_cells;
  }
  c->fused = on;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return ENOAO_OK;
}

enoao_status enoao_set_redecide_pass_limit(enoao_ctx* c, int passes) {
  if (!c) return fail(c, ENOAO_EINVAL, "NULL context");
  if (c->batch) return fail(c, ENOAO_EINVAL, "not available for batched contexts");
  if (passes < -1) return fail(c, ENOAO_EINVAL, "pass limit must be >= 0, or -1 for the default");
  c->redo_passes = passes;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return ENOAO_OK;
}

enoao_status enoao_set_tiles(enoao_ctx* c, int dir, int ta, int ts) {
  if (!c) return fail(c, ENOAO_EINVAL, "NULL context");
  if (c->batch || dir < 0 || dir >= c->cfg.ndim) return fail(c, ENOAO_EINVAL, "dir out of range");
  if (ta == 0) ta = c->ta[dir];
  if (ts == 0) ts = c->ts[dir];
  enoao_status r = check_tiles(c, dir, ta, ts);
  if (r != ENOAO_OK) return r;
  c->ta[dir] = ta;
  c->ts[dir] = ts;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return ENOAO_OK;
}

enoao_status enoao_get_tiles(const enoao_ctx* c, int dir, int* ta, int* ts) {
  if (!c || dir < 0 || dir >= 3) return ENOAO_EINVAL;
  if (ta) *ta = c->ta[dir];
  if (ts) *ts = c->ts[dir];
  return ENOAO_OK;
}

enoao_status enoao_time_sweep(enoao_ctx* c, int dir, int nrep, float* ms) {
  if (!c || !ms) return fail(c, ENOAO_EINVAL, "NULL argument");
  if (c->batch || dir < 0 || dir >= c->cfg.ndim) return fail(c, ENOAO_EINVAL, "dir out of range");
  if (nrep < 1) return fail(c, ENOAO_EINVAL, "nrep must be >= 1");
  enoao_status r = enter(c);
  if (r != ENOAO_OK) return r;
  alpha_current_kernel<<<1, 1, 0, c->s>>>(c->st, consts(c));
  // the last axis combines; earlier axes store L(u) exactly as inside a step
  const int nd = c->cfg.ndim;
  const int mode = dir < nd - 1 ? (kModeRhsStore | (dir > 0 ? kModeRhsAdd : 0))
                                : (kModeCombine | (nd > 1 ? kModeRhsAdd : 0));
  // the sweep as steps launch it (with the re-decision pass after it, when
  // the context uses one; only the sweep kernel is timed)
  const bool list = use_list(c);
  r = launch_sweep(c, dir, 0, mode, c->U[0], c->U[1], nullptr, nullptr, list);  // warm-up
  if (r != ENOAO_OK) return r;
  float total = 0.f;
  for (int k = 0; k < nrep && r == ENOAO_OK; ++k) {
    CU(c, cudaEventRecord(c->t0, c->s));
    r = launch_sweep(c, dir, 0, mode, c->U[0], c->U[1], nullptr, nullptr, list, c->t1);
    if (r != ENOAO_OK) return r;
    CU(c, cudaEventSynchronize(c->t1));
    float one = 0.f;
    CU(c, cudaEventElapsedTime(&one, c->t0, c->t1));
    total += one;
  }
  CU(c, cudaStreamSynchronize(c->s));
  *ms = total / nrep;
  return leave(c);
}

enoao_status enoao_autotune(enoao_ctx* c) {
  if (!c) return fail(c, ENOAO_EINVAL, "NULL context");
  if (c->batch) return batch_autotune(c);
  // Save the state; time one stage-0 sweep per candidate on the live state.
  const size_t bytes = (size_t)c->nv * c->carr * sizeof(double);
  enoao_status r = enter(c);
  if (r != ENOAO_OK) return r;
  CU(c, cudaMemcpyAsync(c->U[2], c->U[0], bytes, cudaMemcpyDeviceToDevice, c->s));
  const bool f32 = fp32(c);
  const bool list = use_list(c);  // candidates timed with the pass steps launch after them
  for (int d = 0; d < c->cfg.ndim; ++d) {
    std::vector<std::pair<int, int>> cands;
    if (d == 0) {
      const int tas[] = {1, 2, 4, 8};
      const int tss[] = {31, 63, 127, 159, 191, 255};
      for (int ta : tas)
        for (int ts : tss)
          if (c->cfg.ndim > 1 || ta == 1) cands.push_back({ta, ts});
    } else {
      const int tas[] = {8, 16, 32, 64};
      const int tss[] = {7, 15, 23, 31, 47, 63};
      for (int ta : tas)
        for (int ts : tss) cands.push_back({ta, ts});
    }
    const int best_ta0 = c->ta[d], best_ts0 = c->ts[d];
    float best = 1e30f;
    int bta = best_ta0, bts = best_ts0;
    for (auto& p : cands) {
      if (check_tiles(c, d, p.first, p.second) != ENOAO_OK) continue;
      c->ta[d] = p.first;
      c->ts[d] = p.second;
      // the mode of the axis in a step's stage 0 (earlier axes store L(u), the
      // last adds it and combines into U1); the live state U^n is untouched
      const int nd = c->cfg.ndim;
      const int mode = d < nd - 1 ? (kModeRhsStore | (d > 0 ? kModeRhsAdd : 0))
                                  : (kModeCombine | (nd > 1 ? kModeRhsAdd : 0));
      alpha_current_kernel<<<1, 1, 0, c->s>>>(c->st, consts(c));
      r = launch_sweep(c, d, 0, mode, c->U[2], c->U[1], nullptr, nullptr, list);  // warm-up
      if (r != ENOAO_OK) continue;
      CU(c, cudaEventRecord(c->t0, c->s));
      for (int k = 0; k < 3; ++k)
        launch_sweep(c, d, 0, mode, c->U[2], c->U[1], nullptr, nullptr, list);
      CU(c, cudaEventRecord(c->t1, c->s));
      CU(c, cudaEventSynchronize(c->t1));
      float ms = 0.f;
      CU(c, cudaEventElapsedTime(&ms, c->t0, c->t1));
      if (ms < best) {
        best = ms;
        bta = p.first;
        bts = p.second;
      }
    }
    c->ta[d] = bta;
    c->ts[d] = bts;
    (void)f32;
  }
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->err.clear();
  r = leave(c);
  if (r != ENOAO_OK) return r;
  CU(c, cudaStreamSynchronize(c->s));
  return ENOAO_OK;
}

}  // extern "C"
