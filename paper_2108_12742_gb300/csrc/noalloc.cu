// One third-order TVD Runge-Kutta step of a 1D problem that allocates no
// memory: the two intermediate stage states and the step's device-side state
// live in one fixed, file-scope device array instead of cudaMalloc'd buffers.
//
// Who needs it: callers that own every byte of device memory up front and
// forbid libraries to allocate (an application that reserves the whole GPU
// for its own pool allocator, an embedded solver with a fixed memory budget),
// and time-stepping loops that cannot afford the device-wide implicit
// synchronisation that cudaMalloc / cudaFree may cause.  The caller passes the
// input and output states; everything else the step needs is in the array.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "enoao.h"
#include "enoao_internal.h"
#include "state_speed.cuh"

namespace enoao {
void set_thread_error(const char* msg);
}

using namespace enoao;

namespace {

// Largest problem the fixed array can hold: 2^18 cells of at most three
// conserved variables (1D Euler), two FP64 stage states and two FP32 stage
// increments -> 18 MiB of device memory on every GPU on which the library is
// loaded, held until the process exits.
constexpr long long kMaxCells = 1ll << 18;
constexpr int kMaxNv = 3;
constexpr long long kStateDoubles = kMaxNv * kMaxCells;
constexpr long long kStepStateDoubles = (sizeof(StepState) + sizeof(double) - 1) / sizeof(double);
static_assert(kStepStateDoubles <= 64, "StepState must fit its reserved slot");

// [U1 | U2 | I0 I1 (FP32) | StepState slot]
static __device__ __align__(256) double g_noalloc_scratch[3 * kStateDoubles + 64];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};  // device address of the array per device

enoao_status nofail(enoao_status st, const std::string& msg) {
  set_thread_error(msg.c_str());
  return st;
}

// Clears the step state and fixes alpha from U^n (max |u| + c, or |a| for
// scalar advection) and the caller's dt.
__global__ void noalloc_begin_kernel(StepState* st, double dt) {
  memset(st, 0, sizeof(StepState));
  st->err_cell = 0x7fffffffffffffffll;
  st->dt = dt;
  st->par = 1;
}

// alpha with the operations the regular path uses (state_speed.cuh): FP32
// bulk speeds for the step's U^n alpha in FP32 bulk (bulk = 1), FP64 speeds
// otherwise and for the per-stage alphas of both precisions.
__global__ void noalloc_alpha_kernel(const double* __restrict__ U, long long n, int nv,
                                     double gamma, double adv, StepState* st, int bulk) {
  double a = 0.0;
  if (nv == 1) {
    a = fabs(adv);
  } else {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
      const double u[3] = {U[i], U[n + i], U[2 * n + i]};
      double s[3];
      const bool ok = bulk ? speeds32<3, false>(u, gamma, s) : speeds64<3, false>(u, gamma, s);
      if (!ok) {
        atomicOr(&st->err, kErrNonPhys);
        atomicMin(&st->err_cell, i);
        continue;
      }
      a = fmax(a, s[0]);
    }
  }
  for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
  if ((threadIdx.x & 31) == 0 && a > 0.0)
    atomicMax(&st->alpha_acc[0][0], (unsigned long long)__double_as_longlong(a));
}

__global__ void noalloc_alpha_set_kernel(StepState* st) {
  st->alpha[0] = __longlong_as_double((long long)st->alpha_acc[0][0]);
  st->alpha_acc[0][0] = 0ull;  // ready for a per-stage alpha
}

// Device address of the fixed array on the current device, set up once per
// device (the first call on a device does it).
enoao_status scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nofail(ENOAO_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return nofail(ENOAO_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return nofail(ENOAO_ECUDA, std::string("cudaGetSymbolAddress of the fixed scratch array: ") +
                                     cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return ENOAO_OK;
}

}  // namespace

extern "C" enoao_status enoao_step_noalloc(const enoao_config* cfg, const double* U_in,
                                           double* U_out, double dt, void* cuda_stream) {
  if (!cfg || !U_in || !U_out) return nofail(ENOAO_EINVAL, "NULL argument");
  if (cfg->ndim != 1) return nofail(ENOAO_EINVAL, "enoao_step_noalloc takes 1D problems only");
  if (cfg->system != ENOAO_EULER && cfg->system != ENOAO_SCALAR_ADVECTION)
    return nofail(ENOAO_EINVAL, "unknown system");
  if (cfg->order != 5 && cfg->order != 7) return nofail(ENOAO_EINVAL, "order must be 5 or 7");
  if (cfg->precision != ENOAO_FP64 && cfg->precision != ENOAO_FP32_BULK)
    return nofail(ENOAO_EINVAL, "unknown precision");
  if (cfg->alpha_mode == ENOAO_ALPHA_PER_FIELD)
    return nofail(ENOAO_EINVAL, "per-field alpha is not available in the allocation-free step");
  if (cfg->alpha_mode != ENOAO_ALPHA_PER_STEP && cfg->alpha_mode != ENOAO_ALPHA_PER_STAGE)
    return nofail(ENOAO_EINVAL, "unknown alpha_mode");
  if (cfg->bc[0] != ENOAO_PERIODIC && cfg->bc[0] != ENOAO_TRANSMISSIVE)
    return nofail(ENOAO_EINVAL, "unknown boundary condition");
  const long long n = cfg->n[0];
  const int G = cfg->order / 2 + 2;
  if (n < 2 * G + 1)
    return nofail(ENOAO_EINVAL, "problem has " + std::to_string(n) + " cells; at least " +
                                    std::to_string(2 * G + 1) + " are needed");
  if (n > kMaxCells)
    return nofail(ENOAO_EINVAL, "problem has " + std::to_string(n) +
                                    " cells; enoao_step_noalloc holds at most " +
                                    std::to_string(kMaxCells) + " (use enoao_create instead)");
  if (!(cfg->hi[0] > cfg->lo[0])) return nofail(ENOAO_EINVAL, "hi must exceed lo");
  if (cfg->system == ENOAO_EULER && !(cfg->gamma > 1.0)) return nofail(ENOAO_EINVAL, "gamma must exceed 1");
  if (!(dt > 0.0)) return nofail(ENOAO_EINVAL, "dt must be positive");

  // both states must be device memory of the current device (a host pointer
  // handed to the kernels would fault or silently read the wrong memory)
  {
    int cur = 0;
    cudaError_t pe = cudaGetDevice(&cur);
    const double* ptrs[2] = {U_in, U_out};
    for (int k = 0; k < 2 && pe == cudaSuccess; ++k) {
      cudaPointerAttributes pa;
      pe = cudaPointerGetAttributes(&pa, ptrs[k]);
      if (pe != cudaSuccess) break;
      if ((pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) || pa.device != cur)
        return nofail(ENOAO_EINVAL, std::string(k ? "U_out" : "U_in") +
                                        " is not device memory of the current device");
    }
    if (pe != cudaSuccess)
      return nofail(ENOAO_ECUDA, std::string("pointer check: ") + cudaGetErrorString(pe));
  }
  double* scratch = nullptr;
  enoao_status r = scratch_for_current_device(&scratch);
  if (r != ENOAO_OK) return r;
  const int nv = cfg->system == ENOAO_EULER ? 3 : 1;
  double* U1 = scratch;
  double* U2 = scratch + kStateDoubles;
  float* I0 = reinterpret_cast<float*>(scratch + 2 * kStateDoubles);  // FP32 bulk increments
  float* I1 = I0 + kStateDoubles;
  StepState* st = reinterpret_cast<StepState*>(scratch + 3 * kStateDoubles);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

  noalloc_begin_kernel<<<1, 1, 0, s>>>(st, dt);
  const int ablocks = (int)std::min<long long>((n + 255) / 256, 64);
  noalloc_alpha_kernel<<<ablocks, 256, 0, s>>>(U_in, n, nv, cfg->gamma, cfg->adv_speed, st,
                                               cfg->precision == ENOAO_FP32_BULK);
  noalloc_alpha_set_kernel<<<1, 1, 0, s>>>(st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return nofail(ENOAO_ECUDA, std::string("launch: ") + cudaGetErrorString(e));

  const bool f32 = cfg->precision == ENOAO_FP32_BULK;
  SweepArgs a;
  memset(&a, 0, sizeof a);
  a.st = st;
  a.n[0] = n;
  a.n[1] = a.n[2] = 1;
  a.ncell = n;
  a.nfaces = n + 1;
  a.cstride = n;  // U1/U2 use the caller's layout [nv][n]
  a.ndim = 1;
  a.dir = 0;
  a.bc = cfg->bc[0];
  a.ta = 1;
  a.ts = f32 ? 127 : 63;
  a.se = sweep_row_pitch(nv, cfg->order, f32, 0, a.ta, a.ts);
  a.tiles_s = (n + a.ts - 1) / a.ts;
  a.tiles_a = a.tiles_b = 1;
  a.ntiles = a.tiles_s;
  a.inv_dx = 1.0 / ((cfg->hi[0] - cfg->lo[0]) / (double)n);
  a.gamma = cfg->gamma;
  a.adv_speed = cfg->adv_speed;
  a.delta = cfg->delta;
  a.tie_rel = cfg->tie_rel;
  set_derived_constants(a);
  a.redo_passes = 64 * nv;
  const size_t smem = sweep_smem_bytes(nv, cfg->order, f32, a.ta, a.ts, a.se);
  const int block = 128;
  int per_sm = 1;
  e = f32 ? sweep_configure_fp32(nv, cfg->order, smem) : sweep_configure_fp64(nv, cfg->order, smem);
  if (e == cudaSuccess)
    e = f32 ? sweep_occupancy_fp32(nv, cfg->order, block, smem, &per_sm)
            : sweep_occupancy_fp64(nv, cfg->order, block, smem, &per_sm);
  if (e != cudaSuccess) return nofail(ENOAO_ECUDA, std::string("sweep setup: ") + cudaGetErrorString(e));
  const int grid = (int)std::max<long long>(1, std::min<long long>(a.ntiles, (long long)sms * per_sm));
  // stage 0: U1 = U^n + dt L(U^n); stage 1: U2 = 3/4 U^n + 1/4 (U1 + dt L(U1));
  // stage 2: U_out = 1/3 U^n + 2/3 (U2 + dt L(U2))
  const double* ins[3] = {U_in, U1, U2};
  double* outs[3] = {U1, U2, U_out};
  const bool per_stage = nv > 1 && cfg->alpha_mode == ENOAO_ALPHA_PER_STAGE;
  for (int stage = 0; stage < 3; ++stage) {
    if (stage > 0 && per_stage) {
      // this stage splits with the alpha of its own input state
      noalloc_alpha_kernel<<<ablocks, 256, 0, s>>>(ins[stage], n, nv, cfg->gamma, cfg->adv_speed, st, 0);
      noalloc_alpha_set_kernel<<<1, 1, 0, s>>>(st);
    }
    a.u_in = ins[stage];
    a.u0 = U_in;
    a.u_out = outs[stage];
    a.inc_in = stage == 0 ? nullptr : (stage == 1 ? I0 : I1);
    a.inc_out = stage == 0 ? I0 : (stage == 1 ? I1 : nullptr);
    a.stage = stage;
    a.mode = kModeCombine;
    e = f32 ? sweep_launch_fp32(nv, cfg->order, a, grid, block, smem, s)
            : sweep_launch_fp64(nv, cfg->order, a, grid, block, smem, s);
    if (e != cudaSuccess) return nofail(ENOAO_ECUDA, std::string("sweep launch: ") + cudaGetErrorString(e));
  }
  int err = 0;
  long long cell = 0;
  e = cudaMemcpyAsync(&err, &st->err, sizeof err, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&cell, &st->err_cell, sizeof cell, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return nofail(ENOAO_ECUDA, std::string("step: ") + cudaGetErrorString(e));
  if (err & kErrNonPhys)
    return nofail(ENOAO_ENONPHYS, "non-physical state (rho <= 0, p <= 0 or NaN) at cell " +
                                      std::to_string(cell));
  if (err & kErrTimeout) return nofail(ENOAO_ETIMEOUT, "device wait timed out");
  if (err & kErrRedoFull) return nofail(ENOAO_ECUDA, "internal error: re-decision list overflow");
  return ENOAO_OK;
}
