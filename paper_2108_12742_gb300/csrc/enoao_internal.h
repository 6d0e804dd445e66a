// Internal declarations shared by the host runtime and the kernels of the
// ENO-AO library (not part of the public C interface).
#pragma once

#include <cstdint>

namespace enoao {

constexpr int kMaxNv = 5;

// Device-resident time-stepping state.  Written by the step kernels, read by
// every sweep launch, so alpha and dt never travel to the host inside a step.
struct StepState {
  double alpha[3];          // Lax-Friedrichs alpha per axis of the current step
  double dt;                // current step size
  double t;                 // time at the start of the current step
  double t_end;             // target time of enoao_advance (inf for step counts)
  double cfl;               // CFL number (dt = cfl / sum alpha_d / dx_d)
  double dt_fixed;          // > 0: fixed step size instead of the CFL rule
  long long steps;          // completed steps
  long long max_steps;      // stop after this many steps (<= 0: none)
  int skip;                 // 1: the current step is not taken (done / limit)
  int last;                 // 1: the current step lands on t_end
  int done;                 // 1: t_end reached
  int pending;              // 1: a step was begun and is not yet finalised
  unsigned long long alpha_acc[2][3];  // running max of |u_d| + c (bit patterns);
                                       // step n reads [n % 2], its last stage fills [par]
  int par;                  // alpha_acc slot the current step's last stage fills
  int err;                  // error bits (kErrNonPhys, kErrTimeout, kErrRedoFull)
  long long err_cell;       // first cell (min index) that raised kErrNonPhys
  unsigned long long fallbacks;  // FP32-bulk decisions re-done in FP64
  unsigned long long decisions;  // stencil decisions taken
  unsigned long long tile_next;  // dynamic tile queue of the running sweep launch
  unsigned int blocks_done;      // blocks of the running sweep launch that have left it
  unsigned int redo_n;            // faces listed for FP64 re-decision by the running sweep
  unsigned long long alpha_stage[3];  // per-stage alpha: running max over the
                                      // state stage 0 or 1 writes (bit patterns)
  unsigned int redo_epoch;        // sweeps that listed faces: tags the changed-face marks
  unsigned int redo_done;         // blocks of the running apply pass that have left it
  // per-field alpha (Euler): per axis max |u_d - c|, max |u_d|, max |u_d + c|
  double alpha_f[3][3];                   // of the current step
  unsigned long long alpha_acc_f[2][3][3];  // running maxima (bit patterns), as alpha_acc
};


// Ghost cells along the split axis of a sub-domain are layers of the state
// arrays themselves (filled by halo exchange), read as they are.
constexpr int kBcHalo = 2;

constexpr int kErrNonPhys = 1;
constexpr int kErrTimeout = 2;
constexpr int kErrRedoFull = 4;  // re-decision list full (cannot happen: one slot per face)

// Modes of a sweep launch (bit set).
constexpr int kModeRhsStore = 1;   // write this axis' L(u) into rhs
constexpr int kModeRhsAdd = 2;     // add the stored rhs of earlier axes
constexpr int kModeCombine = 4;    // Runge-Kutta combine into u_out
constexpr int kModeAlpha = 8;      // accumulate alpha of u_out: for the next step
                                   // (stage 2) or the next stage (stages 0, 1)
constexpr int kModeFlux = 16;      // write interface fluxes (and choices)

struct SweepArgs {
  const double* u_in;   // U^(s): stencil source, [nv][N]
  const double* u0;     // U^n for the Runge-Kutta combine
  double* u_out;        // combined state
  void* rhs;            // accumulated L(u) of earlier axes ([nv][N], bulk type)
  const float* inc_in;  // FP32 bulk combine: the FP32 stage increment of the previous
                        // stage ([nv][N], stages 1 and 2: I0 = dt L(U^n), I1 = I0 + dt L(U1))
  float* inc_out;       // FP32 bulk combine: this stage's increment (stages 0 and 1)
  double* fhat;         // kModeFlux: interface fluxes [nv][faces]
  int8_t* idx_out;      // kModeFlux: choices [nv][2][faces] (nullable)
  unsigned long long* redo;  // FP32 bulk, stepping: faces listed for the grid-wide FP64
                        // re-decision pass (face index << 16 | flagged choices, bit
                        // field * 2 + sign), a slot per face of the axis; null: the
                        // sweep re-decides its near-ties itself
  float* redo_dc;       // per listed face: change of its correction C (nv, sweep order)
  unsigned* redo_mark;  // per face of the axis: redo_epoch when its correction changed
  double redo_coef;     // weight of dt L(u) in the stage's combine (1, 1/4, 2/3)
  long long redo_cap;   // slots of redo
  StepState* st;
  long long n[3];       // cells per axis
  long long ncell;      // total cells
  long long nfaces;     // faces of the swept axis, ncell / nd * (nd + 1) (flux output layout)
  long long cstride;    // distance between two conserved components in the state arrays
  long long org;        // array cell of the first interior cell (sub-domains keep ghost
                        // layers in their arrays along the split axis; 0 otherwise)
  int ndim;
  int dir;              // swept axis
  int bc;               // boundary condition along dir (kBcHalo: ghosts stored in the arrays)
  int mode;
  int stage;            // Runge-Kutta stage 0..2
  int ta, ts;           // tile: lines x faces
  int se;               // shared-memory row pitch in cells (sweep_row_pitch)
  int field;            // 1: per-field splitting constants (st->alpha_f), Euler only
  int lean;             // FP32 bulk, ENO-AO5, in-sweep re-decision: the seven-block variant
  int tma_box;          // TMA: box extent along the swept axis (cells, with alignment slack)
  unsigned tma_bytes;   // TMA: bytes of one box
  int tma_raw_bytes;    // TMA: shared memory reserved for the box (a multiple of 128)
  int redo_passes;      // FP32 bulk: bound on the in-sweep re-decision passes of a warp
                        // round; reaching it sets kErrTimeout (64 nv by default)
  long long tiles_s;    // tiles along dir
  long long tiles_a;    // tiles across the line index
  long long tiles_b;    // tiles along the remaining axis (dir != 0)
  long long ntiles;
  double inv_dx;        // 1 / dx along dir
  double dx_all[3];     // dx per axis (alpha accumulation needs none, kept for checks)
  double gamma;
  double adv_speed;
  double delta;
  double tie_rel;
  // gamma - 1 in FP64 and the constants in FP32 (FP32 bulk), set from the
  // fields above by set_derived_constants wherever they are set: kernels read
  // them from the parameter space instead of narrowing them themselves, which
  // the compiler may redo at every use (a conversion on the FP64 unit each).
  double gm1;
  float gm1_f, adv_f, delta_f, tie_rel_f, inv_dx_f;
};

// Derived constants of a SweepArgs (round to nearest, as the device would).
__host__ __device__ inline void set_derived_constants(SweepArgs& a) {
  a.gm1 = a.gamma - 1.0;
  a.gm1_f = (float)a.gm1;
  a.adv_f = (float)a.adv_speed;
  a.delta_f = (float)a.delta;
  a.tie_rel_f = (float)a.tie_rel;
  a.inv_dx_f = (float)a.inv_dx;
}

// Host-side entry points of the instantiation units (sweep_fp64.cu,
// sweep_fp32.cu); return cudaError_t values.
}  // namespace enoao
#include <cuda.h>
#include <cuda_runtime.h>
namespace enoao {
// tmap: the stencil source as a tensor map for TMA staging of raw tiles (FP32
// bulk sweeps that re-decide in the sweep), or NULL for direct loads.
cudaError_t sweep_launch_fp64(int nv, int order, const SweepArgs& a, int grid, int block,
                              size_t smem, cudaStream_t s);
cudaError_t sweep_launch_fp32(int nv, int order, const SweepArgs& a, int grid, int block,
                              size_t smem, cudaStream_t s, const CUtensorMap* tmap = nullptr);
cudaError_t sweep_configure_fp64(int nv, int order, size_t smem);
// variant: 0 the regular in-sweep / listing kernels, 1 TMA staging, 2 LEAN
cudaError_t sweep_configure_fp32(int nv, int order, size_t smem, int variant = 0);
cudaError_t sweep_occupancy_fp64(int nv, int order, int block, size_t smem, int* per_sm);
cudaError_t sweep_occupancy_fp32(int nv, int order, int block, size_t smem, int* per_sm,
                                 int variant = 0);
cudaError_t redo_launch_fp32(int nv, int order, const SweepArgs& a, int grid, cudaStream_t s);
// per-field splitting constants (a.field; Euler systems, nv 3..5)
cudaError_t sweep_launch_fp64_field(int nv, int order, const SweepArgs& a, int grid, int block,
                                    size_t smem, cudaStream_t s);
cudaError_t sweep_launch_fp32_field(int nv, int order, const SweepArgs& a, int grid, int block,
                                    size_t smem, cudaStream_t s);
cudaError_t sweep_configure_fp64_field(int nv, int order, size_t smem);
cudaError_t sweep_configure_fp32_field(int nv, int order, size_t smem);
cudaError_t sweep_occupancy_fp64_field(int nv, int order, int block, size_t smem, int* per_sm);
cudaError_t sweep_occupancy_fp32_field(int nv, int order, int block, size_t smem, int* per_sm);
// the fused 2D stage kernel (both axes in one launch; FP32 bulk, nv 1 or 4):
// ax the x sweep's arguments, ay the y sweep's; lean: the seven-block ENO-AO5 form
cudaError_t fused2d_launch_fp32(int nv, int order, const SweepArgs& ax, const SweepArgs& ay,
                                int grid, int block, size_t smem, cudaStream_t s, int lean);
cudaError_t fused2d_configure_fp32(int nv, int order, size_t smem, int lean);
cudaError_t fused2d_occupancy_fp32(int nv, int order, int block, size_t smem, int* per_sm,
                                   int lean);

// Raises a kernel's dynamic shared-memory limit to at least smem, never
// lowers it: the limit belongs to the kernel, not to one launch, and the
// axes and tiles of one kernel (and launches captured earlier into a graph)
// need different sizes.
template <typename Kernel>
cudaError_t raise_smem_limit(Kernel* kernel, size_t smem) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  if ((size_t)fa.maxDynamicSharedSizeBytes >= smem) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Dynamic shared memory of one sweep block: per extended cell, the split
// differences (2 nv), the face corrections (nv), the Roe ingredients (nv for
// the Euler equations) and, in FP32 bulk mode, one word of near-tie flags.
// Row pitch (cells) of a tile's shared-memory rows.  x sweeps read along a
// row (any pitch); y/z sweeps put lines on lanes, so the pitch must spread a
// warp's lanes over distinct banks: odd for 32- and 64-line tiles, for 8-byte
// elements and for FP32 four-component cells (one 16-byte vector per cell:
// each quarter-warp access then covers eight distinct 16-byte bank groups),
// 2 (mod 4) for other 16-line FP32 tiles (a warp spans two cells of 16 lines).
inline int sweep_row_pitch(int nv, int order, int fp32, int dir, int ta, int ts) {
  const int G = order / 2 + 2;
  int se = ts + 2 * G;
  if (dir == 0) return se;
  if (fp32 && ta == 16 && nv != 4) {
    while (se % 4 != 2) ++se;
  } else {
    if (se % 2 == 0) ++se;
  }
  return se;
}

inline size_t sweep_smem_bytes(int nv, int order, int fp32, int ta, int ts, int se) {
  (void)ts;
  const size_t cells = (size_t)ta * (size_t)se;
  const int per = 3 * nv + (nv > 1 ? nv : 0) + (fp32 ? 1 : 0);
  return cells * per * (fp32 ? 4 : 8);
}

}  // namespace enoao
