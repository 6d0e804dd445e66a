// Context of the C interface (host side), shared by the runtime units.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "enoao.h"
#include "enoao_internal.h"

namespace enoao {
struct BatchState;
void batch_destroy(BatchState* b);
enoao_status batch_create(enoao_ctx* ctx, const enoao_config* proto, int nprob,
                          const int64_t* n, const double* lo, const double* hi);
enoao_status batch_advance(enoao_ctx* ctx, int64_t nsteps, double cfl, bool sync);
enoao_status batch_init_state(enoao_ctx* ctx, const double* U, int on_device);
enoao_status batch_get_state(enoao_ctx* ctx, double* U, int on_device);
enoao_status batch_stats(enoao_ctx* ctx, enoao_stats* out);
enoao_status batch_autotune(enoao_ctx* ctx);
}  // namespace enoao

struct enoao_ctx {
  enoao_config cfg{};
  int nv = 0;
  long long ncell = 0;
  double dx[3] = {1, 1, 1};
  cudaStream_t user = nullptr;   // caller's stream
  cudaStream_t s = nullptr;      // library stream (non-blocking, capturable)
  cudaEvent_t ev_a = nullptr, ev_b = nullptr, t0 = nullptr, t1 = nullptr;
  double* U[3] = {nullptr, nullptr, nullptr};  // U^n, U1, U2
  void* rhs = nullptr;
  float* inc[2] = {nullptr, nullptr};  // FP32 bulk: stage increments I0, I1 ([nv][carr])
  // fused 2D stage (enoao_set_fused_stage): on/off and the tiles of its two
  // parts (x: lines, cells; y: lines, cells)
  int fused = 0;
  int fused_tiles[4] = {4, 64, 8, 48};
  // device scratch of enoao_reconstruct_fluxes with host buffers (grown on demand)
  double* flux_scratch = nullptr;
  size_t flux_scratch_bytes = 0;
  int8_t* idx_scratch = nullptr;
  size_t idx_scratch_bytes = 0;
  enoao::StepState* st = nullptr;       // device
  enoao::StepState* st_host = nullptr;  // pinned mirror
  int ta[3] = {0, 0, 0}, ts[3] = {0, 0, 0}, block[3] = {128, 128, 128};
  int sms = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  std::string err;
  enoao::BatchState* batch = nullptr;
  int device = 0;
  // FP32 bulk: faces listed for the grid-wide FP64 re-decision pass
  int redecide = ENOAO_REDECIDE_AUTO;
  unsigned long long* redo = nullptr;  // a slot per face of the axis with most faces
  float* redo_dc = nullptr;            // nv per slot
  unsigned* redo_mark = nullptr;       // per face
  long long redo_cap = 0;
  int redo_passes = -1;                // in-sweep re-decision pass bound (-1: 64 nv)
  int tma = 0;                         // FP32 bulk: stage raw tiles by TMA where eligible
  // Arrays: carr cells per conserved component, the interior from cell org on.
  // A sub-domain (enoao_create_subdomain) owns layers [sub_off, sub_off + n[last])
  // of a grid split along its last axis and keeps halo() ghost layers on each
  // side of that axis in its arrays; otherwise carr = ncell and org = 0.
  long long carr = 0;
  long long org = 0;
  int sub = 0;
  long long plane = 0;    // cells of one layer across the split axis
  long long sub_off = 0;  // global index of the first interior layer
  int sub_bc = 0;         // the global boundary condition along the split axis
};
