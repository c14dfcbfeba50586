// Context state shared by the C-ABI entry points (capi.cu) and the solvers (solver.cu).
#pragma once

#include <cuda_runtime.h>

#include <utility>
#include <vector>

#include "internal.cuh"
#include "mesh.hpp"
#include "pbf.h"
#include "step.cuh"
#include "vec_kernels.cuh"

namespace pbf {

pbf_status set_error(pbf_status s, const char* msg);

struct CtxBase;
// Set-up of pbf_estimate_dt_noalloc on the current device (noalloc.cu), run by
// pbf_ctx_create: after it the entry point allocates nothing.
pbf_status noalloc_prepare(CtxBase* ctx);

struct CtxBase {
  const HostMesh* mesh = nullptr;
  int64_t generation = 0;
  int degree = 1, npc = 8, batch = 1;
  int64_t n_dofs = 0, n_cells = 0, n_hang = 0, n_top = 0;
  bool f32 = false, nonlin = false, latent = false;
  int cap = 0;          // CAP_CONST, CAP_QUADRATURE or CAP_NODAL
  NodalCap nodal;
  pbf_material mat{};
  bool has_loss = false;  // radiation / evaporation on the top faces (pbf_ctx_set_surface_loss)
  LossK loss;
  bool has_phase = false;  // phase-dependent conductivity with history (pbf_ctx_set_phase)
  PhaseR<float> phf;
  PhaseR<double> phd;
  void* rc = nullptr;      // consolidated fraction [q][n_cells][batch], operator precision
  CellLaunch base;
  LaserSetup lsetup;
  std::vector<void*> allocs;
  // mesh tables
  int32_t* cell_dofs = nullptr;
  uint8_t* cell_level = nullptr;
  uint8_t* cell_mat = nullptr;
  int32_t* con_ptr = nullptr;
  int32_t* con_idx = nullptr;
  double* con_w = nullptr;
  float* con_wf = nullptr;
  uint8_t* dirichlet = nullptr;
  int32_t* top_cell = nullptr;
  double* top_geo = nullptr;
  double* cell_lo = nullptr;
  double* level_h = nullptr;
  uint8_t* cell_top = nullptr;
  // material / instance data
  double* k_scale_d = nullptr;
  float* k_scale_f = nullptr;
  std::vector<double> k_scale_host;
  double* power = nullptr;  // [batch][kMaxSeg]
  float* powerf = nullptr;  // the same in FP32
  float* cell_lof = nullptr;
  std::vector<double> power_host;
  // work space
  void* f = nullptr;     // operator accumulator (FP32 or FP64) [n_dofs][batch]
  void* fvol = nullptr;  // laser accumulator [n_dofs][batch]
  void* Cacc = nullptr;  // capacity accumulator (latent heat) [n_dofs][batch]
  float* Tf = nullptr;   // FP32 operator: working state T - T_ref rounded to FP32 [n_dofs][batch], gathered
  float* Tlo = nullptr;  // ... and the low part of the FP32 pair Tf + Tlo (explicit steps)
  void* xh = nullptr;    // input values at hanging nodes (FP32 or FP64) [n_hang][batch]
  double* xh64 = nullptr;  // FP64 hanging values for FP64-operator launches of an FP32 context
  void* fh = nullptr;    // operator accumulator at hanging nodes [n_hang][batch]
  void* Ch = nullptr;    // capacity accumulator at hanging nodes
  double* fh64 = nullptr;  // FP64 accumulators for FP64-operator launches of an FP32 context
  double* Ch64 = nullptr;
  // fused explicit step (one instance, FP32 operator): patch tables, the three rotating
  // accumulators (fstep[0] is f), the two working states as FP32 pairs hi + lo, and the
  // inverse constant-c capacity with -1 at Dirichlet dofs
  StepTables step;
  float* fstep[3] = {nullptr, nullptr, nullptr};
  float2* xstep[2] = {nullptr, nullptr};
  float* invC0_fx = nullptr;
  GridBarrier* bar = nullptr;  // grid barrier of the persistent form
  unsigned barrier_test_extra = 0;  // test hook (pbf_ctx_set_barrier_test)
  bool barrier_timed_out = false;   // the last persistent launch's barrier ran out of time
  // fused step of a batch (FP32 operator, batch > 1): owner bits per cell, two working
  // states as FP32 pairs and three rotating accumulators [n_dofs][batch], a device copy of
  // the laser segments, the call's start time in device memory, and the step sequence of
  // the last call replayed as one CUDA graph (rebuilt when its key changes)
  uint32_t* cell_own = nullptr;
  float2* xb[2] = {nullptr, nullptr};
  float* fb[3] = {nullptr, nullptr, nullptr};
  LaserK* laser_dev = nullptr;
  double* t0_dev = nullptr;
  double* C0 = nullptr;  // lumped capacity with the plain c [n_dofs]
  double* invC0_d = nullptr;
  float* invC0_f = nullptr;
  double* part = nullptr;  // reduction partials [reduction_blocks][batch]
  double* scal = nullptr;  // device scalars [batch][16]
  std::vector<double*> vec;  // FP64 work vectors [n_dofs][batch]
  // implicit-operator diagonal cache
  double* diag = nullptr;
  double diag_dt = -1.0;
  // launch sequences of the implicit solve replayed as CUDA graphs (the Chebyshev
  // preconditioner; one whole CG iteration): captured on a private stream, launched on the
  // caller's, rebuilt when their key (dt, bounds, degree, vectors, launch shape) changes
  static constexpr int kGraphKey = 17;
  struct GraphSlot {
    cudaGraphExec_t exec = nullptr;
    double key[kGraphKey] = {};
    long long launches = 0;
  };
  cudaStream_t cap_stream = nullptr;
  GraphSlot cheb_graph, iter_graph, bstep_graph;
  double* pinned = nullptr;  // page-locked host scalar: r.r of the last CG iteration
  // state
  bool poisoned = false;
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events, free_events;
  long long launches = 0;

  void set_material_constants(double dt);
  void release();
  pbf_status check_usable();
  pbf_status cuda(cudaError_t e, const char* what);
  pbf_status set_laser(const pbf_laser* ls, cudaStream_t s);
  pbf_status ensure_vectors(int n);
  cudaError_t dalloc_raw(double** p, size_t n);
  // One operator application: hanging values of the input, the cell kernel (timed when timing
  // is on), and the distribution of hanging-node contributions to their masters.
  // L.x (FP64) or L.xf (FP32) must be set; f and C (nullable) are the dof accumulators.
  cudaError_t apply_cell(CellLaunch L, void* f, void* C, int mode, cudaStream_t s);
  // f_diff, f_vol and C~ at T in FP64 (laser set beforehand; any output may be null)
  // fre (nullable): with a surface loss, its part goes there instead of into fv
  cudaError_t residual_f64(const double* T, double t, double* fd, double* fv, double* C, cudaStream_t s,
                           double* fre = nullptr);
  // nsteps forward-Euler steps in place on T (laser set beforehand); the fused form runs when
  // the context's shape is 4-9 (6: persistent, not with a volumetric source; 7-9: the lean
  // kernel) and fused_ok(4); shapes 6-9 run as 5 where fused_ok(shape) is false
  cudaError_t explicit_steps(double* T, double t0, double dt, int nsteps, cudaStream_t s);
  // lean: -1 the fused step kernel, 0..2 its lean form with the register budget kLeanForms[lean]
  cudaError_t explicit_steps_fused(double* T, double t0, double dt, int nsteps, bool pdl, int lean, cudaStream_t s);
  cudaError_t explicit_steps_persistent(double* T, double t0, double dt, int nsteps, cudaStream_t s);
  // the batched fused form: buffers allocated on first use; surface lasers only
  pbf_status ensure_bfused();
  cudaError_t explicit_steps_bfused(double* T, double t0, double dt, int nsteps, cudaStream_t s);
  bool bfused_ok() const {
    return f32 && batch > 1 && cap != CAP_QUADRATURE && !has_loss && !has_phase &&
           !(lsetup.k.n_seg > 0 && lsetup.k.volumetric);
  }
  // the fused forms of one instance: the fused step kernel (shapes 4, 5) also covers the phase
  // model and the surface loss, the persistent and lean forms (6-9) neither
  bool fused_ok(int variant) const {
    return f32 && batch == 1 && cap != CAP_QUADRATURE && step.n_patches > 0 &&
           (variant <= 5 || (!has_loss && !has_phase));
  }
  // the phase model's fields of a residual-mode launch (store: an explicit step)
  void set_phase(CellLaunch& L, bool store) const {
    L.phase = has_phase ? 1 : 0;
    L.phf = phf;
    L.phd = phd;
    L.rc_f32 = f32 ? 1 : 0;  // the history is kept in the context's precision
    L.rc_in = has_phase ? rc : nullptr;
    L.rc_out = has_phase && store ? rc : nullptr;
  }
  // the surface laser of the cell kernels at time t (off for the volumetric source)
  LaserInline inline_laser(double t, Spot* sp) const;
  // CUDA events around one timed launch (kernel timing on)
  std::pair<cudaEvent_t, cudaEvent_t> timing_begin(cudaStream_t s);
  void timing_end(const std::pair<cudaEvent_t, cudaEvent_t>& ev, cudaStream_t s);
  // adjoint work space
  int32_t* surf_idx = nullptr;
  double* surf_w = nullptr;
  int n_surf = 0;
  double surf_W = 0.0;
};

}  // namespace pbf
