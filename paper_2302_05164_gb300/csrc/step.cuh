// Fused explicit step of the FP32 operator for one instance (kernels_step.cu); internal.
#pragma once

#include <utility>

#include "step_layout.hpp"
#include "vec_kernels.cuh"

namespace pbf {

// Programmatic dependent launch: wait for the previous kernel in the stream to complete (and
// its memory to be visible), and allow the next one to start its prologue.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependency_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }


// Patches of up to kStepCells cells (step_layout.hpp), built once per context on the host
// (cells consecutive in the global Morton order, patches numbered by decreasing work). Each patch lists its unique node
// slots: first the dofs of its cells and the masters of its hanging nodes, in ascending
// order, then its hanging nodes, padded to a multiple of 4 entries so that a block can load
// its list with 16-byte loads. Every dof is owned by exactly one patch, the first that lists
// it; the owner writes the dof's new state. A hanging slot stores (start << 5) | count of its
// constraint row in the patch's hanging table, whose entries give each master's shared-memory
// position and weight: hanging values and contributions never leave the block.
struct StepTables {
  int n_patches = 0;
  int max_nu32 = 0;               // longest slot list, rounded up to a multiple of 32
  int max_hent8 = 0;              // longest hanging table, rounded up to a multiple of 8
  int smem = 0;                   // dynamic shared memory per block (bytes)
  const int32_t* ptr = nullptr;   // [n_patches] start of each list in slot (a multiple of 4)
  const int4* cnt = nullptr;      // [n_patches] {dof slots, all slots, hanging table begin, end}
  const int32_t* slot = nullptr;  // dof d (bit 31: owned here) or a hanging row reference
  const int32_t* cell = nullptr;  // [n_patches][kStepCells] the cell of each lane, -1 if none
  const uint16_t* loc = nullptr;  // [n_patches][npc][kStepCells] shared position of each cell node
  const uint16_t* hloc = nullptr; // hanging tables: master positions ...
  const float* hw = nullptr;      // ... and constraint weights
};

// loc table, slot list, staged values and contributions, hanging tables
inline int step_smem_bytes(int npc, int max_nu32, int max_hent8) {
  return npc * kStepCells * 2 + max_nu32 * 3 * 4 + max_hent8 * (2 + 4);
}

// The fused sequence keeps the working state T - T_ref as an unevaluated pair hi + lo of two
// FP32 numbers (ff_add): hi is the state rounded to FP32, the value the FP32 operator reads.

// One step n of the fused sequence. The kernel first completes step n-1 on the fly:
// T_n = T_{n-1} + dt f_{n-1} / C~ for every slot it stages (the owner stores T_n), then
// accumulates f_n = f(T_n) (diffusion and surface laser) and clears the accumulator of step
// n+1. Three accumulators rotate so that no launch reads a buffer that it also writes.
struct StepState {
  const double* T0 = nullptr;     // step 0: the state T_0 as given (FP64)
  double off = 0.0;               // T_ref
  const float2* x_in = nullptr;   // T_{n-1} - T_ref as hi + lo (unused when first)
  float2* x_out = nullptr;        // T_n - T_ref (owned dofs written)
  const float* f_in = nullptr;    // f_{n-1} (unused when first)
  float* f_acc = nullptr;         // f_n, zero on entry
  float* f_clear = nullptr;       // set to zero on owned dofs (the accumulator of step n+1)
  const float* invC0x = nullptr;  // 1 / lumped capacity with the plain c; -1 at Dirichlet dofs
  NodalCap nc;
  float2 x_dir = {0.f, 0.f};      // T_D - T_ref as hi + lo
  float dt = 0.f;
  int first = 0;                  // step 0: T_0 is the state as given (no update)
  int has_loss = 0;               // radiation / evaporation on the top faces at T_n
  LossK loss;
};

// Model options of the fused step kernel (compile-time mask): the phase model's conductivity
// with its stored history, and the radiation / evaporation loss on top faces.
enum { kStepPhase = 1, kStepLoss = 2 };

// The update of one dof of the fused sequence (Dirichlet dofs, ic < 0, take x_dir).
template <int CAP>
__device__ __forceinline__ float2 euler_ff(float2 x, float fi, float ic, const NodalCap& nc, float2 x_dir, float dt) {
  if (ic < 0.f) return x_dir;
  return ff_add(x, increment_f32<CAP>(x.x, fi, 0.f, ic, nc, dt));
}

// Kernel launch with one optional attribute. attr_kind: 0 plain, 1 programmatic stream
// serialisation, 2 cooperative.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_ex(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, int attr_kind,
                      cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (attr_kind == 1) {
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
  } else {
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
  }
  cfg.attrs = attr_kind ? attr : nullptr;
  cfg.numAttrs = attr_kind ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}


// cap: CAP_CONST or CAP_NODAL. pdl: launch with programmatic stream serialisation, so that
// the block prologue (table loads) overlaps the tail of the previous kernel in the stream.
cudaError_t launch_step(const CellLaunch& L, const StepTables& t, const StepState& st, int cap, bool pdl,
                        cudaStream_t s);

// The lean form of the same step (kernels_step_lean.cu): patch tables read through L1, only
// the staged values and their sums in shared memory, launched with programmatic stream
// serialisation. min_blocks (kLeanForms) selects the register budget it was compiled for.
constexpr int kLeanForms[3] = {14, 12, 10};
cudaError_t launch_step_lean(const CellLaunch& L, const StepTables& t, const StepState& st, int cap, int form,
                             cudaStream_t s);

// Fused step of a batch (kernels_bstep.cu): one launch per step for all instances, state
// [n_dofs][batch] with the instance fastest, the previous step's update applied in the
// gather, hanging nodes resolved from the constraint rows, the laser spot computed on the
// device at *t0 + step dt64 (so that a chunk of steps replays as one graph).
struct BStepArgs {
  const double* T0 = nullptr;     // step 0: the state as given
  double off = 0.0;               // T_ref
  const float2* x_in = nullptr;   // T_{n-1} - T_ref as hi + lo
  float2* x_out = nullptr;        // T_n - T_ref (written by the owning cell)
  const float* f_in = nullptr;    // f_{n-1}
  float* f_acc = nullptr;         // f_n, zero on entry
  float* f_clear = nullptr;       // cleared by the owning cell (the accumulator of step n+1)
  const float* invC0x = nullptr;  // [n_dofs] 1 / lumped capacity with the plain c; -1 at Dirichlet dofs
  NodalCap nc;
  float2 x_dir = {0.f, 0.f};
  float dt = 0.f;
  int first = 0;
  const uint32_t* own = nullptr;  // [n_cells] bit a: this cell stores its node a's dof
  const LaserK* laser = nullptr;  // device copy of the segments (null: no laser)
  const double* t0 = nullptr;     // device scalar: the call's start time
  int step = 0;
  double dt64 = 0.0;
};
cudaError_t launch_bstep(const CellLaunch& L, const BStepArgs& A, int cap, cudaStream_t s);
// T = T_ref + x_in + dt f_in / C~ for n_dofs x B values, clearing f_in and f_other (nullable)
cudaError_t launch_bstep_final(int cap, int64_t n_dofs, int B, const float2* x_in, float* f_in, float* f_other,
                               const float* invC0x, const NodalCap& nc, float2 x_dir, float dt, double off, double* T,
                               cudaStream_t s);

// Persistent form: every step of a sequence in one cooperative launch, a grid-wide barrier
// between steps, the spot of each step computed on the device, and the last update applied
// by the owners after the last barrier (T written in FP64, f_{N-1} and f_{N-2} cleared).
constexpr unsigned kBarrierGroups = 64;
struct GridBarrier {
  unsigned count = 0, gen = 0, err = 0, pad = 0;  // err: a wait ran out of time (set once)
  struct alignas(128) Group {
    unsigned count = 0;
  } group[kBarrierGroups];  // first-level counters, one cache line each
};
struct PersistState {
  StepState st;             // constants; the per-step pointers rotate inside the kernel
  float2* x[2] = {nullptr, nullptr};
  float* f[3] = {nullptr, nullptr, nullptr};
  double* T = nullptr;      // state in (step 0, through st.T0) and out (after the last step)
  int nsteps = 0;
  double t0 = 0.0, dt64 = 0.0;
  LaserInline las;          // surface laser constants (spot and segment filled per step)
  LaserK laser;             // segments (n_seg = 0: no laser)
  GridBarrier* bar = nullptr;  // zeroed before the launch
  unsigned extra_arrivals = 0; // test hook: barriers wait for this many blocks more than launched
};
// blocks: set to the grid size used (all blocks resident; when that covers every patch, each
// block keeps its patch tables in shared memory for the whole sequence). Volumetric lasers
// are not covered.
cudaError_t launch_steps_persistent(const CellLaunch& L, const StepTables& t, const PersistState& ps, int cap,
                                    int* blocks, cudaStream_t s);

// The last update of a sequence, T = off + T_{N-1} + dt f_{N-1} / C~ (FP64 out), clearing f_in
// and f_other (nullable): afterwards all three accumulators are zero again.
cudaError_t launch_step_final(int cap, int64_t n_dofs, const float2* x_in, float* f_in, float* f_other,
                              const float* invC0x, const NodalCap& nc, float2 x_dir, float dt, double off, double* T,
                              cudaStream_t s);

}  // namespace pbf
