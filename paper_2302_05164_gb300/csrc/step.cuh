// Fused explicit step of the FP32 operator for one instance (kernels_step.cu); internal.
#pragma once

#include "vec_kernels.cuh"

namespace pbf {

constexpr int kStepCells = 64;  // cells per patch = threads per block of the fused step kernel

// Patches of kStepCells consecutive (Z-order) cells, built once per context on the host. Each
// patch lists its unique node slots: first the dofs in ascending order, then the hanging
// nodes (as n_dofs + constraint row), padded to a multiple of 4 entries so that a block can
// load its list with 16-byte loads. Every dof is owned by exactly one patch, the first that
// lists it; the owner writes the dof's new state.
struct StepTables {
  int n_patches = 0;
  int max_nu4 = 0;                // longest list, rounded up to a multiple of 4
  int smem = 0;                   // dynamic shared memory per block (bytes)
  const int32_t* ptr = nullptr;   // [n_patches] start of each list in slot (a multiple of 4)
  const int2* cnt = nullptr;      // [n_patches] {dof slots, all slots}
  const int32_t* slot = nullptr;  // dof d or n_dofs + r; bit 31 set where this patch owns dof d
  const uint16_t* loc = nullptr;  // [n_patches][npc][kStepCells] list index of each cell node
};

// One step n of the fused sequence. The kernel first completes step n-1 on the fly:
// T_n = T_{n-1} + dt f_{n-1} / C~ for every slot it stages (the owner stores T_n), then
// accumulates f_n = f(T_n) (diffusion and surface laser) and clears the accumulator of step
// n+1. Three accumulators rotate so that no launch reads a buffer that it also writes.
struct StepState {
  const double* tw_in = nullptr;  // T_{n-1} - T_ref (n = 0: T_0 - T_ref)
  double* tw_out = nullptr;       // T_n - T_ref (owned dofs written)
  const float* f_in = nullptr;    // f_{n-1} (unused when first)
  float* f_acc = nullptr;         // f_n, zero on entry
  float* f_clear = nullptr;       // set to zero on owned dofs (the accumulator of step n+1)
  const float* invC0 = nullptr;   // 1 / lumped capacity with the plain c
  NodalCap nc;
  double tw_dir = 0.0;            // T_D - T_ref
  float dt = 0.f;
  int first = 0;                  // step 0: T_0 is the state as given (no update)
};

// cap: CAP_CONST or CAP_NODAL. pdl: launch with programmatic stream serialisation, so that
// the block prologue (table loads) overlaps the tail of the previous kernel in the stream.
cudaError_t launch_step(const CellLaunch& L, const StepTables& t, const StepState& st, int cap, bool pdl,
                        cudaStream_t s);

// The last update of a sequence, T = T_ref + T_{N-1} + dt f_{N-1} / C~ (FP64 out), clearing
// f_in and f_other (nullable): afterwards all three accumulators are zero again.
cudaError_t launch_step_final(int cap, int64_t n_dofs, const double* tw_in, float* f_in, float* f_other,
                              const float* invC0, const uint8_t* dirichlet, const NodalCap& nc, double tw_dir, float dt,
                              double off, double* T, cudaStream_t s);

}  // namespace pbf
