// Patch layout of the fused explicit step, shared by the host-side table builder
// (step_tables.cpp, a plain C++ translation unit) and the kernels (step.cuh); internal.
#pragma once

#include <cstdint>
#include <vector>

#include "mesh.hpp"

#ifdef __CUDACC__
#define PBF_HOST_DEVICE __host__ __device__
#else
#define PBF_HOST_DEVICE
#endif

namespace pbf {

constexpr int kStepCells = 64;  // cells per patch = threads per block of the fused step kernel

// Shared-memory position of slot j of a patch: an XOR swizzle within each 32-slot block.
// Slots of consecutive Morton-order cells are about 8 apart (the new nodes per Q2 cell), so the
// same local node of the 32 cells of a warp would fall into 4 banks; the swizzle spreads them
// over all 32, and keeps a warp's 32 consecutive slots conflict-free.
PBF_HOST_DEVICE inline int step_swizzle(int j) { return j ^ ((j >> 5) & 31); }

// Patch tables of the fused step kernel, on the host. A patch is up to kStepCells cells that
// are consecutive in the global Morton order of their anchors (over the whole brick, not tree
// by tree), so that coarse regions give compact 4 x 4 x 4 blocks instead of rows of trees and a
// patch shares as few nodes as possible with its neighbours; a patch also holds at most
// kStepMaxHent hanging-table entries (step_tables.cpp). Each patch lists its unique node slots:
// the dofs of its cells and the masters of its hanging nodes, ascending, then its hanging
// nodes. Patches are numbered by decreasing work (slots plus twice the hanging-table entries),
// so the blocks of the expensive patches start first instead of forming the tail of a launch.
// Every dof is owned by the first patch in that numbering that lists it.
struct StepHost {
  std::vector<int32_t> ptr, cnt, slot, cell;
  std::vector<uint16_t> loc, hloc;
  std::vector<float> hw;
  int max_nu = 0, max_hent = 0;
};

// Builds the tables of mesh m (its independent per-patch work on all host cores); leaves
// `out` empty when the fused form does not apply (a dof without an owner, a constraint row of
// more than 31 entries, more than 65,536 slots in a patch).
void build_step_tables(const HostMesh& m, StepHost& out);

}  // namespace pbf
