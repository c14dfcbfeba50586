// Host-side canonical mesh of the library: a linear octree forest (Sec. 4.1 of the paper:
// octree refinement with 2:1 balance, Z-curve order, inactive cells above the active layer),
// dof numbering, hanging-node constraints, colouring, top faces and transfer maps.
#pragma once

#include <memory>

#include <cstdint>
#include <string>
#include <vector>

#include "pbf.h"

namespace pbf {

struct Octant {
  int64_t a[3];  // anchor on the lattice of finest cells
  int level;
};

// Sparse map old dofs -> new dofs (CSR over new dofs); an empty row takes `fill`.
struct TransferMap {
  bool pending = false;
  int64_t n_old = 0, n_new = 0;
  double fill = 0.0;
  std::vector<int32_t> ptr, idx;
  std::vector<double> w;
};

struct HostMesh {
  pbf_mesh_desc desc{};
  std::vector<uint8_t> exists;
  std::vector<pbf_region> regions;
  int p = 1, L = 0;
  int64_t ext[3] = {0, 0, 0};  // lattice extent in finest cells

  std::vector<Octant> oct;    // canonical order
  std::vector<uint64_t> key;  // global Morton key of each anchor (strictly increasing)
  // leaf holding each finest cell of the brick, x fastest (cells of trees that do not exist
  // are not written: locate checks inside() first); built after balancing when the brick has
  // at most kFineGridMax finest cells (null otherwise: locate searches the keys). Not
  // value-initialised, so that the parallel fill is the first touch of its pages.
  std::shared_ptr<int32_t[]> fine_leaf;
  static constexpr int64_t kFineGridMax = (int64_t)1 << 26;
  std::vector<uint8_t> active, material;
  std::vector<int32_t> active_of_leaf;  // leaf -> active index or -1
  std::vector<int32_t> leaf_of_active;

  int npc = 8;
  int64_t n_dofs = 0, n_colours = 0, n_top = 0;
  std::vector<int32_t> cell_dofs;  // [n_active][npc]
  std::vector<int32_t> con_ptr, con_idx;
  std::vector<double> con_w;
  std::vector<int64_t> hang_xyz, dof_xyz;
  std::vector<uint8_t> dirichlet, top;
  std::vector<int32_t> colour;

  int64_t generation = 0;
  TransferMap transfer;
  // history map of the last mesh change: for each active cell and quadrature point (x
  // fastest) the old cell * (p+1)^3 + old point it takes r_c from, or -1 (starts at 0: powder)
  // / -2 (starts at 1); history_old_cells: the old mesh's active cells (0: no map)
  std::vector<int32_t> history_map;
  int64_t history_old_cells = 0;

  int64_t size(const Octant& o) const { return (int64_t)1 << (L - o.level); }
  double coord(int axis, int64_t lattice) const;
  bool inside(const int64_t q[3]) const;  // inside the brick and in an existing tree
  uint64_t morton_key(const int64_t q[3]) const;
  int64_t locate(const int64_t q[3]) const;  // leaf holding finest cell q, or -1
};

// Builds everything from m.desc / m.exists / m.regions. `mat_hint` (nullable): material per
// leaf to keep instead of the powder-band rule. Returns PBF_OK or an error with *err set.
pbf_status build_mesh(HostMesh& m, const std::vector<uint8_t>* mat_hint, std::string* err);

// Sets up desc copies (regions, tree mask) and validates the descriptor.
pbf_status init_mesh(HostMesh& m, const pbf_mesh_desc& d, std::string* err);

// Interpolation map from the field of `old_m` to the dofs of `new_m` (same brick, degree and
// maximum level): dofs outside the old active domain get `fill`.
void make_transfer(const HostMesh& old_m, const HostMesh& new_m, double fill, TransferMap& out);

// History map of a mesh change (see HostMesh::history_map): each quadrature point of a new
// active cell takes the value of the nearest (per axis) quadrature point of the first old
// active cell, in cell order, whose closure holds it; points outside the old active domain
// start as a new cell does.
void make_history_map(const HostMesh& old_m, const HostMesh& new_m, std::vector<int32_t>& out);

// The coarsening restriction of Sec. 4.1 as pin regions: every active cell of m whose smallest
// consolidated fraction (rc_min, per active cell) lies below r_coarsen keeps its parent's box
// refined to its own level, so that its family of eight cannot merge.
void gate_pins(const HostMesh& m, const double* rc_min, double r_coarsen, std::vector<pbf_region>& out);

}  // namespace pbf
