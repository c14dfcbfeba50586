// Canonical mesh construction for the library (host C++).
//
// Design: a linear octree. Leaves are kept sorted by a global key (tree index, then the
// Morton interleave of the anchor inside the tree, x least significant), which is the
// paper's Z-curve order (Sec. 4.1). A lattice point is located by binary search on the
// keys. Nodes are grouped by sorting (node key, cell slot) pairs; hanging nodes are found by
// probing the leaves around each node. The rules reproduce the canonical specification of
// the repository exactly (bit for bit), including the floating-point geometry tests.
#include "mesh.hpp"

#ifdef _OPENMP
#include <omp.h>
#endif

#include <algorithm>
#ifdef _OPENMP
#include <parallel/algorithm>
#endif
#include <array>
#include <cmath>
#include <cstring>
#include <functional>

namespace pbf {

double HostMesh::coord(int axis, int64_t lattice) const {
  return desc.origin[axis] + desc.tree_h[axis] * ((double)lattice / (double)((int64_t)1 << L));
}

bool HostMesh::inside(const int64_t q[3]) const {
  for (int a = 0; a < 3; ++a)
    if (q[a] < 0 || q[a] >= ext[a]) return false;
  if (exists.empty()) return true;
  int64_t t = (q[0] >> L) + desc.ntree[0] * ((q[1] >> L) + (int64_t)desc.ntree[1] * (q[2] >> L));
  return exists[(size_t)t] != 0;
}

static inline uint64_t spread3(uint64_t v, int bits) {
  uint64_t r = 0;
  for (int b = 0; b < bits; ++b) r |= ((v >> b) & 1ull) << (3 * b);
  return r;
}

uint64_t HostMesh::morton_key(const int64_t q[3]) const {
  uint64_t t = (uint64_t)((q[0] >> L) + desc.ntree[0] * ((q[1] >> L) + (int64_t)desc.ntree[1] * (q[2] >> L)));
  uint64_t mask = ((uint64_t)1 << L) - 1;
  uint64_t m = spread3((uint64_t)q[0] & mask, L) | (spread3((uint64_t)q[1] & mask, L) << 1) |
               (spread3((uint64_t)q[2] & mask, L) << 2);
  return (t << (3 * L)) | m;
}

int64_t HostMesh::locate(const int64_t q[3]) const {
  if (!inside(q)) return -1;
  if (fine_leaf) return fine_leaf[(size_t)(q[0] + ext[0] * (q[1] + ext[1] * q[2]))];
  uint64_t k = morton_key(q);
  auto it = std::upper_bound(key.begin(), key.end(), k);
  if (it == key.begin()) return -1;
  int64_t i = (int64_t)(it - key.begin()) - 1;
  const Octant& o = oct[(size_t)i];
  int64_t s = size(o);
  for (int a = 0; a < 3; ++a)
    if (q[a] < o.a[a] || q[a] >= o.a[a] + s) return -1;
  return i;
}

pbf_status init_mesh(HostMesh& m, const pbf_mesh_desc& d, std::string* err) {
  if (d.degree != 1 && d.degree != 2) return *err = "degree must be 1 or 2", PBF_EINVAL;
  if (d.max_level < 0 || d.max_level > 12) return *err = "max_level must be in [0, 12]", PBF_EINVAL;
  for (int a = 0; a < 3; ++a) {
    if (d.ntree[a] < 1 || ((int64_t)d.ntree[a] << d.max_level) >= ((int64_t)1 << 20))
      return *err = "ntree out of range", PBF_EINVAL;
    if (!(d.tree_h[a] > 0.0)) return *err = "tree_h must be positive", PBF_EINVAL;
  }
  if (d.n_regions < 0 || (d.n_regions > 0 && !d.regions)) return *err = "bad region list", PBF_EINVAL;
  m.desc = d;
  m.p = d.degree;
  m.L = d.max_level;
  m.npc = (m.p + 1) * (m.p + 1) * (m.p + 1);
  for (int a = 0; a < 3; ++a) m.ext[a] = (int64_t)d.ntree[a] << m.L;
  m.exists.clear();
  if (d.tree_exists) m.exists.assign(d.tree_exists, d.tree_exists + (size_t)d.ntree[0] * d.ntree[1] * d.ntree[2]);
  m.regions.assign(d.regions, d.regions + d.n_regions);
  for (const pbf_region& r : m.regions)
    if (r.kind != PBF_REGION_BALL && r.kind != PBF_REGION_BOX) return *err = "bad region kind", PBF_EINVAL;
  m.desc.tree_exists = nullptr;
  m.desc.regions = nullptr;
  return PBF_OK;
}

// ---- refinement ----------------------------------------------------------------------

static int region_target(const HostMesh& m, const Octant& o) {
  int64_t s = m.size(o);
  double lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = m.coord(a, o.a[a]);
    hi[a] = m.coord(a, o.a[a] + s);
  }
  int best = 0;
  for (const pbf_region& r : m.regions) {
    const double* cmin = r.a;
    const double* cmax = r.kind == PBF_REGION_BALL ? r.a : r.b;
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      double g = 0.0;
      if (cmin[a] > hi[a]) g = cmin[a] - hi[a];
      else if (lo[a] > cmax[a]) g = lo[a] - cmax[a];
      d2 += g * g;
    }
    if (d2 < r.radius * r.radius && r.level > best) best = r.level;
  }
  return best < m.L ? best : m.L;
}

static void push_children(const HostMesh& m, const Octant& o, std::vector<Octant>& out) {
  int64_t h = m.size(o) >> 1;
  for (int c = 0; c < 8; ++c)
    out.push_back(Octant{{o.a[0] + (c & 1) * h, o.a[1] + ((c >> 1) & 1) * h, o.a[2] + ((c >> 2) & 1) * h}, o.level + 1});
}

static void refine_tree(const HostMesh& m, const Octant& o, std::vector<Octant>& out) {
  if (o.level < region_target(m, o)) {
    std::vector<Octant> kids;
    push_children(m, o, kids);
    for (const Octant& k : kids) refine_tree(m, k, out);
  } else {
    out.push_back(o);
  }
}

static void rekey(HostMesh& m) {
  m.key.resize(m.oct.size());
  for (size_t i = 0; i < m.oct.size(); ++i) m.key[i] = m.morton_key(m.oct[i].a);
}

static void balance(HostMesh& m) {
  const int64_t n_fine = m.ext[0] * m.ext[1] * m.ext[2];
  const bool use_grid = n_fine <= HostMesh::kFineGridMax;
  std::unique_ptr<uint8_t[]> level_of;  // the level of the leaf holding each finest cell
  if (use_grid) level_of.reset(new uint8_t[(size_t)n_fine]);
  for (;;) {
    const int64_t nl = (int64_t)m.oct.size();
    if (use_grid) {
#pragma omp parallel for schedule(dynamic, 256)
      for (int64_t i = 0; i < nl; ++i) {
        const Octant& o = m.oct[(size_t)i];
        const int64_t s = m.size(o);
        for (int64_t z = o.a[2]; z < o.a[2] + s; ++z)
          for (int64_t y = o.a[1]; y < o.a[1] + s; ++y)
            std::memset(level_of.get() + (size_t)(o.a[0] + m.ext[0] * (y + m.ext[1] * z)), o.level, (size_t)s);
      }
    }
    // mark the leaves that are more than one level coarser than a vertex neighbour (the
    // leaves are scanned in parallel; a mark is only ever set to 1). Only a leaf of level 2 or
    // finer can have such a neighbour; the level grid answers whether a neighbour is too
    // coarse, and only such a neighbour is looked up by its key.
    std::vector<uint8_t> split(m.oct.size(), 0);
    int any = 0;
#pragma omp parallel for schedule(static, 4096) reduction(| : any)
    for (int64_t i = 0; i < nl; ++i) {
      const Octant& o = m.oct[(size_t)i];
      if (o.level < 2) continue;
      int64_t s = m.size(o);
      for (int nb = 0; nb < 27; ++nb) {
        if (nb == 13) continue;
        int64_t q[3] = {o.a[0] + (nb % 3 - 1) * s, o.a[1] + ((nb / 3) % 3 - 1) * s, o.a[2] + (nb / 9 - 1) * s};
        if (use_grid && (!m.inside(q) || level_of[(size_t)(q[0] + m.ext[0] * (q[1] + m.ext[1] * q[2]))] >= o.level - 1))
          continue;
        int64_t j = m.locate(q);
        if (j >= 0 && m.oct[(size_t)j].level < o.level - 1) {
#pragma omp atomic write
          split[(size_t)j] = 1;
          any = 1;
        }
      }
    }
    if (!any) return;
    std::vector<Octant> next;
    next.reserve(m.oct.size() + 8);
    for (size_t i = 0; i < m.oct.size(); ++i) {
      if (split[i]) push_children(m, m.oct[i], next);
      else next.push_back(m.oct[i]);
    }
    m.oct.swap(next);
    rekey(m);
  }
}

// ---- nodes ----------------------------------------------------------------------------

static inline uint64_t pack_node(const int64_t n[3]) {
  return ((uint64_t)n[2] << 42) | ((uint64_t)n[1] << 21) | (uint64_t)n[0];
}

// 1D Lagrange weights of degree p at position u (node-lattice units) on a cell whose nodes
// sit at 0, s, .., p s.
static void weights_1d(int p, int64_t u, int64_t s, double w[3]) {
  double t = (double)u / (double)s;  // node-spacing units: nodes at t = 0..p
  if (p == 1) {
    w[0] = 1.0 - t;
    w[1] = t;
  } else {
    w[0] = 0.5 * (t - 1.0) * (t - 2.0);
    w[1] = t * (2.0 - t);
    w[2] = 0.5 * t * (t - 1.0);
  }
}

struct NodeTable {
  std::vector<uint64_t> keys;  // sorted unique
  std::vector<int64_t> xyz;    // [n][3]
  int64_t find(const int64_t n[3]) const {
    uint64_t k = pack_node(n);
    auto it = std::lower_bound(keys.begin(), keys.end(), k);
    return (it != keys.end() && *it == k) ? (int64_t)(it - keys.begin()) : -1;
  }
};

// Calls f(q) for the finest cells q around node n (node-lattice units): along each axis the
// cells on either side of the node's position half a node spacing away (one cell where the
// node lies inside a finest cell; none below 0). These are the cells whose closure may hold n.
template <typename F>
static void for_each_cell_around(int p, const int64_t n[3], F f) {
  int64_t c[3][2];
  int nc[3];
  for (int a = 0; a < 3; ++a) {
    nc[a] = 0;
    const int64_t lo = 2 * n[a] - 1, hi = 2 * n[a] + 1;  // half node-lattice units
    if (lo >= 0) c[a][nc[a]++] = lo / (2 * p);
    if (nc[a] == 0 || c[a][0] != hi / (2 * p)) c[a][nc[a]++] = hi / (2 * p);
  }
  for (int k = 0; k < nc[2]; ++k)
    for (int j = 0; j < nc[1]; ++j)
      for (int i = 0; i < nc[0]; ++i) {
        const int64_t q[3] = {c[0][i], c[1][j], c[2][k]};
        f(q);
      }
}

// The active cells whose closure holds node n; returns the smallest active index among those
// that do not have n as a nodal point (-1: none, i.e. the node is a proper dof).
static int32_t first_coarse_holder(const HostMesh& m, const int64_t n[3]) {
  int32_t best = -1;
  for_each_cell_around(m.p, n, [&](const int64_t q[3]) {
    int64_t leaf = m.locate(q);
    if (leaf < 0 || !m.active[(size_t)leaf]) return;
    const Octant& c = m.oct[(size_t)leaf];
    int64_t s = m.size(c);
    bool nodal = true;
    for (int a = 0; a < 3; ++a)
      if ((n[a] - m.p * c.a[a]) % s != 0) nodal = false;
    if (nodal) return;
    int32_t ai = m.active_of_leaf[(size_t)leaf];
    if (best < 0 || ai < best) best = ai;
  });
  return best;
}

// Sorts (node key, slot) pairs; with OpenMP the pieces are sorted in parallel and merged.
static void sort_pairs(std::vector<std::pair<uint64_t, int64_t>>& v) {
#ifdef _OPENMP
  __gnu_parallel::sort(v.begin(), v.end());
#else
  std::sort(v.begin(), v.end());
#endif
}

// out[i] = the number of j < i with pred(j), for i in [0, n): a prefix sum over fixed chunks,
// on all host cores (the result does not depend on the number of threads).
template <typename Pred>
static void exclusive_count(int64_t n, Pred pred, int32_t* out) {
  const int64_t chunk = 1 << 16;
  const int64_t nch = (n + chunk - 1) / chunk;
  std::vector<int32_t> base((size_t)nch + 1, 0);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nch; ++c) {
    int32_t k = 0;
    for (int64_t i = c * chunk; i < std::min(n, (c + 1) * chunk); ++i) k += pred(i) ? 1 : 0;
    base[(size_t)c + 1] = k;
  }
  for (int64_t c = 0; c < nch; ++c) base[(size_t)c + 1] += base[(size_t)c];
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nch; ++c) {
    int32_t k = base[(size_t)c];
    for (int64_t i = c * chunk; i < std::min(n, (c + 1) * chunk); ++i) {
      out[(size_t)i] = k;
      k += pred(i) ? 1 : 0;
    }
  }
}

pbf_status build_mesh(HostMesh& m, const std::vector<uint8_t>* mat_hint, std::string* err) {
  const int p = m.p;
  // forest
  m.oct.clear();
  for (int tz = 0; tz < m.desc.ntree[2]; ++tz)
    for (int ty = 0; ty < m.desc.ntree[1]; ++ty)
      for (int tx = 0; tx < m.desc.ntree[0]; ++tx) {
        Octant root{{(int64_t)tx << m.L, (int64_t)ty << m.L, (int64_t)tz << m.L}, 0};
        if (m.inside(root.a)) refine_tree(m, root, m.oct);
      }
  if (m.oct.empty()) return *err = "no trees exist", PBF_EINVAL;
  m.fine_leaf.reset();
  rekey(m);
  balance(m);
  size_t nl = m.oct.size();
  // the finest-cell index of the balanced leaves, for constant-time locate from here on
  if (m.ext[0] * m.ext[1] * m.ext[2] <= HostMesh::kFineGridMax) {
    std::shared_ptr<int32_t[]> fl(new int32_t[(size_t)(m.ext[0] * m.ext[1] * m.ext[2])]);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < (int64_t)nl; ++i) {
      const Octant& o = m.oct[(size_t)i];
      const int64_t s = m.size(o);
      for (int64_t z = o.a[2]; z < o.a[2] + s; ++z)
        for (int64_t y = o.a[1]; y < o.a[1] + s; ++y) {
          int32_t* row = fl.get() + (size_t)(m.ext[0] * (y + m.ext[1] * z));
          for (int64_t x = o.a[0]; x < o.a[0] + s; ++x) row[x] = (int32_t)i;
        }
    }
    m.fine_leaf = std::move(fl);
  }
  // activity and material
  m.active.assign(nl, 0);
  m.material.assign(nl, 0);
  m.active_of_leaf.assign(nl, -1);
  m.leaf_of_active.clear();
  for (size_t i = 0; i < nl; ++i) {
    const Octant& o = m.oct[i];
    double z0 = m.coord(2, o.a[2]), z1 = m.coord(2, o.a[2] + m.size(o));
    m.active[i] = z0 < m.desc.active_top_z;
    double zc = 0.5 * (z0 + z1);
    m.material[i] = (zc >= m.desc.powder_z0 && zc < m.desc.powder_z1) ? 1 : 0;
    if (mat_hint) m.material[i] = (*mat_hint)[i];
    if (m.active[i]) {
      m.active_of_leaf[i] = (int32_t)m.leaf_of_active.size();
      m.leaf_of_active.push_back((int32_t)i);
    }
  }
  size_t na = m.leaf_of_active.size();
  const int npc = m.npc;
  // node table: the (node, slot) entries sorted by node, then slot. When the node's index on
  // the node lattice (z, y, x lexicographic: the order of pack_node) and the slot fit in one
  // 64-bit word together, an entry is that word (half the bytes to sort); otherwise a
  // (pack_node key, slot) pair. Either way the order is total, so the result is the same in
  // parallel.
  const int64_t nsl = (int64_t)(na * (size_t)npc);
  const int64_t NX = p * m.ext[0] + 1, NY = p * m.ext[1] + 1, NZ = p * m.ext[2] + 1;
  auto bit_length = [](uint64_t v) {
    int b = 0;
    while (b < 64 && (v >> b) != 0) ++b;
    return b;
  };
  const int sbits = bit_length((uint64_t)std::max<int64_t>(nsl - 1, 0));
  const bool packed = bit_length((uint64_t)NX) + bit_length((uint64_t)NY) + bit_length((uint64_t)NZ) <= 62 &&
                      bit_length((uint64_t)(NX * NY * NZ - 1)) + sbits <= 64;
  const uint64_t smask = sbits == 0 ? 0 : (~0ull >> (64 - sbits));
  std::vector<uint64_t> word;
  std::vector<std::pair<uint64_t, int64_t>> ents;
  if (packed) word.resize((size_t)nsl);
  else ents.resize((size_t)nsl);
#pragma omp parallel for schedule(static, 1024)
  for (int64_t c = 0; c < (int64_t)na; ++c) {
    const Octant& o = m.oct[(size_t)m.leaf_of_active[(size_t)c]];
    int64_t s = m.size(o);
    for (int l = 0; l < npc; ++l) {
      int ijk[3] = {l % (p + 1), (l / (p + 1)) % (p + 1), l / ((p + 1) * (p + 1))};
      int64_t n[3];
      for (int a = 0; a < 3; ++a) n[a] = p * o.a[a] + ijk[a] * s;
      const size_t slot = (size_t)c * (size_t)npc + (size_t)l;
      if (packed) word[slot] = ((uint64_t)(n[0] + NX * (n[1] + NY * n[2])) << sbits) | (uint64_t)slot;
      else ents[slot] = {pack_node(n), (int64_t)slot};
    }
  }
  if (packed) {
#ifdef _OPENMP
    __gnu_parallel::sort(word.begin(), word.end());
#else
    std::sort(word.begin(), word.end());
#endif
  } else {
    sort_pairs(ents);
  }
  // entry e: a key equal for the entries of one node, its slot, and the node's position
  auto node_of = [&](int64_t e) { return packed ? word[(size_t)e] >> sbits : ents[(size_t)e].first; };
  auto slot_of = [&](int64_t e) { return packed ? (int64_t)(word[(size_t)e] & smask) : ents[(size_t)e].second; };
  auto position = [&](int64_t e, int64_t* xyz) {
    if (packed) {
      const int64_t i = (int64_t)(word[(size_t)e] >> sbits);
      xyz[0] = i % NX;
      xyz[1] = (i / NX) % NY;
      xyz[2] = i / (NX * NY);
    } else {
      const uint64_t k = ents[(size_t)e].first;
      xyz[0] = (int64_t)(k & 0x1FFFFF);
      xyz[1] = (int64_t)((k >> 21) & 0x1FFFFF);
      xyz[2] = (int64_t)(k >> 42);
    }
  };
  // unique nodes: entry e starts a node when its key differs from the previous one, and the
  // node's index is the number of starts up to e (a prefix sum); the entries of a node are
  // sorted by slot, so its first entry holds its first slot
  const int64_t ne = nsl;
  auto starts = [&](int64_t e) { return e == 0 || node_of(e) != node_of(e - 1); };
  std::vector<int32_t> starts_before((size_t)ne);
  exclusive_count(ne, starts, starts_before.data());
  const size_t nn = ne == 0 ? 0 : (size_t)starts_before.back() + (starts(ne - 1) ? 1 : 0);
  NodeTable nodes;
  nodes.keys.resize(nn);
  nodes.xyz.resize(3 * nn);
  std::vector<int32_t> first_slot(nn);
  std::vector<int32_t> node_of_slot(na * (size_t)npc);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < ne; ++e) {
    const bool st = starts(e);
    const size_t nd = (size_t)(starts_before[(size_t)e] + (st ? 1 : 0) - 1);
    const int64_t sl = slot_of(e);
    if (st) {
      int64_t* xyz = &nodes.xyz[3 * nd];
      position(e, xyz);
      nodes.keys[nd] = pack_node(xyz);
      first_slot[nd] = (int32_t)sl;
    }
    node_of_slot[(size_t)sl] = (int32_t)nd;
  }
  std::vector<int32_t> holder(nn);
#pragma omp parallel for schedule(static, 4096)
  for (int64_t i = 0; i < (int64_t)nn; ++i) holder[(size_t)i] = first_coarse_holder(m, &nodes.xyz[(size_t)i * 3]);
  // first-touch numbering of dofs and of constraint rows: a node is numbered at its first slot,
  // so its number is the count of first slots of its kind (free or hanging) before that one.
  // Kind of each slot: 0 not its node's first, 1 the first of a free node, 2 of a hanging one.
  const int64_t ns = (int64_t)node_of_slot.size();
  std::vector<uint8_t> kind((size_t)ns);
#pragma omp parallel for schedule(static)
  for (int64_t sl = 0; sl < ns; ++sl) {
    const int32_t nd = node_of_slot[(size_t)sl];
    kind[(size_t)sl] = first_slot[(size_t)nd] != (int32_t)sl ? 0 : (holder[(size_t)nd] < 0 ? 1 : 2);
  }
  std::vector<int32_t> dof_before((size_t)ns), row_before((size_t)ns);
  exclusive_count(ns, [&](int64_t sl) { return kind[(size_t)sl] == 1; }, dof_before.data());
  exclusive_count(ns, [&](int64_t sl) { return kind[(size_t)sl] == 2; }, row_before.data());
  std::vector<int32_t> dof(nn, -1), row(nn, -1);
  int64_t n_dofs = 0, n_rows64 = 0;
  if (ns > 0) {
    n_dofs = dof_before[(size_t)ns - 1] + (kind[(size_t)ns - 1] == 1 ? 1 : 0);
    n_rows64 = row_before[(size_t)ns - 1] + (kind[(size_t)ns - 1] == 2 ? 1 : 0);
  }
  m.n_dofs = n_dofs;
  const int32_t n_rows = (int32_t)n_rows64;
  std::vector<int32_t> row_node((size_t)n_rows);
  m.dof_xyz.assign((size_t)n_dofs * 3, 0);
#pragma omp parallel for schedule(static)
  for (int64_t sl = 0; sl < ns; ++sl) {
    if (kind[(size_t)sl] == 0) continue;
    const int32_t nd = node_of_slot[(size_t)sl];
    if (kind[(size_t)sl] == 2) {
      row[(size_t)nd] = row_before[(size_t)sl];
      row_node[(size_t)row_before[(size_t)sl]] = nd;
    } else {
      const int32_t d = dof_before[(size_t)sl];
      dof[(size_t)nd] = d;
      for (int a = 0; a < 3; ++a) m.dof_xyz[(size_t)d * 3 + (size_t)a] = nodes.xyz[(size_t)nd * 3 + (size_t)a];
    }
  }
  if (m.n_dofs >= ((int64_t)1 << 31)) return *err = "too many dofs", PBF_EINVAL;
  // constraint rows, with chains substituted: rows whose masters are all free are expanded on
  // all host cores, the others (chains through hanging masters) afterwards in row order,
  // reusing the expanded rows; each row's arithmetic is the same either way
  using Row = std::vector<std::pair<int32_t, double>>;
  std::vector<Row> memo((size_t)n_rows);
  std::vector<uint8_t> done((size_t)n_rows, 0);
  // the expansion of hanging node nd into `out`; sub(r) gives row r's expansion or null when it
  // is not available (then nothing is written and false is returned)
  auto expand_row = [&](int32_t nd, const auto& sub, Row& out) -> bool {
    const Octant& c = m.oct[(size_t)m.leaf_of_active[(size_t)holder[(size_t)nd]]];
    int64_t s = m.size(c);
    double w1[3][3];
    for (int a = 0; a < 3; ++a) weights_1d(p, nodes.xyz[(size_t)nd * 3 + a] - p * c.a[a], s, w1[a]);
    Row acc;
    for (int l = 0; l < npc; ++l) {
      int ijk[3] = {l % (p + 1), (l / (p + 1)) % (p + 1), l / ((p + 1) * (p + 1))};
      double w = w1[0][ijk[0]] * w1[1][ijk[1]] * w1[2][ijk[2]];
      if (w == 0.0) continue;
      int64_t q[3];
      for (int a = 0; a < 3; ++a) q[a] = p * c.a[a] + ijk[a] * s;
      int32_t mn = (int32_t)nodes.find(q);
      if (holder[(size_t)mn] >= 0) {
        const Row* r = sub(row[(size_t)mn]);
        if (!r) return false;
        for (const auto& e : *r) acc.push_back({e.first, w * e.second});
      } else {
        acc.push_back({dof[(size_t)mn], w});
      }
    }
    std::stable_sort(acc.begin(), acc.end(),
                     [](const std::pair<int32_t, double>& x, const std::pair<int32_t, double>& y) { return x.first < y.first; });
    out.clear();
    for (size_t e = 0; e < acc.size();) {
      size_t f = e;
      double sum = 0.0;
      while (f < acc.size() && acc[f].first == acc[e].first) sum += acc[f++].second;
      if (sum != 0.0) out.push_back({acc[e].first, sum});
      e = f;
    }
    return true;
  };
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t r = 0; r < (int64_t)n_rows; ++r) {
    auto none = [](int32_t) -> const Row* { return nullptr; };
    if (expand_row(row_node[(size_t)r], none, memo[(size_t)r])) done[(size_t)r] = 1;
  }
  std::function<const Row*(int32_t)> chain = [&](int32_t r) -> const Row* {
    if (!done[(size_t)r]) {
      expand_row(row_node[(size_t)r], chain, memo[(size_t)r]);
      done[(size_t)r] = 1;
    }
    return &memo[(size_t)r];
  };
  for (int32_t r = 0; r < n_rows; ++r) chain(r);
  m.con_ptr.assign(1, 0);
  m.con_idx.clear();
  m.con_w.clear();
  m.hang_xyz.clear();
  for (int32_t r = 0; r < n_rows; ++r) {
    int32_t nd = row_node[(size_t)r];
    for (const auto& e : memo[(size_t)r]) {
      m.con_idx.push_back(e.first);
      m.con_w.push_back(e.second);
    }
    m.con_ptr.push_back((int32_t)m.con_idx.size());
    for (int a = 0; a < 3; ++a) m.hang_xyz.push_back(nodes.xyz[(size_t)nd * 3 + a]);
  }
  // cell table
  m.cell_dofs.resize(na * (size_t)npc);
#pragma omp parallel for schedule(static)
  for (int64_t slot = 0; slot < ns; ++slot) {
    const int32_t nd = node_of_slot[(size_t)slot];
    m.cell_dofs[(size_t)slot] = holder[(size_t)nd] >= 0 ? -1 - row[(size_t)nd] : dof[(size_t)nd];
  }
  // Dirichlet dofs
  m.dirichlet.assign((size_t)m.n_dofs, 0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m.n_dofs; ++i)
    for (int a = 0; a < 3; ++a) {
      int64_t v = m.dof_xyz[(size_t)i * 3 + a];
      if ((m.desc.dirichlet_faces & (1u << (2 * a))) && v == 0) m.dirichlet[(size_t)i] = 1;
      if ((m.desc.dirichlet_faces & (1u << (2 * a + 1))) && v == p * m.ext[a]) m.dirichlet[(size_t)i] = 1;
    }
  // greedy colouring with per-dof colour masks of W 64-bit words: one word while 64 colours
  // suffice (the meshes here need at most about 32), else again with four (up to 256 colours);
  // the colours are the same either way
  auto colour_cells = [&](const int W) -> bool {
    std::vector<uint64_t> used((size_t)m.n_dofs * (size_t)W, 0);
    m.colour.assign(na, 0);
    m.n_colours = 0;
    std::vector<int32_t> touched;
    for (size_t c = 0; c < na; ++c) {
      touched.clear();
      for (int l = 0; l < npc; ++l) {
        int32_t v = m.cell_dofs[c * (size_t)npc + (size_t)l];
        if (v >= 0) touched.push_back(v);
        else
          for (int32_t e = m.con_ptr[(size_t)(-1 - v)]; e < m.con_ptr[(size_t)(-v)]; ++e) touched.push_back(m.con_idx[(size_t)e]);
      }
      uint64_t busy[4] = {0, 0, 0, 0};
      for (int32_t t : touched)
        for (int w = 0; w < W; ++w) busy[w] |= used[(size_t)t * (size_t)W + (size_t)w];
      int col = -1;
      for (int w = 0; w < W && col < 0; ++w)
        if (~busy[w]) col = 64 * w + __builtin_ctzll(~busy[w]);
      if (col < 0) return false;
      m.colour[c] = col;
      if (col + 1 > m.n_colours) m.n_colours = col + 1;
      for (int32_t t : touched) used[(size_t)t * (size_t)W + (size_t)(col / 64)] |= 1ull << (col % 64);
    }
    return true;
  };
  if (!colour_cells(1) && !colour_cells(4)) return *err = "colouring needs more than 256 colours", PBF_EINVAL;
  // top faces
  m.top.assign(na, 0);
  m.n_top = 0;
  for (size_t c = 0; c < na; ++c) {
    const Octant& o = m.oct[(size_t)m.leaf_of_active[c]];
    int64_t up[3] = {o.a[0], o.a[1], o.a[2] + m.size(o)};
    bool open = !m.inside(up) || !(m.coord(2, up[2]) < m.desc.active_top_z);
    m.top[c] = open;
    m.n_top += open;
  }
  ++m.generation;
  return PBF_OK;
}

// ---- transfer ----------------------------------------------------------------------------

void make_transfer(const HostMesh& om, const HostMesh& nm, double fill, TransferMap& out) {
  const int p = om.p, npc = om.npc;
  out.pending = true;
  out.n_old = om.n_dofs;
  out.n_new = nm.n_dofs;
  out.fill = fill;
  // the rows are built in parallel over fixed chunks of new dofs, each chunk into its own
  // buffers (taken by the threads as they come free: the rows that interpolate cluster in the
  // refined region), and concatenated in dof order (the same result for any number of threads)
  const int64_t n_new = nm.n_dofs;
  constexpr int64_t kChunk = 4096;
  const int64_t n_chunks = (n_new + kChunk - 1) / kChunk;
  std::vector<std::vector<int32_t>> t_idx((size_t)n_chunks);
  std::vector<std::vector<double>> t_w((size_t)n_chunks);
  std::vector<int32_t> row_len((size_t)n_new, 0);
#pragma omp parallel
  {
    std::vector<std::pair<int32_t, double>> acc;
#pragma omp for schedule(dynamic, 1)
    for (int64_t ch = 0; ch < n_chunks; ++ch) {
      const int64_t lo = ch * kChunk, hi = std::min(n_new, lo + kChunk);
      std::vector<int32_t>& my_idx = t_idx[(size_t)ch];
      std::vector<double>& my_w = t_w[(size_t)ch];
      for (int64_t i = lo; i < hi; ++i) {
        const int64_t* n = &nm.dof_xyz[(size_t)i * 3];
        // first old active cell (cell order) whose closure holds the point
        int32_t best = -1;
        for_each_cell_around(p, n, [&](const int64_t q[3]) {
          int64_t leaf = om.locate(q);
          if (leaf < 0 || !om.active[(size_t)leaf]) return;
          int32_t ai = om.active_of_leaf[(size_t)leaf];
          if (best < 0 || ai < best) best = ai;
        });
        if (best < 0) continue;
        const Octant& c = om.oct[(size_t)om.leaf_of_active[(size_t)best]];
        int64_t s = om.size(c);
        // a nodal point of that cell: its one weight is exactly 1, so its row is the node's own
        // (a dof, or its constraint row, whose masters are sorted and merged already)
        int loc = 0, stride = 1;
        bool nodal = true;
        for (int a = 0; a < 3 && nodal; ++a) {
          const int64_t u = n[a] - p * c.a[a];
          nodal = u % s == 0;
          loc += (int)(u / s) * stride;
          stride *= p + 1;
        }
        if (nodal) {
          const int32_t v = om.cell_dofs[(size_t)best * (size_t)npc + (size_t)loc];
          if (v >= 0) {
            my_idx.push_back(v);
            my_w.push_back(1.0);
            row_len[(size_t)i] = 1;
          } else {
            const int32_t e0 = om.con_ptr[(size_t)(-1 - v)], e1 = om.con_ptr[(size_t)(-v)];
            my_idx.insert(my_idx.end(), om.con_idx.begin() + e0, om.con_idx.begin() + e1);
            my_w.insert(my_w.end(), om.con_w.begin() + e0, om.con_w.begin() + e1);
            row_len[(size_t)i] = e1 - e0;
          }
          continue;
        }
        double w1[3][3];
        for (int a = 0; a < 3; ++a) weights_1d(p, n[a] - p * c.a[a], s, w1[a]);
        acc.clear();
        for (int l = 0; l < npc; ++l) {
          int ijk[3] = {l % (p + 1), (l / (p + 1)) % (p + 1), l / ((p + 1) * (p + 1))};
          double w = w1[0][ijk[0]] * w1[1][ijk[1]] * w1[2][ijk[2]];
          if (w == 0.0) continue;
          int32_t v = om.cell_dofs[(size_t)best * (size_t)npc + (size_t)l];
          if (v >= 0) acc.push_back({v, w});
          else
            for (int32_t e = om.con_ptr[(size_t)(-1 - v)]; e < om.con_ptr[(size_t)(-v)]; ++e)
              acc.push_back({om.con_idx[(size_t)e], w * om.con_w[(size_t)e]});
        }
        // by old dof, entries of one dof in the order above (a stable insertion sort: the lists
        // are short)
        for (size_t e = 1; e < acc.size(); ++e) {
          const std::pair<int32_t, double> x = acc[e];
          size_t f = e;
          for (; f > 0 && acc[f - 1].first > x.first; --f) acc[f] = acc[f - 1];
          acc[f] = x;
        }
        int32_t len = 0;
        for (size_t e = 0; e < acc.size();) {
          size_t f = e;
          double sum = 0.0;
          while (f < acc.size() && acc[f].first == acc[e].first) sum += acc[f++].second;
          if (sum != 0.0) {
            my_idx.push_back(acc[e].first);
            my_w.push_back(sum);
            ++len;
          }
          e = f;
        }
        row_len[(size_t)i] = len;
      }
    }
  }
  out.ptr.assign((size_t)n_new + 1, 0);
  for (int64_t i = 0; i < n_new; ++i) out.ptr[(size_t)i + 1] = out.ptr[(size_t)i] + row_len[(size_t)i];
  out.idx.clear();
  out.w.clear();
  out.idx.reserve((size_t)out.ptr.back());
  out.w.reserve((size_t)out.ptr.back());
  for (int64_t ch = 0; ch < n_chunks; ++ch) {
    out.idx.insert(out.idx.end(), t_idx[(size_t)ch].begin(), t_idx[(size_t)ch].end());
    out.w.insert(out.w.end(), t_w[(size_t)ch].begin(), t_w[(size_t)ch].end());
  }
}

// Gauss-Legendre points on [0, 1] for p + 1 = 2 or 3 points.
static double gauss_point(int p, int q) {
  if (p == 1) return q == 0 ? 0.5 - 0.5 / std::sqrt(3.0) : 0.5 + 0.5 / std::sqrt(3.0);
  const double h = 0.5 * std::sqrt(0.6);
  return q == 0 ? 0.5 - h : (q == 1 ? 0.5 : 0.5 + h);
}

void make_history_map(const HostMesh& om, const HostMesh& nm, std::vector<int32_t>& out) {
  const int nq = nm.p + 1, nq3 = nq * nq * nq;
  const size_t ncell = nm.leaf_of_active.size();
  out.assign(ncell * (size_t)nq3, -1);
  double g[3];
  for (int q = 0; q < nq; ++q) g[q] = gauss_point(nm.p, q);
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t ci = 0; ci < (int64_t)ncell; ++ci) {
    const size_t c = (size_t)ci;
    const size_t leaf = (size_t)nm.leaf_of_active[c];
    const Octant& o = nm.oct[leaf];
    const double S = (double)nm.size(o);
    const int32_t init = nm.material[leaf] == 1 ? -1 : -2;
    for (int q = 0; q < nq3; ++q) {
      const int qi[3] = {q % nq, (q / nq) % nq, q / (nq * nq)};
      double P[3];
      int64_t f[3][2];
      int nf[3];
      for (int a = 0; a < 3; ++a) {
        P[a] = (double)o.a[a] + S * g[qi[a]];
        f[a][0] = (int64_t)std::floor(P[a]);
        nf[a] = 1;
        if ((double)f[a][0] == P[a]) f[a][nf[a]++] = f[a][0] - 1;  // on a cell boundary
      }
      int64_t best = -1, best_leaf = -1;
      for (int i = 0; i < nf[0]; ++i)
        for (int j = 0; j < nf[1]; ++j)
          for (int k = 0; k < nf[2]; ++k) {
            const int64_t fine[3] = {f[0][i], f[1][j], f[2][k]};
            const int64_t l = om.locate(fine);
            if (l < 0) continue;
            const int32_t ac = om.active_of_leaf[(size_t)l];
            if (ac >= 0 && (best < 0 || ac < best)) {
              best = ac;
              best_leaf = l;
            }
          }
      int32_t v = init;
      if (best >= 0) {
        const Octant& ol = om.oct[(size_t)best_leaf];
        const double So = (double)om.size(ol);
        int qo[3];
        for (int a = 0; a < 3; ++a) {
          const double xi = (P[a] - (double)ol.a[a]) / So;
          int arg = 0;
          for (int t = 1; t < nq; ++t)
            if (std::fabs(xi - g[t]) < std::fabs(xi - g[arg])) arg = t;
          qo[a] = arg;
        }
        v = (int32_t)(best * nq3 + qo[0] + nq * (qo[1] + nq * qo[2]));
      }
      out[c * (size_t)nq3 + (size_t)q] = v;
    }
  }
}

void gate_pins(const HostMesh& m, const double* rc_min, double r_coarsen, std::vector<pbf_region>& out) {
  std::vector<std::array<int64_t, 4>> fam;  // level, parent anchor
  for (size_t c = 0; c < m.leaf_of_active.size(); ++c) {
    const Octant& o = m.oct[(size_t)m.leaf_of_active[c]];
    if (o.level == 0 || !(rc_min[c] < r_coarsen)) continue;
    const int64_t ps = 2 * m.size(o);
    fam.push_back({(int64_t)o.level, o.a[0] / ps * ps, o.a[1] / ps * ps, o.a[2] / ps * ps});
  }
  std::sort(fam.begin(), fam.end());
  fam.erase(std::unique(fam.begin(), fam.end()), fam.end());
  for (const auto& f : fam) {
    const int lv = (int)f[0];
    const int64_t ps = (int64_t)1 << (m.L - lv + 1);
    pbf_region r{};
    r.kind = PBF_REGION_BOX;
    r.level = lv;
    double eps_min = 1e300;
    for (int a = 0; a < 3; ++a) {
      const double eps = 0.25 * m.desc.tree_h[a] / (double)((int64_t)1 << m.L);
      r.a[a] = m.coord(a, f[1 + a]) + eps;
      r.b[a] = m.coord(a, f[1 + a] + ps) - eps;
      eps_min = std::min(eps_min, eps);
    }
    r.radius = 0.5 * eps_min;
    out.push_back(r);
  }
}

}  // namespace pbf
