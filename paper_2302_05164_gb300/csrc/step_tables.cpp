// Host-side patch tables of the fused explicit step (step_layout.hpp). The per-patch work
// (slot keys, cell-local positions, slot lists, hanging tables) runs on all host cores; the
// partition into patches, the ownership of dofs and the concatenation follow the patch
// numbering, so the tables do not depend on the number of threads.
#include "step_layout.hpp"

#include <algorithm>
#include <climits>
#include <utility>

#ifdef _OPENMP
#include <parallel/algorithm>
#endif

namespace pbf {
namespace {

// Hanging-table entries a patch may hold. Without a bound the patches at refinement
// interfaces carry about ten times the average (C2: up to 1,137 entries against 106); the
// largest patch sets every block's shared memory, and the heavy blocks set the step's critical
// path. Measured on C2 (us per step, fused step with programmatic dependent launch): no bound
// 25.9, 768: 25.8, 704: 25.7, 640: 22.85, 576: 23.0, 512: 23.8, 384: 24.5, 256: 26.3, 192: 27.0.
// Below about 640 the extra patches and re-staged slots cost more than the balance gains;
// from about 700 on the step is as slow as without a bound.
constexpr int64_t kStepMaxHent = 640;

uint64_t spread_bits3(uint64_t v) {
  uint64_t r = 0;
  for (int b = 0; b < 21; ++b) r |= ((v >> b) & 1u) << (3 * b);
  return r;
}

// Keys of a patch (dofs, and n_dofs + r for hanging row r) with a position each, by open
// addressing (a patch lists at most a few thousand keys; one table per thread, reset for each
// use). find() returns -1 for a key that is not present.
class KeyIndex {
 public:
  void reset(size_t n) {
    int bits = 6;
    while (((size_t)1 << bits) < 2 * n) ++bits;
    shift_ = 32 - bits;
    mask_ = (1u << bits) - 1;
    key_.assign((size_t)1 << bits, -1);
    pos_.resize((size_t)1 << bits);
  }
  // adds k with position j; false (and nothing changes) when k is present already
  bool insert(int32_t k, int32_t j) {
    uint32_t h = slot(k);
    while (key_[h] >= 0) {
      if (key_[h] == k) return false;
      h = (h + 1) & mask_;
    }
    key_[h] = k;
    pos_[h] = j;
    return true;
  }
  void build(const int32_t* kb, int32_t nu) {
    reset((size_t)nu);
    for (int32_t j = 0; j < nu; ++j) insert(kb[j], j);
  }
  int32_t find(int32_t k) const {
    uint32_t h = slot(k);
    for (uint32_t n = 0; n <= mask_; ++n, h = (h + 1) & mask_) {
      if (key_[h] == k) return pos_[h];
      if (key_[h] < 0) return -1;
    }
    return -1;
  }

 private:
  uint32_t slot(int32_t k) const { return ((uint32_t)k * 2654435761u) >> shift_; }
  std::vector<int32_t> key_, pos_;
  uint32_t mask_ = 0;
  int shift_ = 26;
};

// The slot keys of one patch, sorted and unique: dof d, or n_dofs + r for hanging row r, with
// the masters of its hanging rows; hent = the hanging-table entries of its rows. raw and seen
// are the calling thread's work space.
void patch_keys(const HostMesh& m, const std::vector<std::pair<uint64_t, int32_t>>& order, size_t c0, size_t c1,
                std::vector<int32_t>& keys, int64_t& hent, std::vector<int32_t>& raw, KeyIndex& seen) {
  const size_t npc = (size_t)m.npc;
  const int32_t nd32 = (int32_t)m.n_dofs;
  raw.clear();
  for (size_t c = c0; c < c1; ++c)
    for (size_t a = 0; a < npc; ++a) {
      const int32_t d = m.cell_dofs[(size_t)order[c].second * npc + a];
      if (d >= 0) {
        raw.push_back(d);
      } else {
        const int32_t r = -1 - d;
        raw.push_back(nd32 + r);
        for (int32_t e = m.con_ptr[(size_t)r]; e < m.con_ptr[(size_t)r + 1]; ++e) raw.push_back(m.con_idx[(size_t)e]);
      }
    }
  // the distinct keys (each key of a patch recurs in up to eight of its cells), then sorted
  seen.reset(raw.size());
  keys.clear();
  for (int32_t k : raw)
    if (seen.insert(k, 0)) keys.push_back(k);
  std::sort(keys.begin(), keys.end());
  hent = 0;
  for (int32_t k : keys)
    if (k >= nd32) hent += m.con_ptr[(size_t)(k - nd32) + 1] - m.con_ptr[(size_t)(k - nd32)];
}

}  // namespace

void build_step_tables(const HostMesh& m, StepHost& out) {
  out = StepHost();
  const size_t nc = m.leaf_of_active.size(), npc = (size_t)m.npc;
  const int32_t nd32 = (int32_t)m.n_dofs;
  if (nc == 0) return;
  // cells in the global Morton order of their anchors (keys of distinct cells differ)
  std::vector<std::pair<uint64_t, int32_t>> order(nc);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < (int64_t)nc; ++c) {
    const Octant& o = m.oct[(size_t)m.leaf_of_active[(size_t)c]];
    const uint64_t k = spread_bits3((uint64_t)o.a[0]) | (spread_bits3((uint64_t)o.a[1]) << 1) |
                       (spread_bits3((uint64_t)o.a[2]) << 2);
    order[(size_t)c] = {k, (int32_t)c};
  }
#ifdef _OPENMP
  __gnu_parallel::sort(order.begin(), order.end());
#else
  std::sort(order.begin(), order.end());
#endif
  // patches: runs of consecutive cells in that order, at most kStepCells cells and at most
  // kStepMaxHent hanging-table entries each (a cell with more starts a patch of its own)
  std::vector<size_t> pb{0};
  {
    const size_t n_rows = m.con_ptr.empty() ? 0 : m.con_ptr.size() - 1;
    std::vector<uint8_t> in_patch(n_rows, 0);
    std::vector<int32_t> rows, cell_rows;
    int64_t hent = 0;
    for (size_t c = 0; c < nc; ++c) {
      cell_rows.clear();
      for (size_t a = 0; a < npc; ++a) {
        const int32_t d = m.cell_dofs[(size_t)order[c].second * npc + a];
        if (d < 0 && std::find(cell_rows.begin(), cell_rows.end(), -1 - d) == cell_rows.end()) cell_rows.push_back(-1 - d);
      }
      auto added = [&]() {
        int64_t h = 0;
        for (int32_t r : cell_rows)
          if (!in_patch[(size_t)r]) h += m.con_ptr[(size_t)r + 1] - m.con_ptr[(size_t)r];
        return h;
      };
      int64_t add = added();
      const size_t len = c - pb.back();
      if (len > 0 && (len == (size_t)kStepCells || hent + add > kStepMaxHent)) {
        for (int32_t r : rows) in_patch[(size_t)r] = 0;
        rows.clear();
        hent = 0;
        pb.push_back(c);
        add = added();
      }
      for (int32_t r : cell_rows)
        if (!in_patch[(size_t)r]) {
          in_patch[(size_t)r] = 1;
          rows.push_back(r);
        }
      hent += add;
    }
    pb.push_back(nc);
  }
  const size_t np = pb.size() - 1;
  // slot keys and work of every patch
  std::vector<std::vector<int32_t>> keys(np);
  std::vector<int64_t> work(np, 0);
#pragma omp parallel
  {
    std::vector<int32_t> raw;
    KeyIndex seen;
#pragma omp for schedule(dynamic, 8)
    for (int64_t p = 0; p < (int64_t)np; ++p) {
      int64_t hent = 0;
      patch_keys(m, order, pb[(size_t)p], pb[(size_t)p + 1], keys[(size_t)p], hent, raw, seen);
      work[(size_t)p] = (int64_t)keys[(size_t)p].size() + 2 * hent;
    }
  }
  std::vector<int32_t> porder(np);
  for (size_t p = 0; p < np; ++p) porder[p] = (int32_t)p;
  std::stable_sort(porder.begin(), porder.end(), [&](int32_t a, int32_t b) { return work[(size_t)a] > work[(size_t)b]; });
  // ownership: each dof belongs to the first patch in that numbering that lists it
  std::vector<int32_t> owner((size_t)m.n_dofs, INT_MAX);
  for (size_t q = 0; q < np; ++q)
    for (int32_t k : keys[(size_t)porder[q]]) {
      if (k >= nd32) break;  // sorted: the hanging rows follow the dofs
      if (owner[(size_t)k] == INT_MAX) owner[(size_t)k] = (int32_t)q;
    }
  // per patch (in its numbering q): cells, cell-local positions, slot list, hanging table
  StepHost& o = out;
  o.loc.assign(np * npc * kStepCells, 0);
  o.cell.assign(np * kStepCells, -1);
  std::vector<std::vector<int32_t>> pslot(np);
  std::vector<std::vector<uint16_t>> phloc(np);
  std::vector<std::vector<float>> phw(np);
  std::vector<int32_t> pnfree(np);
  int bad = 0;
#pragma omp parallel reduction(| : bad)
  {
    KeyIndex index;
#pragma omp for schedule(dynamic, 8)
    for (int64_t qq = 0; qq < (int64_t)np; ++qq) {
      const size_t q = (size_t)qq, p = (size_t)porder[q];
      const int32_t* kb = keys[p].data();
      const int32_t nu = (int32_t)keys[p].size();
      pnfree[q] = (int32_t)(std::lower_bound(kb, kb + nu, nd32) - kb);
      index.build(kb, nu);
      auto pos = [&](int32_t key) {
        const int32_t j = index.find(key);
        if (j < 0) bad = 1;  // every key looked up is listed: a miss means no fused form
        return step_swizzle(j < 0 ? 0 : (int)j);
      };
      for (size_t c = pb[p]; c < pb[p + 1]; ++c) {
        const size_t lane = c - pb[p], cell = (size_t)order[c].second;
        o.cell[q * kStepCells + lane] = (int32_t)cell;
        for (size_t a = 0; a < npc; ++a) {
          const int32_t d = m.cell_dofs[cell * npc + a];
          o.loc[(q * npc + a) * kStepCells + lane] = (uint16_t)pos(d >= 0 ? d : nd32 + (-1 - d));
        }
      }
      std::vector<int32_t>& sl = pslot[q];
      sl.reserve((size_t)nu + 3);
      for (int32_t j = 0; j < nu; ++j) {
        const int32_t k = kb[j];
        if (k < nd32) {
          sl.push_back(owner[(size_t)k] == (int32_t)q ? (int32_t)((uint32_t)k | 0x80000000u) : k);
        } else {
          const int32_t r = k - nd32, e0 = m.con_ptr[(size_t)r], e1 = m.con_ptr[(size_t)r + 1];
          const int32_t start = (int32_t)phloc[q].size();
          if (e1 - e0 > 31 || start >= (1 << 26)) bad = 1;
          for (int32_t e = e0; e < e1; ++e) {
            phloc[q].push_back((uint16_t)pos(m.con_idx[(size_t)e]));
            phw[q].push_back((float)m.con_w[(size_t)e]);
          }
          sl.push_back((start << 5) | (e1 - e0));
        }
      }
      while (sl.size() % 4) sl.push_back(0);
    }
  }
  // concatenation in the patch numbering
  size_t ns = 0, nh = 0;
  o.ptr.resize(np);
  o.cnt.resize(4 * np);
  for (size_t q = 0; q < np; ++q) {
    const int32_t nu = (int32_t)keys[(size_t)porder[q]].size();
    o.ptr[q] = (int32_t)ns;
    o.cnt[4 * q] = pnfree[q];
    o.cnt[4 * q + 1] = nu;
    o.cnt[4 * q + 2] = (int32_t)nh;
    o.cnt[4 * q + 3] = (int32_t)(nh + phloc[q].size());
    o.max_nu = std::max(o.max_nu, (int)nu);
    o.max_hent = std::max(o.max_hent, (int)phloc[q].size());
    ns += pslot[q].size();
    nh += phloc[q].size();
  }
  o.slot.resize(ns);
  o.hloc.resize(nh);
  o.hw.resize(nh);
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t qq = 0; qq < (int64_t)np; ++qq) {
    const size_t q = (size_t)qq;
    std::copy(pslot[q].begin(), pslot[q].end(), o.slot.begin() + o.ptr[q]);
    std::copy(phloc[q].begin(), phloc[q].end(), o.hloc.begin() + o.cnt[4 * q + 2]);
    std::copy(phw[q].begin(), phw[q].end(), o.hw.begin() + o.cnt[4 * q + 2]);
  }
  // every dof needs an owner (each lies in an active cell), and shared-memory positions are
  // 16-bit; otherwise the context has no fused form
  bool ok = !bad && std::find(owner.begin(), owner.end(), INT_MAX) == owner.end();
  if (ok && ((o.max_nu + 31) & ~31) > 65536) ok = false;
  if (!ok) out = StepHost();
}

}  // namespace pbf
