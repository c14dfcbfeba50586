// C ABI of the library (include/pbf.h): mesh objects, device contexts and the hot-path
// entry points. Host orchestration only; every step of the path runs in the kernels of
// kernels_cell.cu and vec_kernels.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "internal.cuh"
#include "mesh.hpp"
#include "pbf.h"
#include "solver.hpp"
#include "step_layout.hpp"
#include "vec_kernels.cuh"

using namespace pbf;

namespace {
thread_local std::string g_err;

pbf_status fail(pbf_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}
}  // namespace

namespace pbf {
pbf_status set_error(pbf_status s, const char* msg) {
  g_err = msg;
  return s;
}
}  // namespace pbf

struct pbf_mesh {
  HostMesh m;
};

extern "C" const char* pbf_last_error(void) { return g_err.c_str(); }
extern "C" const char* pbf_version(void) { return "pbf-gb300 0.1 (sm_103a)"; }

// ======================================================================================
// mesh
// ======================================================================================

extern "C" pbf_status pbf_mesh_create(const pbf_mesh_desc* desc, pbf_mesh** out) {
  if (!desc || !out) return fail(PBF_EINVAL, "null argument");
  *out = nullptr;
  try {
    std::unique_ptr<pbf_mesh> mh(new pbf_mesh());
    std::string err;
    pbf_status st = init_mesh(mh->m, *desc, &err);
    if (st != PBF_OK) return fail(st, "%s", err.c_str());
    st = build_mesh(mh->m, nullptr, &err);
    if (st != PBF_OK) return fail(st, "%s", err.c_str());
    *out = mh.release();
    return PBF_OK;
  } catch (const std::bad_alloc&) {
    return fail(PBF_ENOMEM, "host allocation failed");
  }
}

extern "C" pbf_status pbf_mesh_destroy(pbf_mesh* mesh) {
  delete mesh;
  return PBF_OK;
}

extern "C" pbf_status pbf_mesh_info(const pbf_mesh* mesh, pbf_mesh_info_t* out) {
  if (!mesh || !out) return fail(PBF_EINVAL, "null argument");
  const HostMesh& m = mesh->m;
  out->n_leaves = (int64_t)m.oct.size();
  out->n_active = (int64_t)m.leaf_of_active.size();
  out->n_dofs = m.n_dofs;
  out->n_hanging = (int64_t)m.con_ptr.size() - 1;
  out->n_con_entries = (int64_t)m.con_idx.size();
  out->n_colours = m.n_colours;
  out->n_top_faces = m.n_top;
  out->nodes_per_cell = m.npc;
  out->generation = m.generation;
  return PBF_OK;
}

extern "C" pbf_status pbf_mesh_export(const pbf_mesh* mesh, const pbf_mesh_tables* t) {
  if (!mesh || !t) return fail(PBF_EINVAL, "null argument");
  const HostMesh& m = mesh->m;
  if (t->leaves)
    for (size_t i = 0; i < m.oct.size(); ++i) {
      for (int a = 0; a < 3; ++a) t->leaves[i * 5 + a] = m.oct[i].a[a];
      t->leaves[i * 5 + 3] = m.oct[i].level;
      t->leaves[i * 5 + 4] = m.active[i];
    }
  if (t->material) std::memcpy(t->material, m.material.data(), m.material.size());
  if (t->cell_dofs) std::memcpy(t->cell_dofs, m.cell_dofs.data(), m.cell_dofs.size() * 4);
  if (t->con_ptr) std::memcpy(t->con_ptr, m.con_ptr.data(), m.con_ptr.size() * 4);
  if (t->con_idx) std::memcpy(t->con_idx, m.con_idx.data(), m.con_idx.size() * 4);
  if (t->con_w) std::memcpy(t->con_w, m.con_w.data(), m.con_w.size() * 8);
  if (t->hang_coord) std::memcpy(t->hang_coord, m.hang_xyz.data(), m.hang_xyz.size() * 8);
  if (t->dof_coord) std::memcpy(t->dof_coord, m.dof_xyz.data(), m.dof_xyz.size() * 8);
  if (t->dirichlet) std::memcpy(t->dirichlet, m.dirichlet.data(), m.dirichlet.size());
  if (t->colour) std::memcpy(t->colour, m.colour.data(), m.colour.size() * 4);
  if (t->top) std::memcpy(t->top, m.top.data(), m.top.size());
  return PBF_OK;
}

extern "C" pbf_status pbf_mesh_step_tables(const pbf_mesh* mesh, pbf_step_tables* t) {
  if (!mesh || !t) return fail(PBF_EINVAL, "null argument");
  try {
    StepHost sh;
    build_step_tables(mesh->m, sh);
    const int64_t np = (int64_t)sh.ptr.size(), ns = (int64_t)sh.slot.size(), nh = (int64_t)sh.hloc.size();
    const bool fill = t->ptr || t->cnt || t->slot || t->cell || t->loc || t->hloc || t->hw;
    if (fill && (t->n_patches != np || t->n_slots != ns || t->n_hent != nh))
      return fail(PBF_EINVAL, "table sizes (%lld, %lld, %lld) differ from the mesh's (%lld, %lld, %lld)",
                  (long long)t->n_patches, (long long)t->n_slots, (long long)t->n_hent, (long long)np,
                  (long long)ns, (long long)nh);
    t->n_patches = np;
    t->n_slots = ns;
    t->n_hent = nh;
    t->cells_per_patch = kStepCells;
    t->max_slots = sh.max_nu;
    t->max_hent = sh.max_hent;
    if (t->ptr) std::memcpy(t->ptr, sh.ptr.data(), sh.ptr.size() * 4);
    if (t->cnt) std::memcpy(t->cnt, sh.cnt.data(), sh.cnt.size() * 4);
    if (t->slot) std::memcpy(t->slot, sh.slot.data(), sh.slot.size() * 4);
    if (t->cell) std::memcpy(t->cell, sh.cell.data(), sh.cell.size() * 4);
    if (t->loc) std::memcpy(t->loc, sh.loc.data(), sh.loc.size() * 2);
    if (t->hloc) std::memcpy(t->hloc, sh.hloc.data(), sh.hloc.size() * 2);
    if (t->hw) std::memcpy(t->hw, sh.hw.data(), sh.hw.size() * 4);
    return PBF_OK;
  } catch (const std::bad_alloc&) {
    return fail(PBF_ENOMEM, "host allocation failed");
  }
}

extern "C" pbf_status pbf_mesh_activate_layer(pbf_mesh* mesh, double z_new_top, int material, double T_init) {
  if (!mesh) return fail(PBF_EINVAL, "null mesh");
  if (material < 0 || material > 1) return fail(PBF_EINVAL, "material must be 0 or 1");
  try {
    HostMesh& old = mesh->m;
    if (!(z_new_top >= old.desc.active_top_z)) return fail(PBF_EINVAL, "activation height must not decrease");
    HostMesh nm;
    std::string err;
    pbf_mesh_desc d = old.desc;
    d.tree_exists = old.exists.empty() ? nullptr : old.exists.data();
    d.regions = old.regions.data();
    d.n_regions = (int)old.regions.size();
    d.active_top_z = z_new_top;
    pbf_status st = init_mesh(nm, d, &err);
    if (st != PBF_OK) return fail(st, "%s", err.c_str());
    // same leaves; previously active cells keep their material, new ones take `material`
    std::vector<uint8_t> mat(old.material);
    for (size_t i = 0; i < old.oct.size(); ++i) {
      double z0 = old.coord(2, old.oct[i].a[2]);
      if (!old.active[i] && z0 < z_new_top) mat[i] = (uint8_t)material;
    }
    st = build_mesh(nm, &mat, &err);
    if (st != PBF_OK) return fail(st, "%s", err.c_str());
    nm.generation = old.generation + 1;
    make_transfer(old, nm, T_init, nm.transfer);
    make_history_map(old, nm, nm.history_map);
    nm.history_old_cells = (int64_t)old.leaf_of_active.size();
    mesh->m = std::move(nm);
    return PBF_OK;
  } catch (const std::bad_alloc&) {
    return fail(PBF_ENOMEM, "host allocation failed");
  }
}

static pbf_status adapt_impl(pbf_mesh* mesh, const std::vector<pbf_region>& regions) {
  try {
    HostMesh& old = mesh->m;
    HostMesh nm;
    std::string err;
    pbf_mesh_desc d = old.desc;
    d.tree_exists = old.exists.empty() ? nullptr : old.exists.data();
    d.regions = regions.empty() ? nullptr : regions.data();
    d.n_regions = (int)regions.size();
    pbf_status st = init_mesh(nm, d, &err);
    if (st != PBF_OK) return fail(st, "%s", err.c_str());
    st = build_mesh(nm, nullptr, &err);
    if (st != PBF_OK) return fail(st, "%s", err.c_str());
    // materials from the old leaves (nothing else of the mesh depends on them)
    for (size_t i = 0; i < nm.oct.size(); ++i) {
      int64_t j = old.locate(nm.oct[i].a);
      nm.material[i] = j >= 0 ? old.material[(size_t)j] : 0;
    }
    nm.generation = old.generation + 1;
    make_transfer(old, nm, 0.0, nm.transfer);  // same activation: every new dof lies in the old domain
    make_history_map(old, nm, nm.history_map);
    nm.history_old_cells = (int64_t)old.leaf_of_active.size();
    mesh->m = std::move(nm);
    return PBF_OK;
  } catch (const std::bad_alloc&) {
    return fail(PBF_ENOMEM, "host allocation failed");
  }
}

extern "C" pbf_status pbf_mesh_adapt(pbf_mesh* mesh, int n_regions, const pbf_region* regions) {
  if (!mesh || (n_regions > 0 && !regions) || n_regions < 0) return fail(PBF_EINVAL, "bad arguments");
  return adapt_impl(mesh, std::vector<pbf_region>(regions, regions + n_regions));
}

extern "C" pbf_status pbf_mesh_adapt_gated(pbf_mesh* mesh, int n_regions, const pbf_region* regions,
                                           const double* cell_rc_min, double r_coarsen) {
  if (!mesh || (n_regions > 0 && !regions) || n_regions < 0 || !cell_rc_min || !(r_coarsen >= 0.0))
    return fail(PBF_EINVAL, "bad arguments");
  try {
    std::vector<pbf_region> all(regions, regions + n_regions);
    gate_pins(mesh->m, cell_rc_min, r_coarsen, all);
    return adapt_impl(mesh, all);
  } catch (const std::bad_alloc&) {
    return fail(PBF_ENOMEM, "host allocation failed");
  }
}

extern "C" pbf_status pbf_mesh_transfer(pbf_mesh* mesh, const double* T_old_dev, double* T_new_dev, int batch,
                                        pbf_stream stream) {
  if (!mesh || !T_old_dev || !T_new_dev || batch < 1) return fail(PBF_EINVAL, "bad arguments");
  TransferMap& tr = mesh->m.transfer;
  if (!tr.pending) return fail(PBF_ESTATE, "no pending transfer");
  cudaStream_t s = (cudaStream_t)stream;
  int32_t *ptr = nullptr, *idx = nullptr;
  double* w = nullptr;
  auto cleanup = [&]() {
    cudaFree(ptr);
    cudaFree(idx);
    cudaFree(w);
  };
  if (cudaMalloc(&ptr, tr.ptr.size() * 4) != cudaSuccess || cudaMalloc(&idx, std::max<size_t>(1, tr.idx.size()) * 4) != cudaSuccess ||
      cudaMalloc(&w, std::max<size_t>(1, tr.w.size()) * 8) != cudaSuccess) {
    cleanup();
    return fail(PBF_ENOMEM, "device allocation failed");
  }
  cudaError_t e = cudaMemcpyAsync(ptr, tr.ptr.data(), tr.ptr.size() * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !tr.idx.empty()) e = cudaMemcpyAsync(idx, tr.idx.data(), tr.idx.size() * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !tr.w.empty()) e = cudaMemcpyAsync(w, tr.w.data(), tr.w.size() * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_transfer(tr.n_new, batch, ptr, idx, w, T_old_dev, tr.fill, T_new_dev, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cleanup();
  if (e != cudaSuccess) return fail(PBF_ECUDA, "transfer: %s", cudaGetErrorString(e));
  tr.pending = false;
  return PBF_OK;
}

extern "C" pbf_status pbf_mesh_history_map(const pbf_mesh* mesh, int64_t* n_old_cells_out, int32_t* map) {
  if (!mesh) return fail(PBF_EINVAL, "null mesh");
  const HostMesh& m = mesh->m;
  if (m.generation <= 1) return fail(PBF_ESTATE, "no mesh change recorded");
  if (n_old_cells_out) *n_old_cells_out = m.history_old_cells;
  if (map) std::memcpy(map, m.history_map.data(), m.history_map.size() * 4);
  return PBF_OK;
}

extern "C" pbf_status pbf_mesh_transfer_map(const pbf_mesh* mesh, pbf_transfer_map* t) {
  if (!mesh || !t) return fail(PBF_EINVAL, "null argument");
  const TransferMap& tr = mesh->m.transfer;
  if (!tr.pending) return fail(PBF_ESTATE, "no pending transfer");
  const int64_t ne = (int64_t)tr.idx.size();
  if ((t->ptr || t->idx || t->w) && (t->n_old != tr.n_old || t->n_new != tr.n_new || t->n_entries != ne))
    return fail(PBF_EINVAL, "map sizes (%lld, %lld, %lld) differ from the mesh's (%lld, %lld, %lld)",
                (long long)t->n_old, (long long)t->n_new, (long long)t->n_entries, (long long)tr.n_old,
                (long long)tr.n_new, (long long)ne);
  t->n_old = tr.n_old;
  t->n_new = tr.n_new;
  t->n_entries = ne;
  t->fill = tr.fill;
  if (t->ptr) std::memcpy(t->ptr, tr.ptr.data(), tr.ptr.size() * 4);
  if (t->idx) std::memcpy(t->idx, tr.idx.data(), tr.idx.size() * 4);
  if (t->w) std::memcpy(t->w, tr.w.data(), tr.w.size() * 8);
  return PBF_OK;
}

// ======================================================================================
// context
// ======================================================================================

pbf_status pbf_ctx_impl_create(const pbf_mesh* mesh, const pbf_material* mat, pbf_precision prec, int batch,
                               pbf_ctx** out);

extern "C" pbf_status pbf_ctx_create(const pbf_mesh* mesh, const pbf_material* mat, pbf_precision prec, int batch,
                                     pbf_ctx** out) {
  if (!mesh || !mat || !out) return fail(PBF_EINVAL, "null argument");
  if (batch < 1 || batch > 1024) return fail(PBF_EINVAL, "batch must be in [1, 1024]");
  if (prec != PBF_F64 && prec != PBF_F32OP) return fail(PBF_EINVAL, "bad precision");
  if (!(mat->rho > 0) || !(mat->c > 0) || !(mat->k0 > 0)) return fail(PBF_EINVAL, "rho, c, k0 must be positive");
  return pbf_ctx_impl_create(mesh, mat, prec, batch, out);
}

// ---- context object ---------------------------------------------------------------------

struct pbf_ctx : public CtxBase {};

namespace {

template <typename T>
cudaError_t dalloc(pbf_ctx* c, T** p, size_t n) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(1, n) * sizeof(T));
  if (e == cudaSuccess) {
    c->allocs.push_back(q);
    *p = (T*)q;
  }
  return e;
}

template <typename T>
cudaError_t upload(pbf_ctx* c, T** p, const T* src, size_t n) {
  cudaError_t e = dalloc(c, p, n);
  if (e == cudaSuccess && n) e = cudaMemcpy(*p, src, n * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

}  // namespace

pbf_status pbf_ctx_impl_create(const pbf_mesh* mesh, const pbf_material* mat, pbf_precision prec, int batch,
                               pbf_ctx** out) {
  const HostMesh& m = mesh->m;
  std::unique_ptr<pbf_ctx> c(new pbf_ctx());
  c->mesh = &mesh->m;
  c->generation = m.generation;
  c->degree = m.p;
  c->npc = m.npc;
  c->batch = batch;
  c->n_dofs = m.n_dofs;
  c->n_cells = (int64_t)m.leaf_of_active.size();
  c->n_hang = (int64_t)m.con_ptr.size() - 1;
  c->f32 = prec == PBF_F32OP;
  c->mat = *mat;
  const bool has_latent = mat->sigma > 0.0 && mat->latent != 0.0;
  if (mat->lumping != PBF_LUMP_QUADRATURE && mat->lumping != PBF_LUMP_NODAL) return fail(PBF_EINVAL, "bad lumping");
  c->cap = !has_latent ? CAP_CONST : (mat->lumping == PBF_LUMP_NODAL ? CAP_NODAL : CAP_QUADRATURE);
  c->latent = c->cap == CAP_QUADRATURE;  // capacity integrated by the cell kernel
  if (has_latent) {
    const double lat_norm = mat->latent / (mat->sigma * std::sqrt(2.0 * kPi));
    c->nodal.lat_ratio = lat_norm / mat->c;
    c->nodal.Tm = mat->Tm;
    c->nodal.inv_sigma = 1.0 / mat->sigma;
    c->nodal.lat_ratio_f = (float)c->nodal.lat_ratio;
    c->nodal.tm_off_f = (float)(mat->T_ref - mat->Tm);
    c->nodal.inv_sigma_f = (float)c->nodal.inv_sigma;
    // lat_ratio exp(-z^2/2) < 2^-26 for z^2 > 2 (ln lat_ratio + 26 ln 2); one more unit of
    // margin for the approximate exponential
    c->nodal.z2_cut_f = c->nodal.lat_ratio > 0.0
                            ? (float)(2.0 * (std::log(c->nodal.lat_ratio) + 26.0 * std::log(2.0)) + 1.0)
                            : 0.f;
  }
  c->nonlin = mat->Tk1 > mat->Tk0 && mat->k1 != mat->k0;
  // kernels index with 32-bit integers: every (entity x instance) count stays below 2^31
  if (c->n_cells * (int64_t)c->npc >= ((int64_t)1 << 31) || c->n_dofs * (int64_t)batch >= ((int64_t)1 << 31) ||
      c->n_cells * (int64_t)batch * c->npc >= ((int64_t)1 << 31) || c->n_hang * (int64_t)batch >= ((int64_t)1 << 31))
    return fail(PBF_EINVAL, "mesh x batch too large for 32-bit indexing");
  const size_t nc = (size_t)c->n_cells, npc = (size_t)c->npc, nd = (size_t)c->n_dofs;
  // host staging of per-cell tables
  std::vector<int32_t> soa(nc * npc);
  for (size_t e = 0; e < nc; ++e)
    for (size_t a = 0; a < npc; ++a) soa[a * nc + e] = m.cell_dofs[e * npc + a];
  std::vector<uint8_t> lvl(nc), cm(nc);
  std::vector<double> lo(nc * 3);
  std::vector<int32_t> top_cell;
  std::vector<double> top_geo;
  for (size_t e = 0; e < nc; ++e) {
    const Octant& o = m.oct[(size_t)m.leaf_of_active[e]];
    lvl[e] = (uint8_t)o.level;
    cm[e] = m.material[(size_t)m.leaf_of_active[e]];
    for (int a = 0; a < 3; ++a) lo[e * 3 + a] = m.coord(a, o.a[a]);
    if (m.top[e]) {
      top_cell.push_back((int32_t)e);
      const int64_t s = m.size(o);
      top_geo.push_back(m.coord(0, o.a[0]));
      top_geo.push_back(m.coord(1, o.a[1]));
      top_geo.push_back(m.coord(0, o.a[0] + s) - m.coord(0, o.a[0]));
      top_geo.push_back(m.coord(1, o.a[1] + s) - m.coord(1, o.a[1]));
    }
  }
  std::vector<float> con_wf(m.con_w.begin(), m.con_w.end());
  std::vector<uint8_t> ctop(m.top.begin(), m.top.end());
  std::vector<float> lof(lo.size());
  for (size_t e = 0; e < nc; ++e)
    for (int a = 0; a < 3; ++a) lof[e * 3 + a] = (float)lo[e * 3 + a];
  // patch tables of the fused step kernel (one instance, FP32 operator)
  StepHost sh;
  if (batch == 1 && prec == PBF_F32OP && nc > 0) build_step_tables(m, sh);
  std::vector<int32_t>& sptr = sh.ptr;
  std::vector<int32_t>& scnt = sh.cnt;
  std::vector<int32_t>& sslot = sh.slot;
  std::vector<int32_t>& scell = sh.cell;
  std::vector<uint16_t>& sloc = sh.loc;
  std::vector<uint16_t>& shloc = sh.hloc;
  std::vector<float>& shw = sh.hw;
  const int max_nu = sh.max_nu;
  int32_t *d_sptr = nullptr, *d_scnt = nullptr, *d_sslot = nullptr, *d_scell = nullptr;
  uint16_t *d_sloc = nullptr, *d_shloc = nullptr;
  float* d_shw = nullptr;
  std::vector<double> level_h((size_t)kMaxLevels * 3, 0.0);
  CellLaunch& L = c->base;
  for (int l = 0; l <= m.L && l < kMaxLevels; ++l) {
    double h[3];
    for (int a = 0; a < 3; ++a) h[a] = m.desc.tree_h[a] / (double)((int64_t)1 << l);
    double detJ = h[0] * h[1] * h[2];
    L.gd.detJ[l] = detJ;
    L.gf.detJ[l] = (float)detJ;
    for (int a = 0; a < 3; ++a) {
      L.gd.h[l][a] = h[a];
      L.gf.h[l][a] = (float)h[a];
      level_h[(size_t)l * 3 + a] = h[a];
      L.gd.ih2[l][a] = 1.0 / (h[a] * h[a]);
      L.gf.ih2[l][a] = (float)(1.0 / (h[a] * h[a]));
    }
  }
  cudaError_t e = cudaSuccess;
#define UP(ptr, vec) \
  if (e == cudaSuccess) e = upload(c.get(), &ptr, vec.data(), vec.size())
  UP(c->cell_dofs, soa);
  UP(c->cell_level, lvl);
  UP(c->cell_mat, cm);
  UP(c->con_ptr, m.con_ptr);
  UP(c->con_idx, m.con_idx);
  UP(c->con_w, m.con_w);
  UP(c->con_wf, con_wf);
  UP(c->dirichlet, m.dirichlet);
  UP(c->top_cell, top_cell);
  UP(c->top_geo, top_geo);
  UP(c->cell_lo, lo);
  UP(c->level_h, level_h);
  UP(c->cell_top, ctop);
  UP(c->cell_lof, lof);
  UP(d_sptr, sptr);
  UP(d_scnt, scnt);
  UP(d_sslot, sslot);
  UP(d_scell, scell);
  UP(d_sloc, sloc);
  UP(d_shloc, shloc);
  UP(d_shw, shw);
#undef UP
  c->n_top = (int64_t)top_cell.size();
  const size_t rsz = c->f32 ? 4 : 8;
  const size_t nv = nd * (size_t)batch;
  if (e == cudaSuccess) e = dalloc(c.get(), (char**)&c->f, nv * rsz);
  if (e == cudaSuccess) e = dalloc(c.get(), (char**)&c->fvol, nv * rsz);
  if (e == cudaSuccess) e = dalloc(c.get(), (char**)&c->Cacc, (c->latent ? nv : 1) * rsz);
  if (e == cudaSuccess && c->f32) e = dalloc(c.get(), &c->Tlo, nv);
  if (e == cudaSuccess && c->f32) e = dalloc(c.get(), &c->Tf, nv);
  const size_t nh = std::max<size_t>(1, (size_t)c->n_hang * (size_t)batch);
  if (e == cudaSuccess) e = dalloc(c.get(), (char**)&c->xh, nh * rsz);
  if (e == cudaSuccess) e = dalloc(c.get(), (char**)&c->fh, nh * rsz);
  if (e == cudaSuccess) e = dalloc(c.get(), (char**)&c->Ch, nh * rsz);
  if (e == cudaSuccess) e = dalloc(c.get(), &c->xh64, nh);
  if (e == cudaSuccess) e = dalloc(c.get(), &c->fh64, nh);
  if (e == cudaSuccess) e = dalloc(c.get(), &c->Ch64, nh);
  if (e == cudaSuccess) e = cudaMemset(c->fh, 0, nh * rsz);
  if (e == cudaSuccess) e = cudaMemset(c->Ch, 0, nh * rsz);
  if (e == cudaSuccess) e = cudaMemset(c->fh64, 0, nh * 8);
  if (e == cudaSuccess) e = cudaMemset(c->Ch64, 0, nh * 8);
  if (e == cudaSuccess) e = dalloc(c.get(), &c->C0, nd);
  if (e == cudaSuccess) e = dalloc(c.get(), &c->invC0_d, nd);
  if (e == cudaSuccess) e = dalloc(c.get(), &c->invC0_f, nd);
  // FP32 1 / C~ with the Dirichlet flag: read by the fused steps of one instance and of a batch
  if (e == cudaSuccess && c->f32) e = dalloc(c.get(), &c->invC0_fx, nd);
  if (e == cudaSuccess) e = dalloc(c.get(), &c->power, (size_t)batch * kMaxSeg);
  if (e == cudaSuccess) e = dalloc(c.get(), &c->powerf, (size_t)batch * kMaxSeg);
  if (e == cudaSuccess) e = dalloc(c.get(), &c->part, (size_t)reduction_blocks() * batch);
  if (e == cudaSuccess) e = dalloc(c.get(), &c->scal, (size_t)batch * 16);
  c->k_scale_host.assign((size_t)batch, 1.0);
  std::vector<float> ksf((size_t)batch, 1.0f);
  if (e == cudaSuccess) e = upload(c.get(), &c->k_scale_d, c->k_scale_host.data(), (size_t)batch);
  if (e == cudaSuccess) e = upload(c.get(), &c->k_scale_f, ksf.data(), (size_t)batch);
  if (e == cudaSuccess) e = cudaMemset(c->f, 0, nv * rsz);
  if (e == cudaSuccess) e = cudaMemset(c->fvol, 0, nv * rsz);
  if (e == cudaSuccess) e = cudaMemset(c->Cacc, 0, (c->latent ? nv : 1) * rsz);
  if (e == cudaSuccess) e = cudaMemset(c->C0, 0, nd * 8);
  if (e == cudaSuccess) e = cudaMemset(c->power, 0, (size_t)batch * kMaxSeg * 8);
  if (e != cudaSuccess) {
    cudaGetLastError();  // do not leave the error for the next caller's launch check
    c->release();
    return fail(e == cudaErrorMemoryAllocation ? PBF_ENOMEM : PBF_ECUDA, "context setup: %s", cudaGetErrorString(e));
  }
  // launch template
  DevMesh& M = L.mesh;
  M.n_cells = (int)c->n_cells;
  M.npc = c->npc;
  M.n_dofs = (int)c->n_dofs;
  M.n_hang = (int)c->n_hang;
  M.batch = batch;
  M.cell_dofs = c->cell_dofs;
  M.cell_level = c->cell_level;
  M.cell_mat = c->cell_mat;
  M.con_ptr = c->con_ptr;
  M.con_idx = c->con_idx;
  M.con_w = c->con_w;
  M.con_wf = c->con_wf;
  M.dirichlet = c->dirichlet;
  M.cell_top = c->cell_top;
  M.cell_lo = c->cell_lo;
  M.cell_lof = c->cell_lof;
  if (!sptr.empty()) {
    StepTables& st = c->step;
    st.n_patches = (int)sptr.size();
    st.max_nu32 = (max_nu + 31) & ~31;
    st.max_hent8 = (sh.max_hent + 7) & ~7;
    st.smem = step_smem_bytes((int)npc, st.max_nu32, st.max_hent8);
    st.ptr = d_sptr;
    st.cnt = reinterpret_cast<const int4*>(d_scnt);
    st.slot = d_sslot;
    st.cell = d_scell;
    st.loc = d_sloc;
    st.hloc = d_shloc;
    st.hw = d_shw;
    c->fstep[0] = (float*)c->f;
    cudaError_t e2 = dalloc(c.get(), &c->fstep[1], nd);
    if (e2 == cudaSuccess) e2 = dalloc(c.get(), &c->fstep[2], nd);
    if (e2 == cudaSuccess) e2 = dalloc(c.get(), &c->xstep[0], nd);
    if (e2 == cudaSuccess) e2 = dalloc(c.get(), &c->xstep[1], nd);
    if (e2 == cudaSuccess) e2 = dalloc(c.get(), &c->bar, 1);
    if (e2 == cudaSuccess) e2 = cudaMemset(c->bar, 0, sizeof(GridBarrier));
    if (e2 == cudaSuccess) e2 = cudaMemset(c->fstep[1], 0, nd * 4);
    if (e2 == cudaSuccess) e2 = cudaMemset(c->fstep[2], 0, nd * 4);
    if (e2 != cudaSuccess) {
      cudaGetLastError();
      c->release();
      return fail(e2 == cudaErrorMemoryAllocation ? PBF_ENOMEM : PBF_ECUDA, "context setup: %s",
                  cudaGetErrorString(e2));
    }
  }
  L.degree = c->degree;
  L.f32 = c->f32;
  L.nonlin_k = c->nonlin;
  L.latent = c->latent;
  L.k_scale_d = c->k_scale_d;
  L.k_scale_f = c->k_scale_f;
  c->set_material_constants(0.0);
  c->lsetup.n_top = (int)c->n_top;
  c->lsetup.top_cell = c->top_cell;
  c->lsetup.top_geo = c->top_geo;
  c->lsetup.cell_lo = c->cell_lo;
  c->lsetup.level_h = c->level_h;
  // constant-c lumped capacity and its inverse (FP64, once)
  {
    CellLaunch Lc = L;
    Lc.f32 = 0;
    Lc.latent = 0;
    Lc.mesh.batch = 1;
    Lc.offset = mat->T_ref;
    std::vector<double> zero(nd, mat->T_ref);
    double* Tz = nullptr;
    e = cudaMalloc(&Tz, std::max<size_t>(1, nd) * 8);
    if (e == cudaSuccess) e = cudaMemcpy(Tz, zero.data(), nd * 8, cudaMemcpyHostToDevice);
    Lc.x = Tz;
    if (e == cudaSuccess) e = c->apply_cell(Lc, nullptr, c->C0, MODE_CAPACITY, 0);
    if (e == cudaSuccess) e = launch_reciprocal((int64_t)nd, c->C0, c->invC0_d, c->invC0_f, c->invC0_fx, c->dirichlet, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(Tz);
    c->launches += 2;
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->release();
      return fail(PBF_ECUDA, "capacity setup: %s", cudaGetErrorString(e));
    }
  }
  // the allocation-free entry point's one-time set-up on this device
  const pbf_status pst = noalloc_prepare(c.get());
  if (pst != PBF_OK) {
    c->release();
    return pst;
  }
  *out = c.release();
  return PBF_OK;
}

void CtxBase::set_material_constants(double dt) {
  CellLaunch& L = base;
  const pbf_material& mt = mat;
  MatR<double> d;
  d.rho = mt.rho;
  d.c = mt.c;
  d.lat_norm = latent ? mt.latent / (mt.sigma * std::sqrt(2.0 * kPi)) : 0.0;
  d.tm_off = mt.T_ref - mt.Tm;
  d.inv_sigma = latent ? 1.0 / mt.sigma : 0.0;
  d.k0 = mt.k0;
  d.dk = nonlin ? mt.k1 - mt.k0 : 0.0;
  d.tk_off = mt.T_ref - mt.Tk0;
  d.inv_dT = nonlin ? 1.0 / (mt.Tk1 - mt.Tk0) : 0.0;
  d.powder_scale = mt.powder_k_scale;
  d.m_impl = dt > 0 ? mt.rho * mt.c / dt : 0.0;
  L.md = d;
  L.mf.rho = (float)d.rho;
  L.mf.c = (float)d.c;
  L.mf.lat_norm = (float)d.lat_norm;
  L.mf.tm_off = (float)d.tm_off;
  L.mf.inv_sigma = (float)d.inv_sigma;
  L.mf.k0 = (float)d.k0;
  L.mf.dk = (float)d.dk;
  L.mf.tk_off = (float)d.tk_off;
  L.mf.inv_dT = (float)d.inv_dT;
  L.mf.powder_scale = (float)d.powder_scale;
  L.mf.m_impl = (float)d.m_impl;
  L.offset = mt.T_ref;
}

void CtxBase::release() {
  for (GraphSlot* g : {&cheb_graph, &iter_graph, &bstep_graph}) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
  }
  if (cap_stream) cudaStreamDestroy(cap_stream);
  cap_stream = nullptr;
  if (pinned) cudaFreeHost(pinned);
  pinned = nullptr;
  for (void* p : allocs) cudaFree(p);
  allocs.clear();
  for (auto& ev : events) {
    cudaEventDestroy(ev.first);
    cudaEventDestroy(ev.second);
  }
  events.clear();
}

extern "C" pbf_status pbf_ctx_destroy(pbf_ctx* ctx) {
  if (!ctx) return PBF_OK;
  ctx->release();
  delete ctx;
  return PBF_OK;
}

pbf_status CtxBase::check_usable() {
  if (poisoned) return fail(PBF_ESTATE, "context is poisoned by an earlier CUDA error");
  if (mesh->generation != generation) return fail(PBF_ESTATE, "mesh changed since the context was created");
  return PBF_OK;
}

pbf_status CtxBase::cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PBF_OK;
  if (barrier_timed_out) {  // a bounded device wait expired: no CUDA error, the context stays usable
    barrier_timed_out = false;
    return fail(PBF_ETIMEOUT, "%s: a grid barrier wait ran out of time (state left undefined)", what);
  }
  cudaGetLastError();
  poisoned = true;
  return fail(PBF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

extern "C" pbf_status pbf_ctx_set_k_scale(pbf_ctx* ctx, const double* s_host) {
  if (!ctx || !s_host) return fail(PBF_EINVAL, "null argument");
  pbf_status st = ctx->check_usable();
  if (st) return st;
  std::vector<float> f((size_t)ctx->batch);
  for (int b = 0; b < ctx->batch; ++b) {
    if (!(s_host[b] > 0)) return fail(PBF_EINVAL, "k scale must be positive");
    ctx->k_scale_host[(size_t)b] = s_host[b];
    f[(size_t)b] = (float)s_host[b];
  }
  cudaError_t e = cudaMemcpy(ctx->k_scale_d, s_host, (size_t)ctx->batch * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ctx->k_scale_f, f.data(), (size_t)ctx->batch * 4, cudaMemcpyHostToDevice);
  // the implicit operator's diagonal depends on s: rebuild it on the next solve (the CG graphs
  // read s and the diagonal through their device pointers and stay valid)
  ctx->diag_dt = -1.0;
  return ctx->cuda(e, "set_k_scale");
}

pbf_status CtxBase::set_laser(const pbf_laser* ls, cudaStream_t s) {
  LaserK& k = lsetup.k;
  if (!ls || ls->n_seg == 0) {
    k.n_seg = 0;
    return PBF_OK;
  }
  if (ls->n_seg < 0 || ls->n_seg > kMaxSeg || !ls->seg || !ls->power) return fail(PBF_EINVAL, "bad laser description");
  if (!(ls->radius > 0)) return fail(PBF_EINVAL, "laser radius must be positive");
  k.n_seg = ls->n_seg;
  k.volumetric = ls->volumetric;
  k.eta = ls->eta;
  k.radius = ls->radius;
  k.h_powder = ls->h_powder;
  k.z_top = mesh->desc.active_top_z;
  for (int i = 0; i < ls->n_seg; ++i)
    for (int j = 0; j < 6; ++j) k.seg[i][j] = ls->seg[i * 6 + j];
  std::vector<double> pw((size_t)batch * kMaxSeg, 0.0);
  for (int b = 0; b < batch; ++b)
    for (int i = 0; i < ls->n_seg; ++i) pw[(size_t)b * kMaxSeg + (size_t)i] = ls->power[(size_t)b * ls->n_seg + (size_t)i];
  if (pw != power_host) {
    power_host = pw;
    std::vector<float> pf(pw.begin(), pw.end());
    cudaError_t e = cudaMemcpyAsync(power, pw.data(), pw.size() * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(powerf, pf.data(), pf.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host staging buffers go out of scope
    if (e != cudaSuccess) return cuda(e, "laser power upload");
  }
  return PBF_OK;
}

cudaError_t CtxBase::apply_cell(CellLaunch L, void* f, void* C, int mode, cudaStream_t s) {
  const bool lf32 = L.f32 != 0;
  // FP64-operator launches in an FP32 context use the FP64 hanging buffers
  void* xhb = lf32 ? xh : (f32 ? (void*)xh64 : xh);
  void* fhb = lf32 ? fh : (f32 ? (void*)fh64 : fh);
  void* Chb = lf32 ? Ch : (f32 ? (void*)Ch64 : Ch);
  cudaError_t e = launch_hang_values(lf32, L.mesh, lf32 ? (const void*)L.xf : (const void*)L.x, xhb, s);
  if (lf32) L.xfh = (const float*)xhb;
  else L.xh = (const double*)xhb;
  ++launches;
  if (e != cudaSuccess) return e;
  const auto ev = timing ? timing_begin(s) : std::pair<cudaEvent_t, cudaEvent_t>{};
  e = launch_cell(L, f, fhb, C, C ? Chb : nullptr, mode, s);
  ++launches;
  if (ev.first) timing_end(ev, s);
  if (e == cudaSuccess && f) e = launch_hang_distribute(lf32, L.mesh, fhb, f, s);
  if (e == cudaSuccess && C) e = launch_hang_distribute(lf32, L.mesh, Chb, C, s);
  launches += (f ? 1 : 0) + (C ? 1 : 0);
  return e;
}

// f_diff, f_vol and C~ at T (laser already set); FP64 outputs, accumulators left at zero.
// With fre_dev, the surface loss's part goes there and f_vol holds the laser alone.
cudaError_t CtxBase::residual_f64(const double* T_dev, double t, double* fdiff_dev, double* fvol_dev, double* C_dev,
                                  cudaStream_t s, double* fre_dev) {
  const int64_t nv = n_dofs * batch;
  const size_t rsz = f32 ? 4 : 8;
  CellLaunch L = base;
  L.x = T_dev;
  set_phase(L, false);
  cudaError_t e = cudaSuccess;
  if (f32) {
    e = launch_prepare_f32(nv, T_dev, mat.T_ref, Tf, nullptr, s);
    L.xf = Tf;
    ++launches;
  }
  if (e == cudaSuccess) e = apply_cell(L, f, latent ? Cacc : nullptr, MODE_RESIDUAL, s);
  if (e == cudaSuccess && lsetup.k.n_seg > 0) {
    e = launch_laser(degree, f32, lsetup, L.mesh, power, spot_at(lsetup.k, t), fvol, s);
    ++launches;
  }
  if (e == cudaSuccess && has_loss && !fre_dev) {
    e = launch_surface_loss(degree, f32, lsetup, L.mesh, f32 ? (const void*)Tf : (const void*)T_dev,
                            f32 ? mat.T_ref : 0.0, loss, fvol, s);
    ++launches;
  }
  if (e == cudaSuccess && fdiff_dev) e = launch_to_f64(f32, nv, f, fdiff_dev, s);
  if (e == cudaSuccess && fvol_dev) e = launch_to_f64(f32, nv, fvol, fvol_dev, s);
  if (e == cudaSuccess && C_dev) {
    if (cap == CAP_QUADRATURE) e = launch_to_f64(f32, nv, Cacc, C_dev, s);
    else if (cap == CAP_NODAL) e = launch_capacity_nodal(n_dofs, batch, C0, T_dev, nodal, C_dev, s);
    else e = launch_broadcast_dofs(n_dofs, batch, C0, C_dev, s);
  }
  launches += 3;
  if (e == cudaSuccess) e = cudaMemsetAsync(f, 0, (size_t)nv * rsz, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(fvol, 0, (size_t)nv * rsz, s);
  if (e == cudaSuccess && latent) e = cudaMemsetAsync(Cacc, 0, (size_t)nv * rsz, s);
  if (e == cudaSuccess && has_loss && fre_dev) {  // the loss alone, through the cleared f_vol buffer
    e = launch_surface_loss(degree, f32, lsetup, L.mesh, f32 ? (const void*)Tf : (const void*)T_dev,
                            f32 ? mat.T_ref : 0.0, loss, fvol, s);
    if (e == cudaSuccess) e = launch_to_f64(f32, nv, fvol, fre_dev, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(fvol, 0, (size_t)nv * rsz, s);
    launches += 2;
  }
  return e;
}

LaserInline CtxBase::inline_laser(double t, Spot* sp_out) const {
  const bool with_laser = lsetup.k.n_seg > 0;
  const Spot sp = with_laser ? spot_at(lsetup.k, t) : Spot();
  if (sp_out) *sp_out = sp;
  LaserInline las;
  if (with_laser && !lsetup.k.volumetric && sp.seg >= 0) {
    const double r = lsetup.k.radius;
    las.on = 1;
    las.seg = sp.seg;
    las.sx = sp.x;
    las.sy = sp.y;
    las.amp = 2.0 * lsetup.k.eta / (kPi * r * r);
    las.ir2 = 2.0 / (r * r);
    las.cut2 = 36.0 * r * r;
    las.power = power;
    las.powerf = powerf;
  }
  return las;
}

// A forward-Euler step sequence on T (laser already set). Per step: hanging values of the
// state (clearing the hanging accumulators), the cell kernel with the surface laser on top
// faces, the distribution of the hanging-node contributions to their masters, and the
// update.
cudaError_t CtxBase::explicit_steps(double* T_dev, double t0, double dt, int nsteps, cudaStream_t s) {
  if (nsteps <= 0) return cudaSuccess;
  if (base.variant >= 4 && bfused_ok()) return explicit_steps_bfused(T_dev, t0, dt, nsteps, s);
  if (base.variant >= 4 && fused_ok(4)) {
    if (base.variant == 6 && fused_ok(6) && !(lsetup.k.n_seg > 0 && lsetup.k.volumetric))
      return explicit_steps_persistent(T_dev, t0, dt, nsteps, s);
    const int lean = base.variant >= 7 && fused_ok(base.variant) ? base.variant - 7 : -1;
    return explicit_steps_fused(T_dev, t0, dt, nsteps, base.variant != 4, lean, s);
  }
  CellLaunch L = base;
  set_phase(L, true);
  const bool volumetric = lsetup.k.n_seg > 0 && lsetup.k.volumetric;
  const int64_t nv = n_dofs * batch;
  cudaError_t e = cudaSuccess;
  const double xd = mat.T_dirichlet - mat.T_ref;
  const float xd_hi = (float)xd;
  const float2 x_dir = make_float2(xd_hi, (float)(xd - (double)xd_hi));
  if (f32) {
    // working state T - T_ref as the FP32 pair Tf + Tlo for the whole call
    e = launch_prepare_f32(nv, T_dev, mat.T_ref, Tf, Tlo, s);
    ++launches;
    L.xf = Tf;
    L.xfh = (const float*)xh;
  } else {
    L.x = T_dev;
    L.xh = (const double*)xh;
  }
  for (int n = 0; n < nsteps && e == cudaSuccess; ++n) {
    Spot sp;
    L.las = inline_laser(t0 + n * dt, &sp);
    e = launch_hang_values_zero(f32, L.mesh, f32 ? (const void*)Tf : (const void*)T_dev, xh, fh, latent ? Ch : nullptr,
                                s);
    ++launches;
    const auto ev = timing && e == cudaSuccess ? timing_begin(s) : std::pair<cudaEvent_t, cudaEvent_t>{};
    if (e == cudaSuccess) e = launch_cell(L, f, fh, latent ? Cacc : nullptr, latent ? Ch : nullptr, MODE_RESIDUAL, s);
    ++launches;
    if (ev.first) timing_end(ev, s);
    if (e == cudaSuccess && volumetric && sp.seg >= 0) {
      e = launch_laser(degree, f32, lsetup, L.mesh, power, sp, f, s);
      ++launches;
    }
    if (e == cudaSuccess && has_loss) {  // radiation / evaporation at the state of step n
      e = launch_surface_loss(degree, f32, lsetup, L.mesh, f32 ? (const void*)Tf : (const void*)T_dev,
                              f32 ? mat.T_ref : 0.0, loss, f, s);
      ++launches;
    }
    // hanging-node contributions to their masters (P_h^T f_h), one thread per row and
    // instance with atomic additions that are contiguous over the instances; the update is
    // then a plain streaming kernel
    if (e == cudaSuccess && n_hang > 0) {
      e = launch_hang_distribute(f32, L.mesh, fh, f, s);
      ++launches;
      if (e == cudaSuccess && latent) {
        e = launch_hang_distribute(f32, L.mesh, Ch, Cacc, s);
        ++launches;
      }
    }
    if (e == cudaSuccess) {
      if (f32)
        e = launch_update_f32(cap, n_dofs, batch, Tf, Tlo, (float*)f, (float*)Cacc, invC0_f, nodal, dirichlet, x_dir,
                              (float)dt, s);
      else
        e = launch_update_f64(cap, n_dofs, batch, T_dev, (double*)f, (double*)Cacc, invC0_d, nodal, dirichlet,
                              mat.T_dirichlet, dt, s);
    }
    ++launches;
  }
  if (f32 && e == cudaSuccess) {
    e = launch_finish_f32(nv, Tf, Tlo, mat.T_ref, T_dev, s);
    ++launches;
  }
  // every accumulator is zero between calls: the distribution cleared f_h and C_h
  return e;
}

// The fused sequence: step n (one launch) completes step n-1 while staging its patches and
// accumulates f_n; a last streaming kernel completes step N-1 and writes T. Accumulators
// rotate through fstep[n % 3] (f_n), fstep[(n + 1) % 3] (cleared for step n+1) and
// fstep[(n + 2) % 3] (f_{n-1}, read); the state, T - T_ref as an FP32 pair hi + lo, alternates
// between xstep[0] and xstep[1].
cudaError_t CtxBase::explicit_steps_fused(double* T_dev, double t0, double dt, int nsteps, bool pdl, int lean,
                                          cudaStream_t s) {
  CellLaunch L = base;
  set_phase(L, true);  // the phase model's history is read and stored by every step
  const bool volumetric = lsetup.k.n_seg > 0 && lsetup.k.volumetric;
  const double xd = mat.T_dirichlet - mat.T_ref;
  const float xd_hi = (float)xd;
  const float2 x_dir = make_float2(xd_hi, (float)(xd - (double)xd_hi));
  cudaError_t e = cudaSuccess;
  StepState st;
  st.T0 = T_dev;
  st.off = mat.T_ref;
  st.invC0x = invC0_fx;
  st.nc = nodal;
  st.x_dir = x_dir;
  st.dt = (float)dt;
  st.has_loss = has_loss ? 1 : 0;
  st.loss = loss;
  for (int n = 0; n < nsteps && e == cudaSuccess; ++n) {
    Spot sp;
    L.las = inline_laser(t0 + n * dt, &sp);
    st.x_in = xstep[n % 2];
    st.x_out = xstep[(n + 1) % 2];
    st.f_in = fstep[(n + 2) % 3];
    st.f_acc = fstep[n % 3];
    st.f_clear = fstep[(n + 1) % 3];
    st.first = n == 0;
    const auto ev = timing ? timing_begin(s) : std::pair<cudaEvent_t, cudaEvent_t>{};
    e = lean >= 0 ? launch_step_lean(L, step, st, cap, lean, s) : launch_step(L, step, st, cap, pdl, s);
    ++launches;
    if (ev.first) timing_end(ev, s);
    if (e == cudaSuccess && volumetric && sp.seg >= 0) {
      e = launch_laser(degree, true, lsetup, L.mesh, power, sp, fstep[n % 3], s);
      ++launches;
    }
  }
  if (e == cudaSuccess) {
    e = launch_step_final(cap, n_dofs, xstep[nsteps % 2], fstep[(nsteps - 1) % 3],
                          nsteps >= 2 ? fstep[(nsteps - 2) % 3] : nullptr, invC0_fx, nodal, x_dir, (float)dt,
                          mat.T_ref, T_dev, s);
    ++launches;
  }
  return e;
}

pbf_status CtxBase::ensure_bfused() {
  if (cell_own) return PBF_OK;
  const size_t nv = (size_t)n_dofs * (size_t)batch;
  // owner bits: the first cell (in cell order) that has a dof as a node stores its state
  std::vector<uint32_t> own((size_t)n_cells, 0u);
  std::vector<uint8_t> seen((size_t)n_dofs, 0);
  for (size_t c = 0; c < (size_t)n_cells; ++c)
    for (int a = 0; a < npc; ++a) {
      const int32_t d = mesh->cell_dofs[c * (size_t)npc + (size_t)a];
      if (d >= 0 && !seen[(size_t)d]) {
        seen[(size_t)d] = 1;
        own[c] |= 1u << a;
      }
    }
  void* p = nullptr;
  cudaError_t e = cudaSuccess;
  auto get = [&](void** out, size_t bytes) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess) {
      allocs.push_back(p);
      *out = p;
    }
  };
  void *own_d = nullptr, *x0 = nullptr, *x1 = nullptr, *f0 = nullptr, *f1 = nullptr, *f2 = nullptr, *ld = nullptr,
       *td = nullptr;
  get(&own_d, own.size() * 4);
  get(&x0, nv * 8);
  get(&x1, nv * 8);
  get(&f0, nv * 4);
  get(&f1, nv * 4);
  get(&f2, nv * 4);
  get(&ld, sizeof(LaserK));
  get(&td, 8);
  if (e == cudaSuccess) e = cudaMemcpy(own_d, own.data(), own.size() * 4, cudaMemcpyHostToDevice);
  for (void* f : {f0, f1, f2})
    if (e == cudaSuccess) e = cudaMemset(f, 0, std::max<size_t>(nv * 4, 16));
  if (e != cudaSuccess) return cuda(e, "batched fused step set-up");
  cell_own = (uint32_t*)own_d;
  xb[0] = (float2*)x0;
  xb[1] = (float2*)x1;
  fb[0] = (float*)f0;
  fb[1] = (float*)f1;
  fb[2] = (float*)f2;
  laser_dev = (LaserK*)ld;
  t0_dev = (double*)td;
  return PBF_OK;
}

// The batched fused sequence: step n (one launch for all instances) completes step n-1 in its
// gather and accumulates f_n into fb[n % 3]; a last streaming kernel completes step N-1 and
// writes T. The laser segments and the start time are in device memory and the spot is
// computed there, so the launches of a call depend only on (nsteps, dt, T) and replay as one
// CUDA graph when those repeat (with kernel timing on they are launched one by one).
cudaError_t CtxBase::explicit_steps_bfused(double* T_dev, double t0, double dt, int nsteps, cudaStream_t s) {
  if (ensure_bfused() != PBF_OK) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMemcpyAsync(laser_dev, &lsetup.k, sizeof(LaserK), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(t0_dev, &t0, 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host copies are read before they go out of scope
  if (e != cudaSuccess) return e;
  const double xd = mat.T_dirichlet - mat.T_ref;
  const float xd_hi = (float)xd;
  CellLaunch L = base;
  L.las = inline_laser(t0, nullptr);
  if (lsetup.k.n_seg > 0) {  // constants of the surface laser; the spot is computed per step
    const double r = lsetup.k.radius;
    L.las.amp = 2.0 * lsetup.k.eta / (kPi * r * r);
    L.las.ir2 = 2.0 / (r * r);
    L.las.cut2 = 36.0 * r * r;
    L.las.power = power;
    L.las.powerf = powerf;
  }
  BStepArgs A;
  A.T0 = T_dev;
  A.off = mat.T_ref;
  A.invC0x = invC0_fx;
  A.nc = nodal;
  A.x_dir = make_float2(xd_hi, (float)(xd - (double)xd_hi));
  A.dt = (float)dt;
  A.own = cell_own;
  A.laser = lsetup.k.n_seg > 0 ? laser_dev : nullptr;
  A.t0 = t0_dev;
  A.dt64 = dt;
  auto body = [&](cudaStream_t st, bool timed) {
    cudaError_t err = cudaSuccess;
    for (int n = 0; n < nsteps && err == cudaSuccess; ++n) {
      A.step = n;
      A.first = n == 0;
      A.x_in = xb[n % 2];
      A.x_out = xb[(n + 1) % 2];
      A.f_in = fb[(n + 2) % 3];
      A.f_acc = fb[n % 3];
      A.f_clear = fb[(n + 1) % 3];
      const auto ev = timed ? timing_begin(st) : std::pair<cudaEvent_t, cudaEvent_t>{};
      err = launch_bstep(L, A, cap, st);
      ++launches;
      if (ev.first) timing_end(ev, st);
    }
    if (err == cudaSuccess)
      err = launch_bstep_final(cap, n_dofs, batch, xb[nsteps % 2], fb[(nsteps - 1) % 3],
                               nsteps >= 2 ? fb[(nsteps - 2) % 3] : nullptr, invC0_fx, nodal, A.x_dir, (float)dt,
                               mat.T_ref, T_dev, st);
    ++launches;
    return err;
  };
  if (timing) return body(s, true);
  double key[kGraphKey] = {};
  key[0] = (double)nsteps;
  key[1] = dt;
  key[2] = (double)(uintptr_t)T_dev;
  key[3] = (double)cap;
  key[4] = (double)(lsetup.k.n_seg > 0);
  key[5] = lsetup.k.eta;  // the surface laser's constants are kernel arguments
  key[6] = lsetup.k.radius;
  GraphSlot& g = bstep_graph;
  if (!g.exec || std::memcmp(key, g.key, sizeof key) != 0) {
    if (g.exec) {
      e = cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
      if (e != cudaSuccess) return e;
    }
    if (!cap_stream) {
      e = cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) return e;
    }
    const long long l0 = launches;
    e = cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t eb = body(cap_stream, false);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cap_stream, &graph);
    if (e == cudaSuccess) e = eb;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    g.launches = launches - l0;
    launches = l0;
    std::memcpy(g.key, key, sizeof key);
  }
  e = cudaGraphLaunch(g.exec, s);
  launches += g.launches;
  return e;
}

// The persistent form: one cooperative launch runs the whole sequence (grid barrier between
// steps). It synchronises to read the barrier's time-out flag.
cudaError_t CtxBase::explicit_steps_persistent(double* T_dev, double t0, double dt, int nsteps, cudaStream_t s) {
  PersistState ps;
  const double xd = mat.T_dirichlet - mat.T_ref;
  const float xd_hi = (float)xd;
  ps.st.T0 = T_dev;
  ps.st.off = mat.T_ref;
  ps.st.invC0x = invC0_fx;
  ps.st.nc = nodal;
  ps.st.x_dir = make_float2(xd_hi, (float)(xd - (double)xd_hi));
  ps.st.dt = (float)dt;
  ps.x[0] = xstep[0];
  ps.x[1] = xstep[1];
  for (int i = 0; i < 3; ++i) ps.f[i] = fstep[i];
  ps.T = T_dev;
  ps.nsteps = nsteps;
  ps.t0 = t0;
  ps.dt64 = dt;
  ps.laser = lsetup.k;
  ps.las = inline_laser(t0, nullptr);
  if (lsetup.k.n_seg > 0) {  // constants of the surface laser; the spot follows per step
    const double r = lsetup.k.radius;
    ps.las.on = 1;
    ps.las.amp = 2.0 * lsetup.k.eta / (kPi * r * r);
    ps.las.ir2 = 2.0 / (r * r);
    ps.las.cut2 = 36.0 * r * r;
    ps.las.power = power;
    ps.las.powerf = powerf;
  }
  ps.bar = bar;
  ps.extra_arrivals = barrier_test_extra;
  barrier_timed_out = false;
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s);
  const auto ev = timing && e == cudaSuccess ? timing_begin(s) : std::pair<cudaEvent_t, cudaEvent_t>{};
  if (e == cudaSuccess) e = launch_steps_persistent(base, step, ps, cap, nullptr, s);
  ++launches;
  if (ev.first) timing_end(ev, s);
  unsigned flag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, &bar->err, sizeof(flag), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && flag) {
    // the sequence stopped part-way: clear the accumulators so that the next call starts
    // from the usual all-zero state
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaMemsetAsync(fstep[i], 0, (size_t)n_dofs * 4, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
      barrier_timed_out = true;
      e = cudaErrorTimeout;
    }
  }
  return e;
}

std::pair<cudaEvent_t, cudaEvent_t> CtxBase::timing_begin(cudaStream_t s) {
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  if (free_events.empty()) {
    if (cudaEventCreate(&ev.first) != cudaSuccess || cudaEventCreate(&ev.second) != cudaSuccess) {
      if (ev.first) cudaEventDestroy(ev.first);
      cudaGetLastError();
      return {nullptr, nullptr};
    }
  } else {
    ev = free_events.back();
    free_events.pop_back();
  }
  cudaEventRecord(ev.first, s);
  return ev;
}

void CtxBase::timing_end(const std::pair<cudaEvent_t, cudaEvent_t>& ev, cudaStream_t s) {
  cudaEventRecord(ev.second, s);
  events.push_back(ev);
}

extern "C" pbf_status pbf_eval_residual(pbf_ctx* ctx, const double* T_dev, const pbf_laser* laser, double t,
                                        double* fdiff_dev, double* fvol_dev, double* C_dev, pbf_stream stream) {
  if (!ctx || !T_dev) return fail(PBF_EINVAL, "null argument");
  pbf_status st = ctx->check_usable();
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  st = ctx->set_laser(laser, s);
  if (st) return st;
  return ctx->cuda(ctx->residual_f64(T_dev, t, fdiff_dev, fvol_dev, C_dev, s), "eval_residual");
}

extern "C" pbf_status pbf_explicit_step(pbf_ctx* ctx, double* T_dev, const pbf_laser* laser, double t0, double dt,
                                        int nsteps, pbf_stream stream) {
  if (!ctx || !T_dev) return fail(PBF_EINVAL, "null argument");
  if (nsteps < 0 || !(dt > 0)) return fail(PBF_EINVAL, "need nsteps >= 0 and dt > 0");
  pbf_status st = ctx->check_usable();
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  st = ctx->set_laser(laser, s);
  if (st) return st;
  return ctx->cuda(ctx->explicit_steps(T_dev, t0, dt, nsteps, s), "explicit_step");
}

extern "C" pbf_status pbf_round_to_f32(const double* x_dev, float* y_dev, int64_t n, pbf_stream stream) {
  if ((!x_dev || !y_dev) && n > 0) return fail(PBF_EINVAL, "null argument");
  if (n < 0) return fail(PBF_EINVAL, "negative length");
  cudaError_t e = launch_round_f32(n, x_dev, y_dev, (cudaStream_t)stream);
  return e == cudaSuccess ? PBF_OK : fail(PBF_ECUDA, "round_to_f32: %s", cudaGetErrorString(e));
}

extern "C" pbf_status pbf_widen_to_f64(const float* x_dev, double* y_dev, int64_t n, pbf_stream stream) {
  if ((!x_dev || !y_dev) && n > 0) return fail(PBF_EINVAL, "null argument");
  if (n < 0) return fail(PBF_EINVAL, "negative length");
  cudaError_t e = launch_f32_to_f64(n, x_dev, y_dev, (cudaStream_t)stream);
  return e == cudaSuccess ? PBF_OK : fail(PBF_ECUDA, "widen_to_f64: %s", cudaGetErrorString(e));
}

extern "C" pbf_status pbf_ctx_autotune(pbf_ctx* ctx, const double* T_dev, int reps, int* variant_out,
                                       float* us_per_step_out, pbf_stream stream) {
  if (!ctx || !T_dev || reps < 1) return fail(PBF_EINVAL, "bad arguments");
  pbf_status st = ctx->check_usable();
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (!ctx->f32) {
    ctx->base.variant = 0;
    if (variant_out) *variant_out = 0;
    return PBF_OK;
  }
  // explicit steps with dt = 0 (the state does not change) on a scratch copy of T, with the
  // laser of the last call, for every shape; kernel timing is off meanwhile
  const int64_t nv = ctx->n_dofs * ctx->batch;
  const bool timing = ctx->timing;
  const int variant = ctx->base.variant;
  ctx->timing = false;
  double* tmp = nullptr;
  cudaError_t e = cudaMalloc(&tmp, (size_t)std::max<int64_t>(1, nv) * 8);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, T_dev, (size_t)nv * 8, cudaMemcpyDeviceToDevice, s);
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  int best = -1;
  float best_ms = 0.f;
  for (int v = 0; v < kCellVariants && e == cudaSuccess; ++v) {
    if (us_per_step_out) us_per_step_out[v] = -1.f;
    // the fused forms of one instance; for a batch shape 4 stands for its fused form
    if (v >= 4 && !ctx->fused_ok(v) && !(v == 4 && ctx->bfused_ok())) continue;
    ctx->base.variant = v;
    e = ctx->explicit_steps(tmp, 0.0, 0.0, 2, s);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(a, s);
    if (e == cudaSuccess) e = ctx->explicit_steps(tmp, 0.0, 0.0, reps, s);
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && us_per_step_out) us_per_step_out[v] = 1000.f * ms / (float)reps;
    if (e == cudaSuccess && (best < 0 || ms < best_ms)) {
      best = v;
      best_ms = ms;
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (tmp) cudaFree(tmp);
  ctx->timing = timing;
  if (e != cudaSuccess) {
    ctx->base.variant = variant;
    return ctx->cuda(e, "autotune");
  }
  ctx->base.variant = best;
  if (variant_out) *variant_out = best;
  return PBF_OK;
}

extern "C" pbf_status pbf_ctx_set_kernel_shape(pbf_ctx* ctx, int shape) {
  if (!ctx || shape < 0 || shape >= kCellVariants) return fail(PBF_EINVAL, "shape must be in [0, %d]", kCellVariants - 1);
  ctx->base.variant = shape;
  return PBF_OK;
}

extern "C" pbf_status pbf_ctx_set_surface_loss(pbf_ctx* ctx, const pbf_surface_loss* q) {
  if (!ctx) return fail(PBF_EINVAL, "null context");
  if (!q) {
    ctx->has_loss = false;
    return PBF_OK;
  }
  if (!(q->emissivity >= 0.0) || !(q->T_amb >= 0.0) || !(q->C_P >= 0.0) ||
      (q->C_P > 0.0 && !(q->T_v > 0.0 && q->T_max > q->T_v && q->C_M > 0.0)))
    return fail(PBF_EINVAL, "surface loss: need emissivity, T_amb, C_P >= 0 and, with evaporation, 0 < T_v < T_max, C_M > 0");
  LossK& k = ctx->loss;
  k.emissivity = q->emissivity;
  k.T_amb = q->T_amb;
  k.C_P = q->C_P;
  k.C_T = q->C_T;
  k.C_M = q->C_M;
  k.T_v = q->T_v;
  k.h_v = q->h_v;
  k.c_h = q->c_h;
  k.T_h0 = q->T_h0;
  k.T_max = q->T_max;
  ctx->has_loss = true;
  return PBF_OK;
}

extern "C" pbf_status pbf_ctx_set_phase(pbf_ctx* ctx, const pbf_phase* ph) {
  if (!ctx) return fail(PBF_EINVAL, "null context");
  pbf_status st = ctx->check_usable();
  if (st) return st;
  if (!ph) {
    ctx->has_phase = false;
    return PBF_OK;
  }
  if (!(ph->T_l > ph->T_s) || !(ph->k_p >= 0.0) || !(ph->k_m >= 0.0) || !(ph->k_s >= 0.0))
    return fail(PBF_EINVAL, "phase model: need T_l > T_s and non-negative conductivities");
  if (ctx->cap == CAP_QUADRATURE) return fail(PBF_EINVAL, "phase model: needs the constant or nodal capacity");
  const int nq = ctx->npc;  // (p+1)^3 quadrature points per cell, as many as nodes
  if (!ctx->rc) {
    char* p = nullptr;
    const cudaError_t e = dalloc(ctx, &p, (size_t)nq * (size_t)ctx->n_cells * (size_t)ctx->batch * (ctx->f32 ? 4 : 8));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(e == cudaErrorMemoryAllocation ? PBF_ENOMEM : PBF_ECUDA, "phase model: %s", cudaGetErrorString(e));
    }
    ctx->rc = p;
  }
  const double t_off = ctx->mat.T_ref - ph->T_s, inv = 1.0 / (ph->T_l - ph->T_s);
  ctx->phd = PhaseR<double>{t_off, inv, ph->k_p, ph->k_s - ph->k_p, ph->k_m - ph->k_s};
  ctx->phf = PhaseR<float>{(float)t_off, (float)inv, (float)ph->k_p, (float)(ph->k_s - ph->k_p), (float)(ph->k_m - ph->k_s)};
  cudaError_t e = launch_phase_init(ctx->f32, nq, ctx->base.mesh, ctx->rc, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  ++ctx->launches;
  if (e != cudaSuccess) return ctx->cuda(e, "phase model");
  ctx->has_phase = true;
  return PBF_OK;
}

// ---- history of the phase model across mesh changes --------------------------------------

extern "C" pbf_status pbf_ctx_history_cell_min(pbf_ctx* ctx, double* rc_min_host, pbf_stream stream) {
  if (!ctx || !rc_min_host) return fail(PBF_EINVAL, "null argument");
  if (!ctx->has_phase) return fail(PBF_EINVAL, "the context has no phase model");
  cudaStream_t s = (cudaStream_t)stream;
  double* tmp = nullptr;
  cudaError_t e = cudaMalloc(&tmp, std::max<size_t>(1, (size_t)ctx->n_cells) * 8);
  if (e == cudaSuccess)
    e = launch_history_min(ctx->f32, ctx->npc, (int)ctx->n_cells, ctx->batch, ctx->rc, tmp, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(rc_min_host, tmp, (size_t)ctx->n_cells * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (tmp) cudaFree(tmp);
  ++ctx->launches;
  return ctx->cuda(e, "history_cell_min");
}

extern "C" pbf_status pbf_ctx_get_history(pbf_ctx* ctx, double* rc_dev, pbf_stream stream) {
  if (!ctx || !rc_dev) return fail(PBF_EINVAL, "null argument");
  if (!ctx->has_phase) return fail(PBF_EINVAL, "the context has no phase model");
  const int64_t n = (int64_t)ctx->npc * ctx->n_cells * ctx->batch;
  ++ctx->launches;
  return ctx->cuda(launch_history_copy(ctx->f32, true, n, ctx->rc, rc_dev, (cudaStream_t)stream), "get_history");
}

extern "C" pbf_status pbf_ctx_set_history(pbf_ctx* ctx, const double* rc_dev, pbf_stream stream) {
  if (!ctx || !rc_dev) return fail(PBF_EINVAL, "null argument");
  pbf_status st = ctx->check_usable();
  if (st) return st;
  if (!ctx->has_phase) return fail(PBF_EINVAL, "the context has no phase model");
  const int64_t n = (int64_t)ctx->npc * ctx->n_cells * ctx->batch;
  ++ctx->launches;
  return ctx->cuda(launch_history_copy(ctx->f32, false, n, rc_dev, ctx->rc, (cudaStream_t)stream), "set_history");
}

extern "C" pbf_status pbf_ctx_transfer_history(pbf_ctx* from, pbf_ctx* to, pbf_stream stream) {
  if (!from || !to) return fail(PBF_EINVAL, "null argument");
  pbf_status st = to->check_usable();
  if (st) return st;
  if (!from->has_phase || !to->has_phase) return fail(PBF_EINVAL, "both contexts need the phase model");
  const HostMesh& m = *to->mesh;
  if (from->mesh != to->mesh || from->generation + 1 != to->generation || m.history_old_cells != from->n_cells ||
      m.history_map.size() != (size_t)to->n_cells * (size_t)to->npc)
    return fail(PBF_ESTATE, "`from` must be a context of the same mesh before its last change");
  if (from->batch != to->batch || from->f32 != to->f32 || from->npc != to->npc)
    return fail(PBF_EINVAL, "the contexts differ in batch, precision or degree");
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* map = nullptr;
  cudaError_t e = cudaMalloc(&map, std::max<size_t>(1, m.history_map.size()) * 4);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(map, m.history_map.data(), m.history_map.size() * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = launch_history_gather(to->f32, to->npc, (int)to->n_cells, (int)from->n_cells, to->batch, map, from->rc, to->rc,
                              s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (map) cudaFree(map);
  ++to->launches;
  return to->cuda(e, "transfer_history");
}

extern "C" pbf_status pbf_ctx_set_barrier_test(pbf_ctx* ctx, int extra_blocks) {
  if (!ctx || extra_blocks < 0) return fail(PBF_EINVAL, "bad arguments");
  ctx->barrier_test_extra = (unsigned)extra_blocks;
  return PBF_OK;
}

extern "C" pbf_status pbf_ctx_set_timing(pbf_ctx* ctx, int enable) {
  if (!ctx) return fail(PBF_EINVAL, "null argument");
  ctx->timing = enable != 0;
  return PBF_OK;
}

extern "C" pbf_status pbf_ctx_kernel_time(pbf_ctx* ctx, double* ms_out, long long* launches_out) {
  if (!ctx) return fail(PBF_EINVAL, "null argument");
  double total = 0.0;
  for (auto& ev : ctx->events) {
    cudaError_t e = cudaEventSynchronize(ev.second);
    if (e != cudaSuccess) return ctx->cuda(e, "kernel_time");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev.first, ev.second);
    total += ms;
    ctx->free_events.push_back(ev);
  }
  if (ms_out) *ms_out = total;
  if (launches_out) *launches_out = (long long)ctx->events.size();
  ctx->events.clear();
  return PBF_OK;
}

extern "C" pbf_status pbf_ctx_launch_count(pbf_ctx* ctx, long long* launches_out) {
  if (!ctx || !launches_out) return fail(PBF_EINVAL, "null argument");
  *launches_out = ctx->launches;
  return PBF_OK;
}

// ---- critical time step (Eq. explicit_time_step) -----------------------------------------

namespace {
// SplitMix64 (Steele, Lea, Flood 2014; public-domain reference by Vigna): deterministic
// start vectors when the caller passes none.
void splitmix_fill(std::vector<double>& v, uint64_t seed) {
  uint64_t x = seed;
  for (double& o : v) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    o = (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  }
}
}  // namespace

pbf_status CtxBase::ensure_vectors(int n) {
  while ((int)vec.size() < n) {
    double* p = nullptr;
    cudaError_t e = dalloc_raw(&p, (size_t)n_dofs * (size_t)batch);
    if (e != cudaSuccess) return cuda(e, "work vector allocation");
    vec.push_back(p);
  }
  return PBF_OK;
}

cudaError_t CtxBase::dalloc_raw(double** p, size_t n) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(1, n) * 8);
  if (e == cudaSuccess) {
    allocs.push_back(q);
    *p = (double*)q;
  }
  return e;
}

extern "C" pbf_status pbf_estimate_dt(pbf_ctx* ctx, const double* x0_dev, int max_iter, double rtol,
                                      double* lambda_out, double* dt_crit_out, int* iters_out, pbf_stream stream) {
  if (!ctx) return fail(PBF_EINVAL, "null argument");
  if (max_iter < 1) return fail(PBF_EINVAL, "max_iter must be positive");
  pbf_status st = ctx->check_usable();
  if (st) return st;
  st = ctx->ensure_vectors(2);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = ctx->n_dofs;
  double *x = ctx->vec[0], *y = ctx->vec[1];
  cudaError_t e;
  if (x0_dev) {
    e = cudaMemcpyAsync(x, x0_dev, (size_t)n * 8, cudaMemcpyDeviceToDevice, s);
  } else {
    std::vector<double> h((size_t)n);
    splitmix_fill(h, 0x5eedull);
    e = cudaMemcpyAsync(x, h.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e == cudaSuccess) e = launch_zero_masked(n, x, ctx->dirichlet, s);
  // linear stiffness in FP64 for instance 0 (k frozen at k0, scale s of instance 0)
  CellLaunch L = ctx->base;
  L.f32 = 0;
  L.nonlin_k = 0;
  L.latent = 0;
  L.offset = 0.0;
  L.mesh.batch = 1;
  L.k_scale_d = ctx->k_scale_d;
  double lambda = 0.0;
  int it = 0;
  double* d_scal = ctx->scal;
  for (; it < max_iter && e == cudaSuccess; ++it) {
    // normalise x in the C~ norm
    e = launch_dot(n, 1, x, x, ctx->C0, nullptr, ctx->part, d_scal, s);
    double nx2 = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nx2, d_scal, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) break;
    if (!(nx2 > 0)) return fail(PBF_EINVAL, "start vector vanishes on the free dofs");
    double inv = 1.0 / std::sqrt(nx2);
    e = cudaMemcpyAsync(d_scal + 1, &inv, 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_scale_masked(n, x, d_scal + 1, nullptr, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(y, 0, (size_t)n * 8, s);
    L.x = x;
    if (e == cudaSuccess) e = ctx->apply_cell(L, y, nullptr, MODE_STIFF, s);
    if (e == cudaSuccess) e = launch_zero_masked(n, y, ctx->dirichlet, s);
    if (e == cudaSuccess) e = launch_dot(n, 1, x, y, nullptr, nullptr, ctx->part, d_scal + 2, s);
    double lam = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&lam, d_scal + 2, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = launch_div_masked(n, x, y, ctx->invC0_d, ctx->dirichlet, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    ctx->launches += 9;
    if (e != cudaSuccess) break;
    bool done = it > 0 && std::fabs(lam - lambda) <= rtol * std::fabs(lam);
    lambda = lam;
    if (done) {
      ++it;
      break;
    }
  }
  if (e != cudaSuccess) return ctx->cuda(e, "estimate_dt");
  if (lambda_out) *lambda_out = lambda;
  if (dt_crit_out) *dt_crit_out = lambda > 0 ? 2.0 / lambda : INFINITY;
  if (iters_out) *iters_out = it;
  return PBF_OK;
}
