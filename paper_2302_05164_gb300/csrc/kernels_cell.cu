// Cell-operator kernels: the matrix-free, sum-factorised evaluation of the heat operator
// (paper Sec. 4.2, Eqs. diffusive_term_evaluation, vector_evaluation, matrix_free_eval).
//
// GPU mapping: one thread per (cell, instance); consecutive threads are consecutive
// instances of a cell, then consecutive cells in Z-curve order, so gathers of a batch are
// coalesced and neighbouring cells share cache lines (the analogue of the paper's
// vectorisation over cell batches, Sec. 4.2.1). Per thread the 1D interpolation and
// gradient contractions run fully unrolled in registers with compile-time coefficients;
// the quadrature-point physics is branch-free (clamps and selects, Sec. 4.2.1 masks);
// values are scattered with atomics onto dofs and, through the constraint rows, onto the
// masters of hanging nodes (G_e^T P^T).
#include <cstdio>
#include <type_traits>

#include "cell_ops.cuh"

namespace pbf {
namespace {

// Gather T_e = P G_e x. Slot a of a cell holds a dof d >= 0 or a hanging node -1-r; hanging
// values were computed beforehand (x_h = P_h x, one small kernel), so every slot is one load
// from one of two arrays, selected without branching: all loads of a cell issue back to back.
template <int P, typename R, typename S>
__device__ __forceinline__ void gather_sel(const DevMesh& M, const S* __restrict__ x, const S* __restrict__ xh,
                                           int cell, int inst, double off, R* u) {
  constexpr int NP = (P + 1) * (P + 1) * (P + 1);
  const int B = M.batch;
  int idx[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) idx[a] = __ldg(&M.cell_dofs[a * M.n_cells + cell]);
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    const int d = idx[a];
    const S* base = d >= 0 ? x : xh;
    const int j = d >= 0 ? d : -1 - d;
    const S v = __ldg(&base[j * B + inst]);
    if (sizeof(S) == 8) u[a] = R((double)v - off);
    else u[a] = R(v);
  }
}

template <int P, typename R>
__device__ __forceinline__ void gather_any(const CellLaunch& L, int cell, int inst, R* u);
template <>
__device__ __forceinline__ void gather_any<1, float>(const CellLaunch& L, int cell, int inst, float* u) {
  gather_sel<1, float, float>(L.mesh, L.xf, L.xfh, cell, inst, 0.0, u);
}
template <>
__device__ __forceinline__ void gather_any<2, float>(const CellLaunch& L, int cell, int inst, float* u) {
  gather_sel<2, float, float>(L.mesh, L.xf, L.xfh, cell, inst, 0.0, u);
}
template <>
__device__ __forceinline__ void gather_any<1, double>(const CellLaunch& L, int cell, int inst, double* u) {
  gather_sel<1, double, double>(L.mesh, L.x, L.xh, cell, inst, L.offset, u);
}
template <>
__device__ __forceinline__ void gather_any<2, double>(const CellLaunch& L, int cell, int inst, double* u) {
  gather_sel<2, double, double>(L.mesh, L.x, L.xh, cell, inst, L.offset, u);
}

// f += G_e^T fe, with hanging-node slots going to fh (distributed by P_h^T afterwards)
template <int P, typename R>
__device__ __forceinline__ void scatter(const DevMesh& M, R* __restrict__ f, R* __restrict__ fh, int cell, int inst,
                                        const R* fe) {
  constexpr int NP = (P + 1) * (P + 1) * (P + 1);
  const int B = M.batch;
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    const int d = __ldg(&M.cell_dofs[a * M.n_cells + cell]);
    R* base = d >= 0 ? f : fh;
    const int j = d >= 0 ? d : -1 - d;
    atomicAdd(&base[j * B + inst], fe[a]);
  }
}

// One kernel for the residual / capacity / stiffness / implicit-operator modes.
template <typename R>
__device__ __forceinline__ const PhaseR<R>& phase_of(const CellLaunch& L);
template <>
__device__ __forceinline__ const PhaseR<float>& phase_of<float>(const CellLaunch& L) { return L.phf; }
template <>
__device__ __forceinline__ const PhaseR<double>& phase_of<double>(const CellLaunch& L) { return L.phd; }

// PH: conductivity from the phase model with history (residual mode) instead of the k(T) ramp.
template <int P, typename R, int MODE, bool NLK, bool LAT, int BS = 128, int MINB = 1, bool PH = false>
__global__ void __launch_bounds__(BS, MINB) k_cell(const CellLaunch L, R* __restrict__ f, R* __restrict__ fh,
                                                   R* __restrict__ C, R* __restrict__ Ch) {
  constexpr int N = P + 1, NP = N * N * N;
  (void)N;
  const DevMesh& M = L.mesh;
  const MatR<R>& mt = mat_of<R>(L);
  const GeoR<R>& geo = geo_of<R>(L);
  const int B = M.batch;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= M.n_cells * B) return;
  const int cell = B == 1 ? tid : tid / B, inst = tid - cell * B;

  R u[NP], v[NP];
  gather_any<P, R>(L, cell, inst, u);
  values_at_qp<P, R>(u, v);

  const int lev = M.cell_level[cell];
  const R detJ = geo.detJ[lev];

  if ((MODE == MODE_RESIDUAL || MODE == MODE_CAPACITY) && C != nullptr) {
    // lumped capacity: int rho c_app(T_h) N_i  (row sums of the consistent capacity)
    R cw[NP], ce[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      R cap = mt.c;
      if (LAT) {
        const R z = (v[q] + mt.tm_off) * mt.inv_sigma;
        cap = mt.c + mt.lat_norm * expo(R(-0.5) * z * z);
      }
      cw[q] = mt.rho * cap * (R(wq3<P>(q)) * detJ);
    }
    integrate_values<P, R>(cw, ce);
    scatter<P, R>(M, C, Ch, cell, inst, ce);
  }
  if (MODE == MODE_CAPACITY) return;

  // conductivity at quadrature points times quadrature weight and det J: the D_e of
  // Eq. diffusive_term_evaluation for a diagonal Jacobian
  const int mat = M.cell_mat[cell];
  const R* ks = kscale_of<R>(L);
  const R scale = (mat == 1 ? mt.powder_scale : R(1)) * (ks ? ks[inst] : R(1));
  const R sgn = (MODE == MODE_RESIDUAL) ? R(-1) : R(1);
  R kw[NP];
  if (PH) {
    // k(T, r_c) with r_c = max(stored r_c, g(T)) per quadrature point; stored in explicit steps
    const PhaseR<R>& ph = phase_of<R>(L);
    const R is = ks ? ks[inst] : R(1);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const R g = clamp01((v[q] + ph.t_off) * ph.inv_dT);
      const int64_t j = ((int64_t)q * M.n_cells + cell) * B + inst;
      R rc = rc_load<R>(L, j);
      rc = rc > g ? rc : g;
      if (L.rc_out) rc_store<R>(L, j, rc);
      kw[q] = sgn * ((ph.kp + rc * ph.dks + g * ph.dkm) * is) * (R(wq3<P>(q)) * detJ);
    }
  } else {
    const R k0 = mt.k0 * scale, dk = mt.dk * scale;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      R k = k0;
      if (NLK) k = k0 + dk * clamp01((v[q] + mt.tk_off) * mt.inv_dT);
      kw[q] = sgn * k * (R(wq3<P>(q)) * detJ);
    }
  }
  R r[NP], g[NP];
  {
    const R cd = geo.ih2[lev][0];
    apply1d<P, 1, 0, false, false>(v, g);
#pragma unroll
    for (int q = 0; q < NP; ++q) g[q] *= kw[q] * cd;
    apply1d<P, 1, 0, true, false>(g, r);
  }
  {
    const R cd = geo.ih2[lev][1];
    apply1d<P, 1, 1, false, false>(v, g);
#pragma unroll
    for (int q = 0; q < NP; ++q) g[q] *= kw[q] * cd;
    apply1d<P, 1, 1, true, true>(g, r);
  }
  {
    const R cd = geo.ih2[lev][2];
    apply1d<P, 1, 2, false, false>(v, g);
#pragma unroll
    for (int q = 0; q < NP; ++q) g[q] *= kw[q] * cd;
    apply1d<P, 1, 2, true, true>(g, r);
  }
  if (MODE == MODE_IMPLICIT) {
#pragma unroll
    for (int q = 0; q < NP; ++q) r[q] += mt.m_impl * (R(wq3<P>(q)) * detJ) * v[q];
  }
  R fe[NP];
  integrate_values<P, R>(r, fe);
  if (MODE == MODE_RESIDUAL && L.las.on && M.cell_top[cell]) add_laser<P, R>(L, L.las, cell, inst, lev, fe);
  scatter<P, R>(M, f, fh, cell, inst, fe);
}

// Diagonal of P^T A_e P for the implicit operator A = C/dt + K (FP64, setup): the cell
// matrix column A_e e_b is computed matrix-free for every local node b, the way the paper
// remarks that a matrix can be assembled from products with unit vectors (Sec. 4.2).
template <int P>
__global__ void __launch_bounds__(64) k_diag(const CellLaunch L, double* __restrict__ diag) {
  constexpr int NP = (P + 1) * (P + 1) * (P + 1);
  const DevMesh& M = L.mesh;
  const MatR<double>& mt = L.md;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= M.n_cells) return;
  const int lev = M.cell_level[cell];
  const double detJ = L.gd.detJ[lev];
  const int mat = M.cell_mat[cell];
  const double k = mt.k0 * (mat == 1 ? mt.powder_scale : 1.0) * (L.k_scale_d ? L.k_scale_d[0] : 1.0);
  for (int b = 0; b < NP; ++b) {
    double u[NP], v[NP], r[NP], g[NP], col[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) u[a] = (a == b) ? 1.0 : 0.0;
    values_at_qp<P, double>(u, v);
#pragma unroll
    for (int a = 0; a < NP; ++a) r[a] = 0.0;
    apply1d<P, 1, 0, false, false>(v, g);
#pragma unroll
    for (int q = 0; q < NP; ++q) g[q] *= k * wq3<P>(q) * detJ * L.gd.ih2[lev][0];
    apply1d<P, 1, 0, true, true>(g, r);
    apply1d<P, 1, 1, false, false>(v, g);
#pragma unroll
    for (int q = 0; q < NP; ++q) g[q] *= k * wq3<P>(q) * detJ * L.gd.ih2[lev][1];
    apply1d<P, 1, 1, true, true>(g, r);
    apply1d<P, 1, 2, false, false>(v, g);
#pragma unroll
    for (int q = 0; q < NP; ++q) g[q] *= k * wq3<P>(q) * detJ * L.gd.ih2[lev][2];
    apply1d<P, 1, 2, true, true>(g, r);
#pragma unroll
    for (int q = 0; q < NP; ++q) r[q] += mt.m_impl * wq3<P>(q) * detJ * v[q];
    integrate_values<P, double>(r, col);
    const int db = M.cell_dofs[b * M.n_cells + cell];
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      const int da = M.cell_dofs[a * M.n_cells + cell];
      if (da >= 0 && db >= 0) {
        if (a == b) atomicAdd(&diag[da], col[a]);
        continue;
      }
      // a hanging node is involved: sum over common masters m of w_am w_bm A_ab
      const int ra0 = da >= 0 ? 0 : M.con_ptr[-1 - da], ra1 = da >= 0 ? 1 : M.con_ptr[-da];
      const int rb0 = db >= 0 ? 0 : M.con_ptr[-1 - db], rb1 = db >= 0 ? 1 : M.con_ptr[-db];
      for (int ea = ra0; ea < ra1; ++ea) {
        const int ma = da >= 0 ? da : M.con_idx[ea];
        const double wa = da >= 0 ? 1.0 : M.con_w[ea];
        for (int eb = rb0; eb < rb1; ++eb) {
          const int mb = db >= 0 ? db : M.con_idx[eb];
          if (mb != ma) continue;
          const double wb = db >= 0 ? 1.0 : M.con_w[eb];
          atomicAdd(&diag[ma], wa * wb * col[a]);
        }
      }
    }
  }
}

// Adjoint of the explicit residual: for the state T and the vectors v, mu it accumulates
//   g_j = sum_e [ -int k(T_h) grad v_h . grad N_j - int k'(T_h) N_j grad v_h . grad T_h
//                 - int rho c_app'(T_h) mu_h N_j ]
// i.e. the transpose of the linearised operator of Eq. matrix_free_eval (the D_e and L_e
// parts) plus, for the quadrature-point capacity, the transposed capacity derivative. PH: the
// phase model's k(T, r) with the history r = max(r_{n-1}, g(T)) as a state of the stepper; the
// kernel also updates the history's adjoint L.sig and adds its path into g through g'(T).
template <int P, typename R, bool NLK, bool QPC, bool PH>
__global__ void __launch_bounds__(128) k_adjoint(const CellLaunch L, R* __restrict__ g, R* __restrict__ gh) {
  static_assert(!(PH && (NLK || QPC)), "the phase model replaces the conductivity ramp; no quadrature capacity");
  constexpr int NP = (P + 1) * (P + 1) * (P + 1);
  const DevMesh& M = L.mesh;
  const MatR<R>& mt = mat_of<R>(L);
  const GeoR<R>& geo = geo_of<R>(L);
  const int B = M.batch;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= M.n_cells * B) return;
  const int cell = B == 1 ? tid : tid / B, inst = tid - cell * B;
  R u[NP], Tq[NP], vq[NP];
  gather_any<P, R>(L, cell, inst, u);
  values_at_qp<P, R>(u, Tq);
  if (sizeof(R) == 4) gather_sel<P, R, float>(M, L.vf, L.vfh, cell, inst, 0.0, u);
  else gather_sel<P, R, double>(M, L.v, L.vh, cell, inst, 0.0, u);
  values_at_qp<P, R>(u, vq);
  const int lev = M.cell_level[cell];
  const R detJ = geo.detJ[lev];
  const int mat = M.cell_mat[cell];
  const R* ks = kscale_of<R>(L);
  const R scale = (mat == 1 ? mt.powder_scale : R(1)) * (ks ? ks[inst] : R(1));
  R kw[NP], val[NP];
  if (PH) {
    // k(T, r) with r = max(r_{n-1}, g(T)), r_{n-1} the history entering the step; val holds
    // -dk/dT W at fixed r: (k_m - k_s) g'(T)
    const PhaseR<R>& ph = phase_of<R>(L);
    const R is = ks ? ks[inst] : R(1);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const R W = R(wq3<P>(q)) * detJ;
      const R z = (Tq[q] + ph.t_off) * ph.inv_dT;
      const R gz = clamp01(z);
      const R st = rc_load<R>(L, ((int64_t)q * M.n_cells + cell) * B + inst);
      const R rc = st > gz ? st : gz;
      kw[q] = -((ph.kp + rc * ph.dks + gz * ph.dkm) * is) * W;
      val[q] = (z > R(0) && z < R(1)) ? -(ph.dkm * is * ph.inv_dT) * W : R(0);
    }
  } else {
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const R W = R(wq3<P>(q)) * detJ;
      const R sx = (Tq[q] + mt.tk_off) * mt.inv_dT;
      R k = mt.k0 * scale;
      if (NLK) k = k + mt.dk * scale * clamp01(sx);
      kw[q] = -k * W;
      // k'(T): slope inside the open ramp, zero outside (and at its ends)
      val[q] = (NLK && sx > R(0) && sx < R(1)) ? -(mt.dk * scale * mt.inv_dT) * W : R(0);
    }
  }
  if (QPC) {
    if (sizeof(R) == 4) gather_sel<P, R, float>(M, L.muf, L.mufh, cell, inst, 0.0, u);
    else gather_sel<P, R, double>(M, L.mu, L.muh, cell, inst, 0.0, u);
    R mq[NP];
    values_at_qp<P, R>(u, mq);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const R z = (Tq[q] + mt.tm_off) * mt.inv_sigma;
      const R dc = -z * mt.inv_sigma * mt.lat_norm * expo(R(-0.5) * z * z);  // c_app'(T)
      mq[q] = -mt.rho * dc * mq[q] * (R(wq3<P>(q)) * detJ);
    }
    // val holds -k'(T) W; the k' term needs grad v . grad T, added below
#pragma unroll
    for (int q = 0; q < NP; ++q) u[q] = mq[q];
  } else {
#pragma unroll
    for (int q = 0; q < NP; ++q) u[q] = R(0);
  }
  R r[NP], gv[NP], gT[NP], gg[NP];  // gg (phase model): grad v . grad T per quadrature point
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    r[q] = R(0);
    gg[q] = R(0);
  }
#define ADJ_DIR(DIR)                                                         \
  {                                                                          \
    const R cd = geo.ih2[lev][DIR];                                          \
    apply1d<P, 1, DIR, false, false>(vq, gv);                                \
    if (NLK || PH) apply1d<P, 1, DIR, false, false>(Tq, gT);                 \
    _Pragma("unroll") for (int q = 0; q < NP; ++q) {                         \
      if (NLK) u[q] += val[q] * cd * gv[q] * gT[q];                          \
      if (PH) gg[q] += cd * gv[q] * gT[q];                                   \
      gv[q] *= kw[q] * cd;                                                   \
    }                                                                        \
    apply1d<P, 1, DIR, true, true>(gv, r);                                   \
  }
  ADJ_DIR(0)
  ADJ_DIR(1)
  ADJ_DIR(2)
#undef ADJ_DIR
  if (PH) {
    // the history's adjoint (divided by dt): sig_n = -W (k_s - k_p) s grad v . grad T + sig_in;
    // where the max takes g (b) it reaches lambda through g'(T) and is not carried further back,
    // else it is carried unchanged (r_n = r_{n-1})
    const PhaseR<R>& ph = phase_of<R>(L);
    const R is = ks ? ks[inst] : R(1);
    R* sig = static_cast<R*>(L.sig);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const R W = R(wq3<P>(q)) * detJ;
      const int64_t j = ((int64_t)q * M.n_cells + cell) * B + inst;
      const R z = (Tq[q] + ph.t_off) * ph.inv_dT;
      const R gz = clamp01(z);
      const bool b = gz > rc_load<R>(L, j);
      const R sg = -W * ph.dks * is * gg[q] + sig[j];
      sig[j] = b ? R(0) : sg;
      u[q] += val[q] * gg[q] + ((b && z < R(1)) ? ph.inv_dT * sg : R(0));
    }
  }
#pragma unroll
  for (int q = 0; q < NP; ++q) r[q] += u[q];
  R fe[NP];
  integrate_values<P, R>(r, fe);
  scatter<P, R>(M, g, gh, cell, inst, fe);
}

template <int P, typename R, bool NLK, bool QPC, bool PH = false>
cudaError_t go_adj(const CellLaunch& L, void* g, void* gh, cudaStream_t s) {
  const int64_t n = (int64_t)L.mesh.n_cells * L.mesh.batch;
  if (n == 0) return cudaSuccess;
  k_adjoint<P, R, NLK, QPC, PH><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(L, (R*)g, (R*)gh);
  return cudaGetLastError();
}

template <int P, typename R>
cudaError_t dispatch_adj(const CellLaunch& L, bool qpc, void* g, void* gh, cudaStream_t s) {
  const bool nl = L.nonlin_k != 0;
  if (L.phase) {  // the phase model: its history and the history's adjoint are needed
    if (qpc || !L.rc_in || !L.sig) return cudaErrorInvalidValue;
    return go_adj<P, R, false, false, true>(L, g, gh, s);
  }
  if (nl && qpc) return go_adj<P, R, true, true>(L, g, gh, s);
  if (nl) return go_adj<P, R, true, false>(L, g, gh, s);
  if (qpc) return go_adj<P, R, false, true>(L, g, gh, s);
  return go_adj<P, R, false, false>(L, g, gh, s);
}

template <int P, typename R, int MODE, bool NLK, bool LAT, int BS = 128, int MINB = 1, bool PH = false>
cudaError_t go_shape(const CellLaunch& L, void* f, void* fh, void* C, void* Ch, cudaStream_t s) {
  const int64_t n = (int64_t)L.mesh.n_cells * L.mesh.batch;
  if (n == 0) return cudaSuccess;
  const int64_t grid = (n + BS - 1) / BS;
  k_cell<P, R, MODE, NLK, LAT, BS, MINB, PH><<<(unsigned)grid, BS, 0, s>>>(L, (R*)f, (R*)fh, (R*)C, (R*)Ch);
  return cudaGetLastError();
}

// The FP32 residual kernel without quadrature-point capacity comes in the autotuner's launch
// shapes; every other combination uses 128 threads with no register cap.
template <int P, typename R, int MODE, bool NLK, bool LAT>
cudaError_t go(const CellLaunch& L, void* f, void* fh, void* C, void* Ch, cudaStream_t s) {
  if (MODE == MODE_RESIDUAL && !LAT && L.phase)  // phase model: one launch shape
    return go_shape<P, R, MODE, false, false, 128, 1, true>(L, f, fh, C, Ch, s);
  if (std::is_same<R, float>::value && MODE == MODE_RESIDUAL && !LAT) {
    switch (L.variant) {
      case 0: return go_shape<P, R, MODE, NLK, LAT>(L, f, fh, C, Ch, s);
      case 2: return go_shape<P, R, MODE, NLK, LAT, 128, 6>(L, f, fh, C, Ch, s);
      case 3: return go_shape<P, R, MODE, NLK, LAT, 64, 10>(L, f, fh, C, Ch, s);
      default:  // 1, and 4-9 (forms of the fused explicit step: residual-only launches use shape 1)
        return go_shape<P, R, MODE, NLK, LAT, 128, 5>(L, f, fh, C, Ch, s);
    }
  }
  return go_shape<P, R, MODE, NLK, LAT>(L, f, fh, C, Ch, s);
}

template <int P, typename R>
cudaError_t dispatch(const CellLaunch& L, void* f, void* fh, void* C, void* Ch, int mode, cudaStream_t s) {
  const bool nl = L.nonlin_k != 0, lat = L.latent != 0;
  switch (mode) {
    case MODE_RESIDUAL:
      if (nl && lat) return go<P, R, MODE_RESIDUAL, true, true>(L, f, fh, C, Ch, s);
      if (nl) return go<P, R, MODE_RESIDUAL, true, false>(L, f, fh, C, Ch, s);
      if (lat) return go<P, R, MODE_RESIDUAL, false, true>(L, f, fh, C, Ch, s);
      return go<P, R, MODE_RESIDUAL, false, false>(L, f, fh, C, Ch, s);
    case MODE_CAPACITY:
      if (lat) return go<P, R, MODE_CAPACITY, false, true>(L, f, fh, C, Ch, s);
      return go<P, R, MODE_CAPACITY, false, false>(L, f, fh, C, Ch, s);
    case MODE_STIFF:
      return go<P, R, MODE_STIFF, false, false>(L, f, fh, C, Ch, s);
    case MODE_IMPLICIT:
      return go<P, R, MODE_IMPLICIT, false, false>(L, f, fh, C, Ch, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_cell(const CellLaunch& L, void* f, void* fh, void* C, void* Ch, int mode, cudaStream_t s) {
  // a mesh with hanging nodes needs their values and accumulators: refuse instead of faulting
  if (L.mesh.n_hang > 0 &&
      ((L.f32 ? (const void*)L.xfh : (const void*)L.xh) == nullptr || fh == nullptr || (C != nullptr && Ch == nullptr)))
    return cudaErrorInvalidValue;
  if (L.degree == 1)
    return L.f32 ? dispatch<1, float>(L, f, fh, C, Ch, mode, s) : dispatch<1, double>(L, f, fh, C, Ch, mode, s);
  if (L.degree == 2)
    return L.f32 ? dispatch<2, float>(L, f, fh, C, Ch, mode, s) : dispatch<2, double>(L, f, fh, C, Ch, mode, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_adjoint(const CellLaunch& L, bool qp_capacity, void* g, void* gh, cudaStream_t s) {
  if (L.mesh.n_hang > 0 && (L.f32 ? (!L.xfh || !L.vfh || (qp_capacity && !L.mufh))
                                  : (!L.xh || !L.vh || (qp_capacity && !L.muh)) || !gh))
    return cudaErrorInvalidValue;
  if (L.degree == 1)
    return L.f32 ? dispatch_adj<1, float>(L, qp_capacity, g, gh, s) : dispatch_adj<1, double>(L, qp_capacity, g, gh, s);
  if (L.degree == 2)
    return L.f32 ? dispatch_adj<2, float>(L, qp_capacity, g, gh, s) : dispatch_adj<2, double>(L, qp_capacity, g, gh, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_diag(const CellLaunch& L, double* diag, cudaStream_t s) {
  const int n = L.mesh.n_cells;
  if (n == 0) return cudaSuccess;
  const int bs = 64;
  if (L.degree == 1) k_diag<1><<<(n + bs - 1) / bs, bs, 0, s>>>(L, diag);
  else k_diag<2><<<(n + bs - 1) / bs, bs, 0, s>>>(L, diag);
  return cudaGetLastError();
}

}  // namespace pbf
