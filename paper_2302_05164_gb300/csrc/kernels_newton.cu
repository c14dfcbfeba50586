// Cell kernels of the nonlinear backward Euler step (paper Sec. 3.2, Eq. backward_euler_nonlinear)
// and its Newton-Raphson iteration (Eqs. Newton_1, Newton_2):
//   residual  r_i = int (rho c/dt) (T - T_n) N_i + int k(T) grad N_i . grad T           (RES)
//   Jacobian  (J w)_i = int (rho c/dt) w N_i + int (k(T) grad w + k'(T) w grad T) . grad N_i (JAC)
// the second with the k'(T) term L_e of the linearised operator, Eq. matrix_free_eval. The
// capacity is the consistent one with the plain c. One thread per cell; both fields are
// gathered with the hanging-node constraints resolved on the fly from the constraint rows,
// interpolated to the Gauss points by sum factorisation (cell_ops.cuh), and the cell vector is
// added with atomics to the dofs and, through the constraint rows, to the masters of hanging
// nodes. R is the arithmetic precision (FP32 operator or FP64); the accumulation is FP64.
#include <algorithm>

#include "cell_ops.cuh"
#include "newton.cuh"

namespace pbf {
namespace {

template <typename R>
__device__ __forceinline__ const PhaseR<R>& phase_of(const CellLaunch& L);
template <>
__device__ __forceinline__ const PhaseR<float>& phase_of<float>(const CellLaunch& L) { return L.phf; }
template <>
__device__ __forceinline__ const PhaseR<double>& phase_of<double>(const CellLaunch& L) { return L.phd; }

// The stored consolidated fraction of quadrature point q of a cell ([q][n_cells], batch 1), in
// the context's element type (the residual pass runs in FP64 in an FP32 context too).
__device__ __forceinline__ double stored_rc(const CellLaunch& L, int q, int cell) {
  return rc_load<double>(L, (int64_t)q * L.mesh.n_cells + cell);
}

// PH: the phase model's k(T, r_c) with r_c = max(stored, g(T)) and its branch-wise k'(T)
// instead of the material ramp (Eq. material_parameter_interp); with L.rc_out set, the
// residual pass also stores r_c = max(stored, g(T)) (the history of the converged state).
template <int P, typename R, bool JAC, bool NLK, bool PH>
__global__ void __launch_bounds__(128) k_newton(const CellLaunch L, const double* __restrict__ T,
                                                const double* __restrict__ w, double* __restrict__ y) {
  constexpr int N = P + 1, NP = N * N * N;
  (void)N;
  const DevMesh& M = L.mesh;
  const MatR<R>& mt = mat_of<R>(L);
  const GeoR<R>& geo = geo_of<R>(L);
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= M.n_cells) return;
  R vT[NP], vw[NP];
  {
    R uT[NP], uw[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      const int d = __ldg(&M.cell_dofs[a * M.n_cells + cell]);
      double t, x;
      if (d >= 0) {
        t = __ldg(&T[d]);
        x = __ldg(&w[d]);
      } else {
        t = 0.0;
        x = 0.0;
        const int row = -1 - d;
        for (int e = __ldg(&M.con_ptr[row]); e < __ldg(&M.con_ptr[row + 1]); ++e) {
          const int m = __ldg(&M.con_idx[e]);
          const double c = __ldg(&M.con_w[e]);
          t += c * __ldg(&T[m]);
          x += c * __ldg(&w[m]);
        }
      }
      uT[a] = R(t - L.offset);
      uw[a] = R(x);
    }
    values_at_qp<P, R>(uT, vT);
    values_at_qp<P, R>(uw, vw);
  }
  const int lev = M.cell_level[cell];
  const R detJ = geo.detJ[lev];
  const R ks = kscale_of<R>(L) ? kscale_of<R>(L)[0] : R(1);
  const R scale = PH ? ks : (M.cell_mat[cell] == 1 ? mt.powder_scale : R(1)) * ks;
  if (PH && !JAC && L.rc_out) {  // store the history of this state
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const PhaseR<R>& ph = phase_of<R>(L);
      const R gq = clamp01((vT[q] + ph.t_off) * ph.inv_dT);
      const int64_t j = (int64_t)q * M.n_cells + cell;
      const double st = rc_load<double>(L, j);
      if ((double)gq > st) rc_store<double>(L, j, (double)gq);
    }
  }
  R r[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) r[q] = mt.m_impl * vw[q] * (R(wq3<P>(q)) * detJ);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    R gT[NP], g[NP];
    const R cd = geo.ih2[lev][d] * detJ;
    if (d == 0) {
      apply1d<P, 1, 0, false, false>(vT, gT);
      if (JAC) apply1d<P, 1, 0, false, false>(vw, g);
    } else if (d == 1) {
      apply1d<P, 1, 1, false, false>(vT, gT);
      if (JAC) apply1d<P, 1, 1, false, false>(vw, g);
    } else {
      apply1d<P, 1, 2, false, false>(vT, gT);
      if (JAC) apply1d<P, 1, 2, false, false>(vw, g);
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      R k = mt.k0, kd = R(0);
      if (PH) {  // scale: the instance's conductivity scale only (the powder factor is not used)
        const PhaseR<R>& ph = phase_of<R>(L);
        const R z = (vT[q] + ph.t_off) * ph.inv_dT;
        const R gq = clamp01(z), st = R(stored_rc(L, q, cell));
        const R rc = st > gq ? st : gq;
        k = ph.kp + rc * ph.dks + gq * ph.dkm;
        kd = (z > R(0) && z < R(1)) ? (gq > st ? ph.dks + ph.dkm : ph.dkm) * ph.inv_dT : R(0);
      } else if (NLK) {
        const R z = (vT[q] + mt.tk_off) * mt.inv_dT;
        k = mt.k0 + mt.dk * clamp01(z);
        kd = (z > R(0) && z < R(1)) ? mt.dk * mt.inv_dT : R(0);
      }
      const R flux = JAC ? k * g[q] + kd * vw[q] * gT[q] : k * gT[q];
      g[q] = flux * scale * (R(wq3<P>(q)) * cd);
    }
    if (d == 0) apply1d<P, 1, 0, true, true>(g, r);
    else if (d == 1) apply1d<P, 1, 1, true, true>(g, r);
    else apply1d<P, 1, 2, true, true>(g, r);
  }
  R fe[NP];
  integrate_values<P, R>(r, fe);
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    const int d = __ldg(&M.cell_dofs[a * M.n_cells + cell]);
    const double v = (double)fe[a];
    if (d >= 0) {
      atomicAdd(&y[d], v);
    } else {
      const int row = -1 - d;
      for (int e = __ldg(&M.con_ptr[row]); e < __ldg(&M.con_ptr[row + 1]); ++e)
        atomicAdd(&y[__ldg(&M.con_idx[e])], __ldg(&M.con_w[e]) * v);
    }
  }
}

template <int P, typename R, bool JAC>
cudaError_t go_newton(const CellLaunch& L, const double* T, const double* w, double* y, cudaStream_t s) {
  const int bs = 128;
  const unsigned grid = (unsigned)((L.mesh.n_cells + bs - 1) / bs);
  if (L.phase) k_newton<P, R, JAC, false, true><<<grid, bs, 0, s>>>(L, T, w, y);
  else if (L.nonlin_k) k_newton<P, R, JAC, true, false><<<grid, bs, 0, s>>>(L, T, w, y);
  else k_newton<P, R, JAC, false, false><<<grid, bs, 0, s>>>(L, T, w, y);
  return cudaGetLastError();
}

template <int P>
cudaError_t dispatch_newton(const CellLaunch& L, bool jac, const double* T, const double* w, double* y,
                            cudaStream_t s) {
  if (L.f32) return jac ? go_newton<P, float, true>(L, T, w, y, s) : go_newton<P, float, false>(L, T, w, y, s);
  return jac ? go_newton<P, double, true>(L, T, w, y, s) : go_newton<P, double, false>(L, T, w, y, s);
}

__global__ void k_sub(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] - b[i];
}

__global__ void k_copy_masked(int64_t n, double* __restrict__ y, const double* __restrict__ v,
                              const uint8_t* __restrict__ mask) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && mask[i]) y[i] = v[i];
}

// BiCGStab vector recurrences with the scalars in device memory (sc, see newton.cuh)
__global__ void k_bicg_p(int64_t n, double* __restrict__ p, const double* __restrict__ r,
                         const double* __restrict__ v, const double* __restrict__ sc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // beta = (rho_new / rho) (alpha / omega)
  const double beta = (sc[kScRhoNew] / sc[kScRho]) * (sc[kScAlpha] / sc[kScOmega]);
  p[i] = r[i] + beta * (p[i] - sc[kScOmega] * v[i]);
}

__global__ void k_bicg_s(int64_t n, double* __restrict__ s, const double* __restrict__ r,
                         const double* __restrict__ v, double* __restrict__ x, const double* __restrict__ yv,
                         double* __restrict__ sc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double alpha = sc[kScRhoNew] / sc[kScRhv];
  if (i == 0) sc[kScAlphaNext] = alpha;
  if (i >= n) return;
  s[i] = r[i] - alpha * v[i];
  x[i] += alpha * yv[i];
}

__global__ void k_bicg_x(int64_t n, double* __restrict__ x, const double* __restrict__ z, double* __restrict__ r,
                         const double* __restrict__ s, const double* __restrict__ t, double* __restrict__ sc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double omega = sc[kScTs] / sc[kScTt];
  if (i >= n) return;
  x[i] += omega * z[i];
  r[i] = s[i] - omega * t[i];
}

// the scalars of the next iteration: rho = rho_new, alpha = alpha_next, omega = (t.s)/(t.t)
__global__ void k_bicg_roll(double* __restrict__ sc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    sc[kScOmega] = sc[kScTs] / sc[kScTt];
    sc[kScRho] = sc[kScRhoNew];
    sc[kScAlpha] = sc[kScAlphaNext];
  }
}

}  // namespace

cudaError_t launch_newton(const CellLaunch& L, bool jac, const double* T, const double* w, double* y, cudaStream_t s) {
  if (L.mesh.batch != 1 || !T || !w || !y) return cudaErrorInvalidValue;
  if (L.mesh.n_cells == 0) return cudaSuccess;
  if (L.degree == 1) return dispatch_newton<1>(L, jac, T, w, y, s);
  if (L.degree == 2) return dispatch_newton<2>(L, jac, T, w, y, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_sub(int64_t n, const double* a, const double* b, double* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_sub<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, a, b, out);
  return cudaGetLastError();
}

cudaError_t launch_copy_masked(int64_t n, double* y, const double* v, const uint8_t* mask, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_copy_masked<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, y, v, mask);
  return cudaGetLastError();
}

cudaError_t launch_bicg_p(int64_t n, double* p, const double* r, const double* v, const double* sc, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_bicg_p<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, p, r, v, sc);
  return cudaGetLastError();
}

cudaError_t launch_bicg_s(int64_t n, double* sv, const double* r, const double* v, double* x, const double* y,
                          double* sc, cudaStream_t s) {
  k_bicg_s<<<(unsigned)(std::max<int64_t>(n, 1) + 255) / 256, 256, 0, s>>>(n, sv, r, v, x, y, sc);
  return cudaGetLastError();
}

cudaError_t launch_bicg_x(int64_t n, double* x, const double* z, double* r, const double* sv, const double* t,
                          double* sc, cudaStream_t s) {
  if (n > 0) k_bicg_x<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, x, z, r, sv, t, sc);
  k_bicg_roll<<<1, 32, 0, s>>>(sc);
  return cudaGetLastError();
}

}  // namespace pbf
