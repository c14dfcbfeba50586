// Launchers of the streaming kernels (vec_kernels.cu); internal to the library.
#pragma once

#include "internal.cuh"

namespace pbf {

struct LaserSetup {
  LaserK k;
  int n_top = 0;
  const int32_t* top_cell = nullptr;  // [n_top] active cell index
  const double* top_geo = nullptr;    // [n_top][4]: x0, y0, hx, hy of the face
  const double* cell_lo = nullptr;    // [n_cells][3] lower corner (volumetric source)
  const double* level_h = nullptr;    // [levels][3]
};

// Radiation and evaporation on the free top surface (Eqs. bc_radiation, bc_evaporation):
// outward flux q_rad + q_evap of the temperature, see pbf_surface_loss.
struct LossK {
  double emissivity = 0.0, T_amb = 0.0;
  double C_P = 0.0, C_T = 0.0, C_M = 0.0, T_v = 0.0, h_v = 0.0, c_h = 0.0, T_h0 = 0.0, T_max = 0.0;
};

__device__ __forceinline__ float expo_r(float x) { return __expf(x); }
__device__ __forceinline__ double expo_r(double x) { return exp(x); }

// dq/dT of the flux below: radiation 4 eps sigma T^3; evaporation, for T_v < T < T_max,
// mdot(T) ((C_T / T^2 - 1 / (2 T)) (h_v + c_h (T - T_h0)) + c_h); constant above the cap.
template <typename R>
__device__ __forceinline__ R surface_flux_deriv(const LossK& q, R T) {
  R d = R(4.0 * q.emissivity * 5.670374419e-8) * T * T * T;
  if (q.C_P > 0.0 && T < R(q.T_max) && T > R(q.T_v)) {
    const R mdot = R(0.82 * q.C_P) * expo_r(R(-q.C_T) * (R(1) / T - R(1.0 / q.T_v))) * sqrt(R(q.C_M) / T);
    d += mdot * ((R(q.C_T) / (T * T) - R(0.5) / T) * (R(q.h_v) + R(q.c_h) * (T - R(q.T_h0))) + R(q.c_h));
  }
  return d;
}

// -int_face N_i q(T_h) dA on one top face of size hx x hy, in precision R: Tf holds the
// temperatures of the face's (P+1)^2 nodes and fe receives the face nodes' contributions
// (both indexed k + (P+1) j, the face's x and y node indices). q = q_rad + q_evap, radiation
// eps sigma (T^4 - T_amb^4) with the Stefan-Boltzmann constant 5.670374419e-8 W m^-2 K^-4 and
// evaporation above T_v with T capped at T_max (Eqs. bc_rad_evap, bc_radiation,
// bc_evaporation), at the face's (P+1)^2 Gauss points.
template <int P, typename R>
__device__ __forceinline__ void add_surface_loss(const LossK& q, const R* Tf, R hx, R hy, R* fe) {
  constexpr int N = P + 1;
  const R eps_s = R(q.emissivity * 5.670374419e-8), Ta4 = R(q.T_amb * q.T_amb * q.T_amb * q.T_amb);
#pragma unroll
  for (int qy = 0; qy < N; ++qy)
#pragma unroll
    for (int qx = 0; qx < N; ++qx) {
      R T = R(0);
#pragma unroll
      for (int j = 0; j < N; ++j)
#pragma unroll
        for (int k = 0; k < N; ++k) T += R(Basis<P>::S(qy, j) * Basis<P>::S(qx, k)) * Tf[k + N * j];
      const R T2 = T * T;
      R flux = eps_s * (T2 * T2 - Ta4);
      const R Tc = T < R(q.T_max) ? T : R(q.T_max);
      if (q.C_P > 0.0 && Tc > R(q.T_v)) {
        const R mdot = R(0.82 * q.C_P) * expo_r(R(-q.C_T) * (R(1) / Tc - R(1.0 / q.T_v))) * sqrt(R(q.C_M) / Tc);
        flux += mdot * (R(q.h_v) + R(q.c_h) * (Tc - R(q.T_h0)));
      }
      const R wq = flux * R(Basis<P>::W(qx) * Basis<P>::W(qy)) * hx * hy;
#pragma unroll
      for (int j = 0; j < N; ++j)
#pragma unroll
        for (int k = 0; k < N; ++k) fe[k + N * j] -= wq * R(Basis<P>::S(qy, j) * Basis<P>::S(qx, k));
    }
}

// Lumped-capacity forms of the update: constant c, quadrature-point row sum accumulated by
// the cell kernel, or nodal apparent capacity c_app(T_i) x row-sum mass.
enum { CAP_CONST = 0, CAP_QUADRATURE = 1, CAP_NODAL = 2 };
struct NodalCap {
  double lat_ratio = 0.0, Tm = 0.0, inv_sigma = 0.0;  // c_app/c = 1 + lat_ratio exp(-((T-Tm) inv_sigma)^2/2)
  float lat_ratio_f = 0.f, tm_off_f = 0.f, inv_sigma_f = 0.f;  // FP32 form on T - T_ref
  // z^2 beyond which lat_ratio exp(-z^2/2) < 2^-26, so that 1 + lat_ratio exp(-z^2/2) rounds
  // to 1 in FP32 and the FP32 forms skip the exponential and the division
  float z2_cut_f = 0.f;
};
// The FP32-operator increment dt f / C~ of one dof (Eq. forward_euler), formed in FP32. C~ is
// the accumulated quadrature row sum ci, or comes from the inverse lumped capacity ic of the
// constant c, scaled for the nodal apparent capacity by 1 / (1 + lat_ratio exp(-z^2/2)) with z
// from the dof's FP32 value T - T_ref (value: only read for the nodal capacity).
template <int CAP>
__device__ __forceinline__ float increment_f32(float value, float fi, float ci, float ic, const NodalCap& nc,
                                               float dt) {
  if (CAP == CAP_QUADRATURE) return dt * fi / ci;
  if (CAP == CAP_NODAL) {
    const float z = (value + nc.tm_off_f) * nc.inv_sigma_f;
    const float z2 = z * z;
    const float r = dt * fi * ic;
    return z2 < nc.z2_cut_f ? __fdividef(r, 1.f + nc.lat_ratio_f * __expf(-0.5f * z2)) : r;
  }
  return dt * fi * ic;
}

// x + b for an unevaluated FP32 pair x = hi + lo (|lo| <= ulp(hi) / 2) and an FP32 b: the
// sum is formed exactly by TwoSum and renormalised by Fast2Sum (Knuth; Dekker), so the pair
// keeps about 48 significant bits without FP64 arithmetic (on this GPU FP64 operations and
// conversions run at about 1/60 of the FP32 rate).
__device__ __forceinline__ float2 ff_add(float2 x, float b) {
  const float s = x.x + b;
  const float bb = s - x.x;
  const float err = (x.x - (s - bb)) + (b - bb);  // s + err == x.x + b exactly
  const float t = x.y + err;
  const float hi = s + t;
  return make_float2(hi, t - (hi - s));
}

cudaError_t launch_update_f64(int cap, int64_t n_dofs, int B, double* T, double* f, double* Cacc,
                              const double* invC0, const NodalCap& nc, const uint8_t* dirichlet, double T_dir,
                              double dt, cudaStream_t s);
// The FP32-operator update of the pair state hi + lo = T - T_ref ([n_dofs][B]); x_dir is the
// pair of T_D - T_ref.
cudaError_t launch_update_f32(int cap, int64_t n_dofs, int B, float* hi, float* lo, float* f, float* Cacc,
                              const float* invC0, const NodalCap& nc, const uint8_t* dirichlet, float2 x_dir, float dt,
                              cudaStream_t s);
// x_h = P_h x with f_h (and C_h, nullable) cleared
cudaError_t launch_hang_values_zero(bool f32, const DevMesh& M, const void* x, void* out, void* fh, void* Ch,
                                    cudaStream_t s);
// C_out[d][b] = C0[d] c_app(T[d][b]) / c (nodal lumping) in FP64
cudaError_t launch_capacity_nodal(int64_t n_dofs, int B, const double* C0, const double* T, const NodalCap& nc,
                                  double* C_out, cudaStream_t s);
// hi + lo = T - off as an FP32 pair (lo nullable: hi only) / T = off + (hi + lo) in FP64
cudaError_t launch_prepare_f32(int64_t n, const double* T, double off, float* hi, float* lo, cudaStream_t s);
cudaError_t launch_finish_f32(int64_t n, const float* hi, const float* lo, double off, double* T, cudaStream_t s);
cudaError_t launch_round_f32(int64_t n, const double* x, float* y, cudaStream_t s);
cudaError_t launch_f32_to_f64(int64_t n, const float* x, double* y, cudaStream_t s);
cudaError_t launch_laser(int degree, bool f32, const LaserSetup& ls, const DevMesh& M, const double* power,
                         const Spot& sp, void* f, cudaStream_t s);
// f += -int_{top faces} N_i (q_rad + q_evap)(T_h) dA, (p+1)^2 Gauss points per face, for the
// state x ([n_dofs][batch] in the operator precision; T = x + T_off; hanging values from the
// constraint rows), constraint-resolved atomic additions onto f.
cudaError_t launch_surface_loss(int degree, bool f32, const LaserSetup& ls, const DevMesh& M, const void* x,
                                double T_off, const LossK& q, void* f, cudaStream_t s);
// The transposed linearisation of that term (adjoint sweep): g -= int_{top faces} q'(T_h) v_h N_j dA
// for the state x (T = x + T_off) and the adjoint vector v, both [n_dofs][batch] in the operator
// precision, constraint-resolved atomic additions onto g.
cudaError_t launch_surface_loss_adjoint(int degree, bool f32, const LaserSetup& ls, const DevMesh& M, const void* x,
                                        double T_off, const void* v, const LossK& q, void* g, cudaStream_t s);
// r_c = 0 in powder cells, 1 elsewhere, for the nq quadrature points of every cell and instance
cudaError_t launch_phase_init(bool f32, int nq, const DevMesh& M, void* rc, cudaStream_t s);
cudaError_t launch_to_f64(bool f32, int64_t n, const void* a, double* out, cudaStream_t s);
cudaError_t launch_broadcast_dofs(int64_t n_dofs, int B, const double* a, double* out, cudaStream_t s);
// inv_d = 1 / c, inv_f = its FP32 rounding; inv_fx (nullable) the same with -1 at Dirichlet dofs
cudaError_t launch_reciprocal(int64_t n, const double* c, double* inv_d, float* inv_f, float* inv_fx,
                              const uint8_t* dirichlet, cudaStream_t s);
// x_h = P_h x (values at hanging nodes) and f += P_h^T f_h (f_h cleared); FP32 or FP64 arrays
cudaError_t launch_hang_values(bool f32, const DevMesh& M, const void* x, void* out, cudaStream_t s);
cudaError_t launch_hang_distribute(bool f32, const DevMesh& M, void* fh, void* f, cudaStream_t s);
cudaError_t launch_axpy2(int64_t n, double alpha, const double* p, const double* Ap, double* x, double* r,
                         cudaStream_t s);
cudaError_t launch_xpby(int64_t n, const double* z, double beta, double* p, cudaStream_t s);
// x += (num/den) p, r -= (num/den) Ap and p = z + (num/den) p with the scalars in device memory
cudaError_t launch_axpy2_dev(int64_t n, const double* num, const double* den, const double* p, const double* Ap,
                             double* x, double* r, cudaStream_t s);
cudaError_t launch_xpby_dev(int64_t n, const double* z, const double* num, const double* den, double* p,
                            cudaStream_t s);
cudaError_t launch_cheb_init(int64_t n, const double* r, const double* diag, double inv_theta, double* res, double* d,
                             double* z, const uint8_t* mask, cudaStream_t s);
cudaError_t launch_cheb_update(int64_t n, const double* Ad, double* res, double* d, double* z, const double* diag,
                               double a, double b, const uint8_t* mask, cudaStream_t s);
cudaError_t launch_jacobi(int64_t n, const double* r, const double* diag, double* z, const uint8_t* mask,
                          cudaStream_t s);
cudaError_t launch_neg_masked(int64_t n, double* y, const uint8_t* mask, cudaStream_t s);
cudaError_t launch_add(int64_t n, double* T, const double* x, cudaStream_t s);
// adjoint sweep helpers (FP64). fre (nullable): the surface loss's part of f, not in fv
cudaError_t launch_adj_prepare(int n, int B, const double* lam, const double* fd, const double* fv, const double* fre,
                               const double* Cm, const uint8_t* dir, double* v, double* mu, double* q1, double* q2,
                               cudaStream_t s);
cudaError_t launch_objective(int ns, int B, const int32_t* sidx, const double* sw, const double* T, double W, double p,
                             double Tt, double invN, int accumulate, double* part, double* J, double* coef,
                             cudaStream_t s);
cudaError_t launch_lambda_objective(int ns, int B, const int32_t* sidx, const double* sw, const double* T, double p,
                                    const double* coef, const uint8_t* dir, double* lam, cudaStream_t s);
cudaError_t launch_lambda_update(bool f32, bool nodal, int n, int B, double* lam, void* g, const double* mu,
                                 const double* C0, const double* T, const NodalCap& nc, const uint8_t* dir, double dt,
                                 cudaStream_t s);
cudaError_t launch_grad_accum(int B, int nseg, int seg, const double* d1, const double* d2, const double* sc,
                              const double* power, double dt, double* grad, cudaStream_t s);
cudaError_t launch_surface_weights(int degree, int n_top, const int32_t* top_cell, const double* top_geo,
                                   const DevMesh& M, double* w, cudaStream_t s);
int reduction_blocks();
// out[b] = sum_d w_d x[d][b] y[d][b] over dofs with !skip[d]; part: [reduction_blocks()][B]
cudaError_t launch_dot(int64_t n_dofs, int B, const double* x, const double* y, const double* w, const uint8_t* skip,
                       double* part, double* out, cudaStream_t s);
cudaError_t launch_scale_masked(int64_t n, double* x, const double* sc, const uint8_t* zero_mask, cudaStream_t s);
cudaError_t launch_div_masked(int64_t n, double* x, const double* y, const double* invC, const uint8_t* mask,
                              cudaStream_t s);
cudaError_t launch_zero_masked(int64_t n, double* y, const uint8_t* mask, cudaStream_t s);
cudaError_t launch_set_masked(int64_t n, double* y, const uint8_t* mask, double v, cudaStream_t s);
cudaError_t launch_transfer(int64_t n_new, int B, const int32_t* ptr, const int32_t* idx, const double* w,
                            const double* Told, double fill, double* Tnew, cudaStream_t s);

// history of the phase model across mesh changes (kernels_history.cu)
// out[c] = min over the quadrature points and instances of r_c ([q][n_cells][B])
cudaError_t launch_history_min(bool f32, int nq, int n_cells, int B, const void* rc, double* out, cudaStream_t s);
// r_c on a changed mesh through the host-built map ([cell][q]: old cell * nq + old q, -1 / -2)
cudaError_t launch_history_gather(bool f32, int nq, int n_new, int n_old, int B, const int32_t* map, const void* rc_old,
                                  void* rc_new, cudaStream_t s);
// r_c to (to_f64) or from an FP64 array of the same layout
cudaError_t launch_history_copy(bool f32, bool to_f64, int64_t n, const void* in, void* out, cudaStream_t s);

}  // namespace pbf
