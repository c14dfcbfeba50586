// Launchers of the nonlinear backward-Euler kernels (kernels_newton.cu); internal.
#pragma once

#include "internal.cuh"

namespace pbf {

// y += the residual (jac = false; w = T - T_n) or the Jacobian applied to w (jac = true) of
// the nonlinear backward Euler step at the state T (FP64 arrays, one instance); L carries
// the mesh, material (m_impl = rho c / dt) and precision. Dirichlet rows are not touched.
cudaError_t launch_newton(const CellLaunch& L, bool jac, const double* T, const double* w, double* y, cudaStream_t s);
// out = a - b
cudaError_t launch_sub(int64_t n, const double* a, const double* b, double* out, cudaStream_t s);
// y_i = v_i where mask_i != 0
cudaError_t launch_copy_masked(int64_t n, double* y, const double* v, const uint8_t* mask, cudaStream_t s);

// BiCGStab scalars in device memory (offsets into the context's 16 device scalars)
constexpr int kScSs = 2, kScRr = 3;  // s.s and r.r for the stopping tests
constexpr int kScRho = 8, kScRhoNew = 9, kScAlpha = 10, kScAlphaNext = 11, kScOmega = 12, kScRhv = 13, kScTs = 14,
              kScTt = 15;
// p = r + beta (p - omega v), beta = (rho_new / rho) (alpha / omega)
cudaError_t launch_bicg_p(int64_t n, double* p, const double* r, const double* v, const double* sc, cudaStream_t s);
// alpha = rho_new / (rh.v) (kept for the next iteration); s = r - alpha v, x += alpha y
cudaError_t launch_bicg_s(int64_t n, double* sv, const double* r, const double* v, double* x, const double* y,
                          double* sc, cudaStream_t s);
// omega = (t.s) / (t.t); x += omega z, r = s - omega t; then rho = rho_new, alpha, omega rolled
cudaError_t launch_bicg_x(int64_t n, double* x, const double* z, double* r, const double* sv, const double* t,
                          double* sc, cudaStream_t s);

}  // namespace pbf
