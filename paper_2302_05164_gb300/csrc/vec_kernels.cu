// Streaming kernels of the library: the forward-Euler update with the lumped-capacity
// inverse (Eq. forward_euler), the laser-source quadrature on top faces, deterministic FP64
// reductions, CG / Chebyshev vector recurrences and the field-transfer gather.
#include "vec_kernels.cuh"

namespace pbf {
namespace {

constexpr int kBS = 256;

inline unsigned grid_for(int64_t n, int bs = kBS) { return (unsigned)((n + bs - 1) / bs); }

// ---- forward-Euler update -------------------------------------------------------------
// T_i <- T_i + dt f_i / C~_i on free dofs, T_i <- T_D on Dirichlet dofs; f (and the capacity
// accumulator) are cleared for the next step.
//
// FP64 operator: in place on the FP64 state.
template <int CAP>
__global__ void k_update_f64(int64_t n, int B, double* __restrict__ T, double* __restrict__ f,
                             double* __restrict__ Cacc, const double* __restrict__ invC0, const NodalCap nc,
                             const uint8_t* __restrict__ dirichlet, double T_dir, double dt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t d = i / B;
  const double fi = f[i];
  f[i] = 0.0;
  double ci = 0.0;
  if (CAP == CAP_QUADRATURE) {
    ci = Cacc[i];
    Cacc[i] = 0.0;
  }
  if (dirichlet[d]) {
    T[i] = T_dir;
    return;
  }
  if (CAP == CAP_QUADRATURE) {
    T[i] += dt * fi / ci;
  } else if (CAP == CAP_NODAL) {
    const double z = (T[i] - nc.Tm) * nc.inv_sigma;
    T[i] += dt * fi * invC0[d] / (1.0 + nc.lat_ratio * exp(-0.5 * z * z));
  } else {
    T[i] += dt * fi * invC0[d];
  }
}

// FP32 operator: the increment dt f / C~ is formed in FP32 and added to the FP64 working
// state Tw = T - T_ref (one FP64 add per dof); the FP32 copy Tf = round(Tw) that the cell
// kernel gathers is refreshed in the same pass.
template <int CAP>
__global__ void k_update_f32(int64_t n, int B, double* __restrict__ Tw, float* __restrict__ Tf,
                             float* __restrict__ f, float* __restrict__ Cacc, const float* __restrict__ invC0,
                             const NodalCap nc, const uint8_t* __restrict__ dirichlet, double tw_dir, float tf_dir,
                             float dt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t d = i / B;
  const float fi = f[i];
  f[i] = 0.f;
  float ci = 0.f;
  if (CAP == CAP_QUADRATURE) {
    ci = Cacc[i];
    Cacc[i] = 0.f;
  }
  if (dirichlet[d]) {
    Tw[i] = tw_dir;
    Tf[i] = tf_dir;
    return;
  }
  const double tw = Tw[i];
  float inc;
  if (CAP == CAP_QUADRATURE) {
    inc = dt * fi / ci;
  } else if (CAP == CAP_NODAL) {
    const float z = (d2f_rn(tw) + nc.tm_off_f) * nc.inv_sigma_f;
    inc = dt * fi * invC0[d] / (1.f + nc.lat_ratio_f * __expf(-0.5f * z * z));
  } else {
    inc = dt * fi * invC0[d];
  }
  const double t = tw + f2d(inc);
  Tw[i] = t;
  Tf[i] = d2f_rn(t);
}

__global__ void k_capacity_nodal(int64_t n, int B, const double* __restrict__ C0, const double* __restrict__ T,
                                 const NodalCap nc, double* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double z = (T[i] - nc.Tm) * nc.inv_sigma;
  out[i] = C0[i / B] * (1.0 + nc.lat_ratio * exp(-0.5 * z * z));
}

// Tw = T - off (FP64), Tf = round_to_f32(Tw); Tw may be null
__global__ void k_prepare_f32(int64_t n, const double* __restrict__ T, double off, double* __restrict__ Tw,
                              float* __restrict__ Tf) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double t = T[i] - off;
  if (Tw) Tw[i] = t;
  Tf[i] = d2f_rn(t);
}

__global__ void k_finish_f32(int64_t n, const double* __restrict__ Tw, double off, double* __restrict__ T) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) T[i] = Tw[i] + off;
}

// ---- laser on top faces ------------------------------------------------------------------
// f_i += int_face N_i 2 eta P/(pi r^2) exp(-2 d^2/r^2) dA, (P+1)^2 Gauss points per face;
// faces farther than 6 r from the spot are skipped (the integrand is below e^-72 there).
// The spot position and active segment come from the host, evaluated once per step.
template <int P, typename R>
__global__ void k_laser_surface(int n_top, int B, const int32_t* __restrict__ top_cell,
                                const double* __restrict__ top_geo, const DevMesh M, const LaserK ls,
                                const double* __restrict__ power, Spot sp, R* __restrict__ f) {
  constexpr int N = P + 1;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n_top * B) return;
  const int face = (int)(i / B), inst = (int)(i - (int64_t)face * B);
  const double lx = sp.x, ly = sp.y;
  const int seg = sp.seg;
  const double x0 = top_geo[4 * face + 0], y0 = top_geo[4 * face + 1];
  const double hx = top_geo[4 * face + 2], hy = top_geo[4 * face + 3];
  const double r = ls.radius;
  const double gx = fmax(0.0, fmax(x0 - lx, lx - (x0 + hx))), gy = fmax(0.0, fmax(y0 - ly, ly - (y0 + hy)));
  if (gx * gx + gy * gy > 36.0 * r * r) return;
  const double P0 = power[(int64_t)inst * kMaxSeg + seg];
  const double amp = 2.0 * ls.eta * P0 / (kPi * r * r);
  const double ir2 = 2.0 / (r * r);
  double fe[N][N];
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int k = 0; k < N; ++k) fe[j][k] = 0.0;
#pragma unroll
  for (int qy = 0; qy < N; ++qy)
#pragma unroll
    for (int qx = 0; qx < N; ++qx) {
      const double x = x0 + Basis<P>::X(qx) * hx, y = y0 + Basis<P>::X(qy) * hy;
      const double d2 = (x - lx) * (x - lx) + (y - ly) * (y - ly);
      const double q = amp * exp(-d2 * ir2) * Basis<P>::W(qx) * Basis<P>::W(qy) * hx * hy;
#pragma unroll
      for (int j = 0; j < N; ++j)
#pragma unroll
        for (int k = 0; k < N; ++k) fe[j][k] += q * Basis<P>::S(qy, j) * Basis<P>::S(qx, k);
    }
  const int cell = top_cell[face];
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int a = k + N * (j + N * P);  // local node (k, j, P) on the top face
      const int d = M.cell_dofs[a * M.n_cells + cell];
      if (d >= 0) {
        atomicAdd(&f[(int64_t)d * B + inst], R(fe[j][k]));
      } else {
        for (int e = M.con_ptr[-1 - d]; e < M.con_ptr[-d]; ++e)
          atomicAdd(&f[(int64_t)M.con_idx[e] * B + inst], R(M.con_w[e] * fe[j][k]));
      }
    }
}

// Cylinder source of depth h_powder below the active top (Eq. heat_soruce_cylindrical with
// the bound read as -h_powder < z^ < 0), integrated with (P+1)^3 Gauss points per cell.
template <int P, typename R>
__global__ void k_laser_volume(int n_cells, int B, const double* __restrict__ cell_lo,
                               const uint8_t* __restrict__ cell_level, const double* __restrict__ level_h,
                               const DevMesh M, const LaserK ls, const double* __restrict__ power, Spot sp,
                               R* __restrict__ f) {
  constexpr int N = P + 1, NP = N * N * N;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n_cells * B) return;
  const int cell = (int)(i / B), inst = (int)(i - (int64_t)cell * B);
  const double lx = sp.x, ly = sp.y;
  const int seg = sp.seg;
  const int lev = cell_level[cell];
  const double x0 = cell_lo[3 * cell], y0 = cell_lo[3 * cell + 1], z0 = cell_lo[3 * cell + 2];
  const double hx = level_h[3 * lev], hy = level_h[3 * lev + 1], hz = level_h[3 * lev + 2];
  const double zt = ls.z_top;
  if (z0 >= zt || z0 + hz <= zt - ls.h_powder) return;
  const double r = ls.radius;
  const double gx = fmax(0.0, fmax(x0 - lx, lx - (x0 + hx))), gy = fmax(0.0, fmax(y0 - ly, ly - (y0 + hy)));
  if (gx * gx + gy * gy > 36.0 * r * r) return;
  const double amp = 2.0 * ls.eta * power[(int64_t)inst * kMaxSeg + seg] / (kPi * r * r * ls.h_powder);
  double fe[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) fe[a] = 0.0;
#pragma unroll
  for (int qz = 0; qz < N; ++qz) {
    const double z = z0 + Basis<P>::X(qz) * hz;
    const double zh = z - zt;
    if (!(zh > -ls.h_powder && zh < 0.0)) continue;
#pragma unroll
    for (int qy = 0; qy < N; ++qy)
#pragma unroll
      for (int qx = 0; qx < N; ++qx) {
        const double x = x0 + Basis<P>::X(qx) * hx, y = y0 + Basis<P>::X(qy) * hy;
        const double d2 = (x - lx) * (x - lx) + (y - ly) * (y - ly);
        const double q = amp * exp(-2.0 * d2 / (r * r)) * Basis<P>::W(qx) * Basis<P>::W(qy) * Basis<P>::W(qz) * hx * hy * hz;
#pragma unroll
        for (int a = 0; a < NP; ++a)
          fe[a] += q * Basis<P>::S(qx, a % N) * Basis<P>::S(qy, (a / N) % N) * Basis<P>::S(qz, a / (N * N));
      }
  }
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    const int d = M.cell_dofs[a * M.n_cells + cell];
    if (d >= 0) {
      atomicAdd(&f[(int64_t)d * B + inst], R(fe[a]));
    } else {
      for (int e = M.con_ptr[-1 - d]; e < M.con_ptr[-d]; ++e)
        atomicAdd(&f[(int64_t)M.con_idx[e] * B + inst], R(M.con_w[e] * fe[a]));
    }
  }
}

template <typename R>
__global__ void k_to_f64(int64_t n, const R* __restrict__ a, double* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (double)a[i];
}

__global__ void k_round_f32(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = d2f_rn(x[i]);
}

__global__ void k_f32_to_f64(int64_t n, const float* __restrict__ x, double* __restrict__ y) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = f2d(x[i]);
}

__global__ void k_broadcast_dofs(int64_t n, int B, const double* __restrict__ a, double* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i / B];
}

__global__ void k_reciprocal(int64_t n, const double* __restrict__ c, double* __restrict__ inv_d,
                             float* __restrict__ inv_f) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double v = 1.0 / c[i];
    inv_d[i] = v;
    inv_f[i] = (float)v;
  }
}

// ---- deterministic reductions -------------------------------------------------------------
// sum_i w_i x_i y_i per instance (w may be null; a mask m zeroes dofs with m != 0). Each
// block reduces a fixed slice in a fixed order; the second pass adds the block partials in
// order, so the result does not depend on scheduling.
constexpr int kRedBlocks = 304;  // 2 x 152 SMs

__global__ void k_dot_partial(int64_t n_dofs, int B, const double* __restrict__ x, const double* __restrict__ y,
                              const double* __restrict__ w, const uint8_t* __restrict__ skip,
                              double* __restrict__ part) {
  // part[blockIdx.x * B + b]
  __shared__ double sh[kBS];
  const int64_t per = (n_dofs + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * per, hi = min(n_dofs, lo + per);
  for (int b = 0; b < B; ++b) {
    double s = 0.0;
    for (int64_t d = lo + threadIdx.x; d < hi; d += blockDim.x) {
      if (skip && skip[d]) continue;
      const double v = x[d * B + b] * y[d * B + b];
      s += w ? w[d] * v : v;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * B + b] = sh[0];
    __syncthreads();
  }
}

__global__ void k_dot_final(int nblk, int B, const double* __restrict__ part, double* __restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double s = 0.0;
  for (int k = 0; k < nblk; ++k) s += part[(int64_t)k * B + b];
  out[b] = s;
}

// ---- vector recurrences -------------------------------------------------------------------
__global__ void k_scale_masked(int64_t n, double* __restrict__ x, const double* __restrict__ s,
                               const uint8_t* __restrict__ zero_mask) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] = (zero_mask && zero_mask[i]) ? 0.0 : x[i] * s[0];
}

// power iteration: x = y / C (free dofs), y on Dirichlet = 0
__global__ void k_div_masked(int64_t n, double* __restrict__ x, const double* __restrict__ y,
                             const double* __restrict__ invC, const uint8_t* __restrict__ mask) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] = mask[i] ? 0.0 : y[i] * invC[i];
}

__global__ void k_zero_masked(int64_t n, double* __restrict__ y, const uint8_t* __restrict__ mask) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && mask[i]) y[i] = 0.0;
}

__global__ void k_set_masked(int64_t n, double* __restrict__ y, const uint8_t* __restrict__ mask, double v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && mask[i]) y[i] = v;
}

// ---- hanging-node constraints around the cell kernel ----------------------------------------
// x_h = P_h x: values at hanging nodes from their masters (before the cell kernel)
template <typename R>
__global__ void k_hang_values(int n_hang, int B, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                              const R* __restrict__ w, const R* __restrict__ x, R* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n_hang * B) return;
  const int r = (int)(i / B), b = (int)(i - (int64_t)r * B);
  R s = R(0);
  for (int e = ptr[r]; e < ptr[r + 1]; ++e) s += w[e] * x[(int64_t)idx[e] * B + b];
  out[i] = s;
}

// f += P_h^T f_h, f_h <- 0 (after the cell kernel)
template <typename R>
__global__ void k_hang_distribute(int n_hang, int B, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                  const R* __restrict__ w, R* __restrict__ fh, R* __restrict__ f) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n_hang * B) return;
  const int r = (int)(i / B), b = (int)(i - (int64_t)r * B);
  const R v = fh[i];
  if (v == R(0)) return;
  fh[i] = R(0);
  for (int e = ptr[r]; e < ptr[r + 1]; ++e) atomicAdd(&f[(int64_t)idx[e] * B + b], w[e] * v);
}

// ---- field transfer -----------------------------------------------------------------------
__global__ void k_transfer(int64_t n_new, int B, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                           const double* __restrict__ w, const double* __restrict__ Told, double fill,
                           double* __restrict__ Tnew) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_new * B) return;
  const int64_t d = i / B;
  const int b = (int)(i - d * B);
  const int e0 = ptr[d], e1 = ptr[d + 1];
  if (e0 == e1) {
    Tnew[i] = fill;
    return;
  }
  double s = 0.0;
  for (int e = e0; e < e1; ++e) s += w[e] * Told[(int64_t)idx[e] * B + b];
  Tnew[i] = s;
}

}  // namespace

// ---- host launchers -------------------------------------------------------------------------

Spot spot_at(const LaserK& k, double t) {
  Spot sp;
  for (int i = 0; i < k.n_seg; ++i) {
    const double* g = k.seg[i];
    if (t >= g[4] && t < g[5]) {
      const double a = (t - g[4]) / (g[5] - g[4]);
      sp.x = g[0] + (g[2] - g[0]) * a;
      sp.y = g[1] + (g[3] - g[1]) * a;
      sp.seg = i;
      return sp;
    }
  }
  return sp;
}

cudaError_t launch_update_f64(int cap, int64_t n_dofs, int B, double* T, double* f, double* Cacc,
                              const double* invC0, const NodalCap& nc, const uint8_t* dirichlet, double T_dir,
                              double dt, cudaStream_t s) {
  const int64_t n = n_dofs * B;
  if (n == 0) return cudaSuccess;
  if (cap == CAP_QUADRATURE) k_update_f64<CAP_QUADRATURE><<<grid_for(n), kBS, 0, s>>>(n, B, T, f, Cacc, invC0, nc, dirichlet, T_dir, dt);
  else if (cap == CAP_NODAL) k_update_f64<CAP_NODAL><<<grid_for(n), kBS, 0, s>>>(n, B, T, f, Cacc, invC0, nc, dirichlet, T_dir, dt);
  else k_update_f64<CAP_CONST><<<grid_for(n), kBS, 0, s>>>(n, B, T, f, Cacc, invC0, nc, dirichlet, T_dir, dt);
  return cudaGetLastError();
}

cudaError_t launch_update_f32(int cap, int64_t n_dofs, int B, double* Tw, float* Tf, float* f, float* Cacc,
                              const float* invC0, const NodalCap& nc, const uint8_t* dirichlet, double tw_dir,
                              float tf_dir, float dt, cudaStream_t s) {
  const int64_t n = n_dofs * B;
  if (n == 0) return cudaSuccess;
  if (cap == CAP_QUADRATURE) k_update_f32<CAP_QUADRATURE><<<grid_for(n), kBS, 0, s>>>(n, B, Tw, Tf, f, Cacc, invC0, nc, dirichlet, tw_dir, tf_dir, dt);
  else if (cap == CAP_NODAL) k_update_f32<CAP_NODAL><<<grid_for(n), kBS, 0, s>>>(n, B, Tw, Tf, f, Cacc, invC0, nc, dirichlet, tw_dir, tf_dir, dt);
  else k_update_f32<CAP_CONST><<<grid_for(n), kBS, 0, s>>>(n, B, Tw, Tf, f, Cacc, invC0, nc, dirichlet, tw_dir, tf_dir, dt);
  return cudaGetLastError();
}

cudaError_t launch_capacity_nodal(int64_t n_dofs, int B, const double* C0, const double* T, const NodalCap& nc,
                                  double* C_out, cudaStream_t s) {
  const int64_t n = n_dofs * B;
  if (n == 0) return cudaSuccess;
  k_capacity_nodal<<<grid_for(n), kBS, 0, s>>>(n, B, C0, T, nc, C_out);
  return cudaGetLastError();
}

cudaError_t launch_prepare_f32(int64_t n, const double* T, double off, double* Tw, float* Tf, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_prepare_f32<<<grid_for(n), kBS, 0, s>>>(n, T, off, Tw, Tf);
  return cudaGetLastError();
}

cudaError_t launch_finish_f32(int64_t n, const double* Tw, double off, double* T, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_finish_f32<<<grid_for(n), kBS, 0, s>>>(n, Tw, off, T);
  return cudaGetLastError();
}

cudaError_t launch_round_f32(int64_t n, const double* x, float* y, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_round_f32<<<grid_for(n), kBS, 0, s>>>(n, x, y);
  return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(int64_t n, const float* x, double* y, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_f32_to_f64<<<grid_for(n), kBS, 0, s>>>(n, x, y);
  return cudaGetLastError();
}

cudaError_t launch_laser(int degree, bool f32, const LaserSetup& ls, const DevMesh& M, const double* power,
                         const Spot& sp, void* f, cudaStream_t s) {
  const int B = M.batch;
  if (sp.seg < 0) return cudaSuccess;
  if (ls.k.volumetric) {
    const int64_t n = (int64_t)M.n_cells * B;
    if (n == 0) return cudaSuccess;
    if (degree == 1) {
      if (f32) k_laser_volume<1, float><<<grid_for(n), 128, 0, s>>>(M.n_cells, B, ls.cell_lo, M.cell_level, ls.level_h, M, ls.k, power, sp, (float*)f);
      else k_laser_volume<1, double><<<grid_for(n), 128, 0, s>>>(M.n_cells, B, ls.cell_lo, M.cell_level, ls.level_h, M, ls.k, power, sp, (double*)f);
    } else {
      if (f32) k_laser_volume<2, float><<<grid_for(n), 128, 0, s>>>(M.n_cells, B, ls.cell_lo, M.cell_level, ls.level_h, M, ls.k, power, sp, (float*)f);
      else k_laser_volume<2, double><<<grid_for(n), 128, 0, s>>>(M.n_cells, B, ls.cell_lo, M.cell_level, ls.level_h, M, ls.k, power, sp, (double*)f);
    }
    return cudaGetLastError();
  }
  const int64_t n = (int64_t)ls.n_top * B;
  if (n == 0) return cudaSuccess;
  if (degree == 1) {
    if (f32) k_laser_surface<1, float><<<grid_for(n, 128), 128, 0, s>>>(ls.n_top, B, ls.top_cell, ls.top_geo, M, ls.k, power, sp, (float*)f);
    else k_laser_surface<1, double><<<grid_for(n, 128), 128, 0, s>>>(ls.n_top, B, ls.top_cell, ls.top_geo, M, ls.k, power, sp, (double*)f);
  } else {
    if (f32) k_laser_surface<2, float><<<grid_for(n, 128), 128, 0, s>>>(ls.n_top, B, ls.top_cell, ls.top_geo, M, ls.k, power, sp, (float*)f);
    else k_laser_surface<2, double><<<grid_for(n, 128), 128, 0, s>>>(ls.n_top, B, ls.top_cell, ls.top_geo, M, ls.k, power, sp, (double*)f);
  }
  return cudaGetLastError();
}

cudaError_t launch_to_f64(bool f32, int64_t n, const void* a, double* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (f32) k_to_f64<float><<<grid_for(n), kBS, 0, s>>>(n, (const float*)a, out);
  else k_to_f64<double><<<grid_for(n), kBS, 0, s>>>(n, (const double*)a, out);
  return cudaGetLastError();
}

cudaError_t launch_broadcast_dofs(int64_t n_dofs, int B, const double* a, double* out, cudaStream_t s) {
  const int64_t n = n_dofs * B;
  if (n == 0) return cudaSuccess;
  k_broadcast_dofs<<<grid_for(n), kBS, 0, s>>>(n, B, a, out);
  return cudaGetLastError();
}

cudaError_t launch_reciprocal(int64_t n, const double* c, double* inv_d, float* inv_f, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_reciprocal<<<grid_for(n), kBS, 0, s>>>(n, c, inv_d, inv_f);
  return cudaGetLastError();
}

cudaError_t launch_hang_values(bool f32, const DevMesh& M, const void* x, void* out, cudaStream_t s) {
  const int64_t n = (int64_t)M.n_hang * M.batch;
  if (n == 0) return cudaSuccess;
  if (f32) k_hang_values<float><<<grid_for(n), kBS, 0, s>>>(M.n_hang, M.batch, M.con_ptr, M.con_idx, M.con_wf, (const float*)x, (float*)out);
  else k_hang_values<double><<<grid_for(n), kBS, 0, s>>>(M.n_hang, M.batch, M.con_ptr, M.con_idx, M.con_w, (const double*)x, (double*)out);
  return cudaGetLastError();
}

cudaError_t launch_hang_distribute(bool f32, const DevMesh& M, void* fh, void* f, cudaStream_t s) {
  const int64_t n = (int64_t)M.n_hang * M.batch;
  if (n == 0) return cudaSuccess;
  if (f32) k_hang_distribute<float><<<grid_for(n), kBS, 0, s>>>(M.n_hang, M.batch, M.con_ptr, M.con_idx, M.con_wf, (float*)fh, (float*)f);
  else k_hang_distribute<double><<<grid_for(n), kBS, 0, s>>>(M.n_hang, M.batch, M.con_ptr, M.con_idx, M.con_w, (double*)fh, (double*)f);
  return cudaGetLastError();
}

int reduction_blocks() { return kRedBlocks; }

cudaError_t launch_dot(int64_t n_dofs, int B, const double* x, const double* y, const double* w, const uint8_t* skip,
                       double* part, double* out, cudaStream_t s) {
  k_dot_partial<<<kRedBlocks, kBS, 0, s>>>(n_dofs, B, x, y, w, skip, part);
  k_dot_final<<<(B + 63) / 64, 64, 0, s>>>(kRedBlocks, B, part, out);
  return cudaGetLastError();
}

cudaError_t launch_scale_masked(int64_t n, double* x, const double* sc, const uint8_t* zero_mask, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_scale_masked<<<grid_for(n), kBS, 0, s>>>(n, x, sc, zero_mask);
  return cudaGetLastError();
}

cudaError_t launch_div_masked(int64_t n, double* x, const double* y, const double* invC, const uint8_t* mask,
                              cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_div_masked<<<grid_for(n), kBS, 0, s>>>(n, x, y, invC, mask);
  return cudaGetLastError();
}

cudaError_t launch_zero_masked(int64_t n, double* y, const uint8_t* mask, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_zero_masked<<<grid_for(n), kBS, 0, s>>>(n, y, mask);
  return cudaGetLastError();
}

cudaError_t launch_set_masked(int64_t n, double* y, const uint8_t* mask, double v, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_set_masked<<<grid_for(n), kBS, 0, s>>>(n, y, mask, v);
  return cudaGetLastError();
}

cudaError_t launch_transfer(int64_t n_new, int B, const int32_t* ptr, const int32_t* idx, const double* w,
                            const double* Told, double fill, double* Tnew, cudaStream_t s) {
  const int64_t n = n_new * B;
  if (n == 0) return cudaSuccess;
  k_transfer<<<grid_for(n), kBS, 0, s>>>(n_new, B, ptr, idx, w, Told, fill, Tnew);
  return cudaGetLastError();
}

}  // namespace pbf
