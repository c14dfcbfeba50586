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
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int d = B == 1 ? i : i / B;
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

__global__ void k_capacity_nodal(int64_t n, int B, const double* __restrict__ C0, const double* __restrict__ T,
                                 const NodalCap nc, double* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double z = (T[i] - nc.Tm) * nc.inv_sigma;
  out[i] = C0[i / B] * (1.0 + nc.lat_ratio * exp(-0.5 * z * z));
}

// FP32 operator: the working state T - T_ref is an unevaluated FP32 pair hi + lo (about 48
// significant bits; hi is the state rounded to FP32, the value the cell kernel gathers). The
// increment dt f / C~ is formed in FP32 from hi and added exactly (update_pair), so the step
// has no FP64 arithmetic; f (and the capacity accumulator) are cleared for the next step.
// Dirichlet dofs take the pair (hd, ld) of T_D - T_ref.
template <int CAP>
__device__ __forceinline__ void update_pair(float& hi, float& lo, float fi, float ci, float ic, bool fixed,
                                            const NodalCap& nc, float hd, float ld, float dt) {
  if (fixed) {
    hi = hd;
    lo = ld;
    return;
  }
  const float2 r = ff_add(make_float2(hi, lo), increment_f32<CAP>(hi, fi, ci, ic, nc, dt));
  hi = r.x;
  lo = r.y;
}

// One element (dof, instance) per thread, any batch size.
template <int CAP>
__global__ void k_update_pair(int64_t n, int B, float* __restrict__ hi, float* __restrict__ lo, float* __restrict__ f,
                              float* __restrict__ Cacc, const float* __restrict__ invC0, const NodalCap nc,
                              const uint8_t* __restrict__ dirichlet, float hd, float ld, float dt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t d = B == 1 ? i : i / B;
  const float fi = f[i];
  f[i] = 0.f;
  float ci = 0.f;
  if (CAP == CAP_QUADRATURE) {
    ci = Cacc[i];
    Cacc[i] = 0.f;
  }
  float h = hi[i], l = lo[i];
  update_pair<CAP>(h, l, fi, ci, CAP == CAP_QUADRATURE ? 0.f : __ldg(&invC0[d]), __ldg(&dirichlet[d]) != 0, nc, hd, ld,
                   dt);
  hi[i] = h;
  lo[i] = l;
}

// Streaming form: each thread takes kUpdGroups groups of four consecutive elements with
// 16-byte accesses (arrays from cudaMalloc are 256-byte aligned; n a multiple of 4) and
// issues every load of its groups before the first use, so that enough bytes are in flight
// per SM. PER_DOF: one instance, a group is four dofs; otherwise B is a multiple of 4 and a
// group is four instances of dof t / B4 (32-bit indices: n_dofs x B < 2^31).
constexpr int kUpdGroups = 2;
template <int CAP, bool PER_DOF>
__global__ void __launch_bounds__(256) k_update_pair_x4(int n4, int B4, float* __restrict__ hi,
                                                         float* __restrict__ lo, float* __restrict__ f,
                                                         float* __restrict__ Cacc, const float* __restrict__ invC0,
                                                         const NodalCap nc, const uint8_t* __restrict__ dirichlet,
                                                         float hd, float ld, float dt) {
  const int t0 = blockIdx.x * (blockDim.x * kUpdGroups) + threadIdx.x;
  float4 f4[kUpdGroups], c4[kUpdGroups], h4[kUpdGroups], l4[kUpdGroups], ic4[kUpdGroups];
  uchar4 fx4[kUpdGroups];
#pragma unroll
  for (int k = 0; k < kUpdGroups; ++k) {
    const int t = t0 + k * blockDim.x;
    if (t >= n4) continue;
    const int i0 = 4 * t;
    f4[k] = __ldcs(reinterpret_cast<const float4*>(f + i0));
    c4[k] = CAP == CAP_QUADRATURE ? __ldcs(reinterpret_cast<const float4*>(Cacc + i0)) : make_float4(0.f, 0.f, 0.f, 0.f);
    h4[k] = __ldcs(reinterpret_cast<const float4*>(hi + i0));
    l4[k] = __ldcs(reinterpret_cast<const float4*>(lo + i0));
    if (PER_DOF) {
      ic4[k] = CAP == CAP_QUADRATURE ? make_float4(0.f, 0.f, 0.f, 0.f) : __ldg(reinterpret_cast<const float4*>(invC0 + i0));
      fx4[k] = __ldg(reinterpret_cast<const uchar4*>(dirichlet + i0));
    } else {
      const int d = t / B4;
      const float ic = CAP == CAP_QUADRATURE ? 0.f : __ldg(&invC0[d]);
      ic4[k] = make_float4(ic, ic, ic, ic);
      const unsigned char fx = __ldg(&dirichlet[d]);
      fx4[k] = make_uchar4(fx, fx, fx, fx);
    }
  }
#pragma unroll
  for (int k = 0; k < kUpdGroups; ++k) {
    const int t = t0 + k * blockDim.x;
    if (t >= n4) continue;
    const int i0 = 4 * t;
    update_pair<CAP>(h4[k].x, l4[k].x, f4[k].x, c4[k].x, ic4[k].x, fx4[k].x != 0, nc, hd, ld, dt);
    update_pair<CAP>(h4[k].y, l4[k].y, f4[k].y, c4[k].y, ic4[k].y, fx4[k].y != 0, nc, hd, ld, dt);
    update_pair<CAP>(h4[k].z, l4[k].z, f4[k].z, c4[k].z, ic4[k].z, fx4[k].z != 0, nc, hd, ld, dt);
    update_pair<CAP>(h4[k].w, l4[k].w, f4[k].w, c4[k].w, ic4[k].w, fx4[k].w != 0, nc, hd, ld, dt);
    __stcs(reinterpret_cast<float4*>(hi + i0), h4[k]);
    __stcs(reinterpret_cast<float4*>(lo + i0), l4[k]);
    __stcs(reinterpret_cast<float4*>(f + i0), make_float4(0.f, 0.f, 0.f, 0.f));
    if (CAP == CAP_QUADRATURE) __stcs(reinterpret_cast<float4*>(Cacc + i0), make_float4(0.f, 0.f, 0.f, 0.f));
  }
}

// hi + lo = T - off (lo may be null: hi only)
__global__ void k_prepare_f32(int64_t n, const double* __restrict__ T, double off, float* __restrict__ hi,
                              float* __restrict__ lo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double t = T[i] - off;
  const float h = d2f_rn(t);
  hi[i] = h;
  if (lo) lo[i] = d2f_rn(t - f2d(h));
}

// T = off + (hi + lo), formed in FP64
__global__ void k_finish_f32(int64_t n, const float* __restrict__ hi, const float* __restrict__ lo, double off,
                             double* __restrict__ T) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) T[i] = off + (f2d(hi[i]) + f2d(lo[i]));
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
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_top * B) return;
  const int face = B == 1 ? i : i / B, inst = i - face * B;
  // face corner relative to the spot (one FP64 subtraction per axis), then the operator
  // precision: the integrand is smooth on the face and its weights sum to the face area
  const double hxd = top_geo[4 * face + 2], hyd = top_geo[4 * face + 3];
  const double ox = top_geo[4 * face + 0] - sp.x, oy = top_geo[4 * face + 1] - sp.y;
  const double r = ls.radius;
  const double gx = fmax(0.0, fmax(ox, -(ox + hxd))), gy = fmax(0.0, fmax(oy, -(oy + hyd)));
  if (gx * gx + gy * gy > 36.0 * r * r) return;
  const R x0 = R(ox), y0 = R(oy), hx = R(hxd), hy = R(hyd);
  const R amp = R(2.0 * ls.eta * power[inst * kMaxSeg + sp.seg] / (kPi * r * r));
  const R ir2 = R(2.0 / (r * r));
  R fe[N][N];
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int k = 0; k < N; ++k) fe[j][k] = R(0);
#pragma unroll
  for (int qy = 0; qy < N; ++qy)
#pragma unroll
    for (int qx = 0; qx < N; ++qx) {
      const R x = x0 + R(Basis<P>::X(qx)) * hx, y = y0 + R(Basis<P>::X(qy)) * hy;
      const R q = amp * expo_r(-(x * x + y * y) * ir2) * R(Basis<P>::W(qx) * Basis<P>::W(qy)) * hx * hy;
#pragma unroll
      for (int j = 0; j < N; ++j)
#pragma unroll
        for (int k = 0; k < N; ++k) fe[j][k] += q * R(Basis<P>::S(qy, j) * Basis<P>::S(qx, k));
    }
  const int cell = top_cell[face];
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int a = k + N * (j + N * P);  // local node (k, j, P) on the top face
      const int d = M.cell_dofs[a * M.n_cells + cell];
      if (d >= 0) {
        atomicAdd(&f[d * B + inst], fe[j][k]);
      } else {
        for (int e = M.con_ptr[-1 - d]; e < M.con_ptr[-d]; ++e)
          atomicAdd(&f[M.con_idx[e] * B + inst], R(M.con_w[e]) * fe[j][k]);
      }
    }
}

// Radiation and evaporation on the active top faces (Eqs. bc_rad_evap, bc_radiation,
// bc_evaporation; Stefan-Boltzmann constant 5.670374419e-8 W m^-2 K^-4): one thread per
// (face, instance) gathers the face's (P+1)^2 node values (hanging ones interpolated from
// their constraint rows), evaluates T at the face's Gauss points, the outward flux
// q = q_rad + q_evap there, and adds -int N_i q dA to the dofs (masters of hanging nodes
// through the same rows).
template <int P, typename R>
__global__ void k_surface_loss(int n_top, int B, const int32_t* __restrict__ top_cell,
                               const double* __restrict__ top_geo, const DevMesh M, const R* __restrict__ x,
                               double T_off, const LossK q, R* __restrict__ f) {
  constexpr int N = P + 1;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_top * B) return;
  const int face = B == 1 ? i : i / B, inst = i - face * B;
  const int cell = top_cell[face];
  const R hx = R(top_geo[4 * face + 2]), hy = R(top_geo[4 * face + 3]);
  R Tf[N * N], fe[N * N];
#pragma unroll
  for (int a = 0; a < N * N; ++a) {
    const int d = M.cell_dofs[(a + N * N * P) * M.n_cells + cell];  // node (a % N, a / N, P)
    R v = R(0);
    if (d >= 0) {
      v = x[(int64_t)d * B + inst];
    } else {
      for (int e = M.con_ptr[-1 - d]; e < M.con_ptr[-d]; ++e)
        v += R(M.con_w[e]) * x[(int64_t)M.con_idx[e] * B + inst];
    }
    Tf[a] = v + R(T_off);
    fe[a] = R(0);
  }
  add_surface_loss<P, R>(q, Tf, hx, hy, fe);
#pragma unroll
  for (int a = 0; a < N * N; ++a) {
    const int d = M.cell_dofs[(a + N * N * P) * M.n_cells + cell];
    if (d >= 0) {
      atomicAdd(&f[(int64_t)d * B + inst], fe[a]);
    } else {
      for (int e = M.con_ptr[-1 - d]; e < M.con_ptr[-d]; ++e)
        atomicAdd(&f[(int64_t)M.con_idx[e] * B + inst], R(M.con_w[e]) * fe[a]);
    }
  }
}

// Transposed linearisation of the surface loss for the adjoint sweep: one thread per (face,
// instance) gathers the face's node values of the state and of the adjoint vector v (hanging
// ones from their constraint rows) and adds -int N_j q'(T_h) v_h dA to g (masters of hanging
// nodes through the same rows).
template <int P, typename R>
__global__ void k_surface_loss_adjoint(int n_top, int B, const int32_t* __restrict__ top_cell,
                                       const double* __restrict__ top_geo, const DevMesh M, const R* __restrict__ x,
                                       double T_off, const R* __restrict__ v, const LossK q, R* __restrict__ g) {
  constexpr int N = P + 1;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_top * B) return;
  const int face = B == 1 ? i : i / B, inst = i - face * B;
  const int cell = top_cell[face];
  const R hx = R(top_geo[4 * face + 2]), hy = R(top_geo[4 * face + 3]);
  R Tf[N * N], vf[N * N], ge[N * N];
#pragma unroll
  for (int a = 0; a < N * N; ++a) {
    const int d = M.cell_dofs[(a + N * N * P) * M.n_cells + cell];  // node (a % N, a / N, P)
    R t = R(0), w = R(0);
    if (d >= 0) {
      t = x[(int64_t)d * B + inst];
      w = v[(int64_t)d * B + inst];
    } else {
      for (int e = M.con_ptr[-1 - d]; e < M.con_ptr[-d]; ++e) {
        t += R(M.con_w[e]) * x[(int64_t)M.con_idx[e] * B + inst];
        w += R(M.con_w[e]) * v[(int64_t)M.con_idx[e] * B + inst];
      }
    }
    Tf[a] = t + R(T_off);
    vf[a] = w;
    ge[a] = R(0);
  }
#pragma unroll
  for (int qy = 0; qy < N; ++qy)
#pragma unroll
    for (int qx = 0; qx < N; ++qx) {
      R T = R(0), vq = R(0);
#pragma unroll
      for (int j = 0; j < N; ++j)
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const R nb = R(Basis<P>::S(qy, j) * Basis<P>::S(qx, k));
          T += nb * Tf[k + N * j];
          vq += nb * vf[k + N * j];
        }
      const R wq = surface_flux_deriv<R>(q, T) * vq * R(Basis<P>::W(qx) * Basis<P>::W(qy)) * hx * hy;
#pragma unroll
      for (int j = 0; j < N; ++j)
#pragma unroll
        for (int k = 0; k < N; ++k) ge[k + N * j] -= wq * R(Basis<P>::S(qy, j) * Basis<P>::S(qx, k));
    }
#pragma unroll
  for (int a = 0; a < N * N; ++a) {
    const int d = M.cell_dofs[(a + N * N * P) * M.n_cells + cell];
    if (d >= 0) {
      atomicAdd(&g[(int64_t)d * B + inst], ge[a]);
    } else {
      for (int e = M.con_ptr[-1 - d]; e < M.con_ptr[-d]; ++e)
        atomicAdd(&g[(int64_t)M.con_idx[e] * B + inst], R(M.con_w[e]) * ge[a]);
    }
  }
}

// Start of the consolidated-fraction history: r_c = 0 in powder cells (material 1), 1 in
// consolidated ones, for every quadrature point and instance ([q][n_cells][batch]).
template <typename R>
__global__ void k_phase_init(int64_t n, int n_cells, int B, const uint8_t* __restrict__ cell_mat, R* __restrict__ rc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int cell = (int)((i / B) % n_cells);
  rc[i] = cell_mat[cell] == 1 ? R(0) : R(1);
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
                             float* __restrict__ inv_f, float* __restrict__ inv_fx,
                             const uint8_t* __restrict__ dirichlet) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double v = 1.0 / c[i];
    inv_d[i] = v;
    inv_f[i] = (float)v;
    if (inv_fx) inv_fx[i] = dirichlet[i] ? -1.f : (float)v;
  }
}

// ---- deterministic reductions -------------------------------------------------------------
// sum_i w_i x_i y_i per instance (w may be null; a mask m zeroes dofs with m != 0). Each
// block reduces a fixed slice in a fixed order; the second pass adds the block partials in
// order, so the result does not depend on scheduling.
// The block count is a constant, not derived from the device, so that the order of the
// additions, and with it every dot product, is the same on any GPU (two blocks per SM of a
// 152-SM GB300).
constexpr int kRedBlocks = 304;

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
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_hang * B) return;
  const int r = B == 1 ? i : i / B, b = i - r * B;
  R s = R(0);
  for (int e = ptr[r]; e < ptr[r + 1]; ++e) s += w[e] * x[idx[e] * B + b];
  out[i] = s;
}

// x_h = P_h x and f_h <- 0, C_h <- 0 (before a cell kernel of the per-cell explicit step)
template <typename R>
__global__ void k_hang_values_zero(int n_hang, int B, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                   const R* __restrict__ w, const R* __restrict__ x, R* __restrict__ out,
                                   R* __restrict__ fh, R* __restrict__ Ch) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_hang * B) return;
  const int r = B == 1 ? i : i / B, b = i - r * B;
  R s = R(0);
  for (int e = ptr[r]; e < ptr[r + 1]; ++e) s += w[e] * x[idx[e] * B + b];
  out[i] = s;
  fh[i] = R(0);
  if (Ch) Ch[i] = R(0);
}

// f += P_h^T f_h, f_h <- 0 (after the cell kernel)
template <typename R>
__global__ void k_hang_distribute(int n_hang, int B, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                  const R* __restrict__ w, R* __restrict__ fh, R* __restrict__ f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_hang * B) return;
  const int r = B == 1 ? i : i / B, b = i - r * B;
  const R v = fh[i];
  if (v == R(0)) return;
  fh[i] = R(0);
  for (int e = ptr[r]; e < ptr[r + 1]; ++e) atomicAdd(&f[idx[e] * B + b], w[e] * v);
}

// ---- CG and Chebyshev recurrences (FP64 vectors; Dirichlet rows held at zero) -----------------
__global__ void k_axpy2(int64_t n, double alpha, const double* __restrict__ p, const double* __restrict__ Ap,
                        double* __restrict__ x, double* __restrict__ r) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] += alpha * p[i];
  r[i] -= alpha * Ap[i];
}

// The same recurrences with the CG scalars read from device memory (alpha = num / den, beta =
// num / den), so that a CG iteration needs no host round trip for them.
__global__ void k_axpy2_dev(int64_t n, const double* __restrict__ num, const double* __restrict__ den,
                            const double* __restrict__ p, const double* __restrict__ Ap, double* __restrict__ x,
                            double* __restrict__ r) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double alpha = num[0] / den[0];
  x[i] += alpha * p[i];
  r[i] -= alpha * Ap[i];
}

__global__ void k_xpby_dev(int64_t n, const double* __restrict__ z, const double* __restrict__ num,
                           const double* __restrict__ den, double* __restrict__ p) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = z[i] + (num[0] / den[0]) * p[i];
}

__global__ void k_xpby(int64_t n, const double* __restrict__ z, double beta, double* __restrict__ p) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = z[i] + beta * p[i];
}

// res = r, d = r / (theta diag), z = d
__global__ void k_cheb_init(int64_t n, const double* __restrict__ r, const double* __restrict__ diag, double inv_theta,
                            double* __restrict__ res, double* __restrict__ d, double* __restrict__ z,
                            const uint8_t* __restrict__ mask) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double ri = mask[i] ? 0.0 : r[i];
  res[i] = ri;
  const double di = ri / diag[i] * inv_theta;
  d[i] = di;
  z[i] = di;
}

// res -= A d; d = a d + b res / diag; z += d
__global__ void k_cheb_update(int64_t n, const double* __restrict__ Ad, double* __restrict__ res, double* __restrict__ d,
                              double* __restrict__ z, const double* __restrict__ diag, double a, double b,
                              const uint8_t* __restrict__ mask) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (mask[i]) {
    res[i] = 0.0;
    d[i] = 0.0;
    return;
  }
  const double ri = res[i] - Ad[i];
  res[i] = ri;
  const double di = a * d[i] + b * ri / diag[i];
  d[i] = di;
  z[i] += di;
}

__global__ void k_jacobi(int64_t n, const double* __restrict__ r, const double* __restrict__ diag,
                         double* __restrict__ z, const uint8_t* __restrict__ mask) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = mask[i] ? 0.0 : r[i] / diag[i];
}

// y = -y on free rows, 0 on Dirichlet rows
__global__ void k_neg_masked(int64_t n, double* __restrict__ y, const uint8_t* __restrict__ mask) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = mask[i] ? 0.0 : -y[i];
}

__global__ void k_add(int64_t n, double* __restrict__ T, const double* __restrict__ x) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) T[i] += x[i];
}

// ---- adjoint sweep ----------------------------------------------------------------------------
// v = lambda / C~, mu = lambda f / C~^2, q1 = f_diff / C~, q2 = f_vol / C~ on free dofs
__global__ void k_adj_prepare(int n, int B, const double* __restrict__ lam, const double* __restrict__ fd,
                              const double* __restrict__ fv, const double* __restrict__ fre,
                              const double* __restrict__ Cm, const uint8_t* __restrict__ dir, double* __restrict__ v,
                              double* __restrict__ mu, double* __restrict__ q1, double* __restrict__ q2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * B) return;
  const int d = B == 1 ? i : i / B;
  if (dir[d]) {
    v[i] = mu[i] = q1[i] = q2[i] = 0.0;
    return;
  }
  const double ic = 1.0 / Cm[i];
  v[i] = lam[i] * ic;
  mu[i] = lam[i] * (fd[i] + fv[i] + (fre ? fre[i] : 0.0)) * ic * ic;
  q1[i] = fd[i] * ic;
  q2[i] = fv[i] * ic;
}

__device__ __forceinline__ double power_of(double t, double p, int ip) {
  if (ip <= 0) return pow(t, p);
  double r = 1.0, b = t;
  for (int e = ip; e; e >>= 1) {
    if (e & 1) r *= b;
    b *= b;
  }
  return r;
}

// part[blk][b] = sum over a slice of the surface list of w_k T[idx_k][b]^p
__global__ void k_pnorm_partial(int ns, int B, const int32_t* __restrict__ sidx, const double* __restrict__ sw,
                                const double* __restrict__ T, double p, int ip, double* __restrict__ part) {
  __shared__ double sh[kBS];
  const int per = (ns + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * per, hi = min(ns, lo + per);
  for (int b = 0; b < B; ++b) {
    double acc = 0.0;
    for (int k = lo + threadIdx.x; k < hi; k += blockDim.x) acc += sw[k] * power_of(T[sidx[k] * B + b], p, ip);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x * B + b] = sh[0];
    __syncthreads();
  }
}

// M_b = (S_b / W)^(1/p); J_b += (M_b - T_t)^2 / N when accumulating;
// coef_b = 2 (M_b - T_t) / N * M_b^(1-p) / W  (dJ/dT_i = coef_b w_i T_i^(p-1))
__global__ void k_objective(int B, int nblk, const double* __restrict__ part, double W, double p, double Tt,
                            double invN, int accumulate, double* __restrict__ J, double* __restrict__ coef) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double S = 0.0;
  for (int k = 0; k < nblk; ++k) S += part[k * B + b];
  const double M = pow(S / W, 1.0 / p);
  if (accumulate) J[b] += (M - Tt) * (M - Tt) * invN;
  coef[b] = 2.0 * (M - Tt) * invN * pow(M, 1.0 - p) / W;
}

// lambda += coef_b w_k T^(p-1) on the surface dofs (not on Dirichlet dofs)
__global__ void k_lambda_objective(int ns, int B, const int32_t* __restrict__ sidx, const double* __restrict__ sw,
                                   const double* __restrict__ T, double p, int ip, const double* __restrict__ coef,
                                   const uint8_t* __restrict__ dir, double* __restrict__ lam) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ns * B) return;
  const int k = B == 1 ? i : i / B, b = i - k * B;
  const int d = sidx[k];
  if (dir[d]) return;
  lam[d * B + b] += coef[b] * sw[k] * power_of(T[d * B + b], p - 1.0, ip > 0 ? ip - 1 : 0);
}

// lambda_k = lambda_{k+1} + dt (g - [nodal] mu C0 c_app'(T)/c) on free dofs, 0 on Dirichlet
template <typename R, bool NODAL>
__global__ void k_lambda_update(int n, int B, double* __restrict__ lam, R* __restrict__ g,
                                const double* __restrict__ mu, const double* __restrict__ C0,
                                const double* __restrict__ T, const NodalCap nc, const uint8_t* __restrict__ dir,
                                double dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * B) return;
  const int d = B == 1 ? i : i / B;
  double gi = (double)g[i];
  g[i] = R(0);
  if (dir[d]) {
    lam[i] = 0.0;
    return;
  }
  if (NODAL) {
    const double z = (T[i] - nc.Tm) * nc.inv_sigma;
    gi -= mu[i] * C0[d] * nc.lat_ratio * (-z * nc.inv_sigma) * exp(-0.5 * z * z);
  }
  lam[i] += dt * gi;
}

// grad[b][seg] += dt d2[b] / P[b][seg];  grad[b][nseg] += dt d1[b] / s_b
__global__ void k_grad_accum(int B, int nseg, int seg, const double* __restrict__ d1, const double* __restrict__ d2,
                             const double* __restrict__ s, const double* __restrict__ power, double dt,
                             double* __restrict__ grad) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  grad[b * (nseg + 1) + nseg] += dt * d1[b] / s[b];
  if (seg >= 0) grad[b * (nseg + 1) + seg] += dt * d2[b] / power[b * kMaxSeg + seg];
}

// w_i += int_top N_i dA over top faces ((P+1)^2 Gauss points), through the constraints
template <int P>
__global__ void k_surface_weights(int n_top, const int32_t* __restrict__ top_cell, const double* __restrict__ top_geo,
                                  const DevMesh M, double* __restrict__ w) {
  constexpr int N = P + 1;
  const int face = blockIdx.x * blockDim.x + threadIdx.x;
  if (face >= n_top) return;
  const double area = top_geo[4 * face + 2] * top_geo[4 * face + 3];
  const int cell = top_cell[face];
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int k = 0; k < N; ++k) {
      double wj = 0.0, wk = 0.0;
#pragma unroll
      for (int q = 0; q < N; ++q) {
        wj += Basis<P>::W(q) * Basis<P>::S(q, j);
        wk += Basis<P>::W(q) * Basis<P>::S(q, k);
      }
      const double val = wj * wk * area;
      const int d = M.cell_dofs[(k + N * (j + N * P)) * M.n_cells + cell];
      if (d >= 0) {
        atomicAdd(&w[d], val);
      } else {
        for (int e = M.con_ptr[-1 - d]; e < M.con_ptr[-d]; ++e) atomicAdd(&w[M.con_idx[e]], M.con_w[e] * val);
      }
    }
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

template <int CAP>
cudaError_t update_pair_cap(int64_t n_dofs, int B, float* hi, float* lo, float* f, float* Cacc, const float* invC0,
                            const NodalCap& nc, const uint8_t* dirichlet, float hd, float ld, float dt, cudaStream_t s) {
  const int64_t n = n_dofs * B;
  if (B % 4 == 0 || (B == 1 && n % 4 == 0)) {
    const int n4 = (int)(n / 4);
    const unsigned grid = grid_for(n4, kBS * kUpdGroups);
    if (B == 1)
      k_update_pair_x4<CAP, true><<<grid, kBS, 0, s>>>(n4, 1, hi, lo, f, Cacc, invC0, nc, dirichlet, hd, ld, dt);
    else
      k_update_pair_x4<CAP, false><<<grid, kBS, 0, s>>>(n4, B / 4, hi, lo, f, Cacc, invC0, nc, dirichlet, hd, ld, dt);
  } else {
    k_update_pair<CAP><<<grid_for(n), kBS, 0, s>>>(n, B, hi, lo, f, Cacc, invC0, nc, dirichlet, hd, ld, dt);
  }
  return cudaGetLastError();
}

cudaError_t launch_update_f32(int cap, int64_t n_dofs, int B, float* hi, float* lo, float* f, float* Cacc,
                              const float* invC0, const NodalCap& nc, const uint8_t* dirichlet, float2 x_dir, float dt,
                              cudaStream_t s) {
  if (n_dofs * B == 0) return cudaSuccess;
  if (cap == CAP_QUADRATURE)
    return update_pair_cap<CAP_QUADRATURE>(n_dofs, B, hi, lo, f, Cacc, invC0, nc, dirichlet, x_dir.x, x_dir.y, dt, s);
  if (cap == CAP_NODAL)
    return update_pair_cap<CAP_NODAL>(n_dofs, B, hi, lo, f, Cacc, invC0, nc, dirichlet, x_dir.x, x_dir.y, dt, s);
  return update_pair_cap<CAP_CONST>(n_dofs, B, hi, lo, f, Cacc, invC0, nc, dirichlet, x_dir.x, x_dir.y, dt, s);
}

cudaError_t launch_hang_values_zero(bool f32, const DevMesh& M, const void* x, void* out, void* fh, void* Ch,
                                    cudaStream_t s) {
  const int64_t n = (int64_t)M.n_hang * M.batch;
  if (n == 0) return cudaSuccess;
  if (f32) k_hang_values_zero<float><<<grid_for(n), kBS, 0, s>>>(M.n_hang, M.batch, M.con_ptr, M.con_idx, M.con_wf, (const float*)x, (float*)out, (float*)fh, (float*)Ch);
  else k_hang_values_zero<double><<<grid_for(n), kBS, 0, s>>>(M.n_hang, M.batch, M.con_ptr, M.con_idx, M.con_w, (const double*)x, (double*)out, (double*)fh, (double*)Ch);
  return cudaGetLastError();
}

cudaError_t launch_capacity_nodal(int64_t n_dofs, int B, const double* C0, const double* T, const NodalCap& nc,
                                  double* C_out, cudaStream_t s) {
  const int64_t n = n_dofs * B;
  if (n == 0) return cudaSuccess;
  k_capacity_nodal<<<grid_for(n), kBS, 0, s>>>(n, B, C0, T, nc, C_out);
  return cudaGetLastError();
}

cudaError_t launch_prepare_f32(int64_t n, const double* T, double off, float* hi, float* lo, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_prepare_f32<<<grid_for(n), kBS, 0, s>>>(n, T, off, hi, lo);
  return cudaGetLastError();
}

cudaError_t launch_finish_f32(int64_t n, const float* hi, const float* lo, double off, double* T, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_finish_f32<<<grid_for(n), kBS, 0, s>>>(n, hi, lo, off, T);
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
      if (f32) k_laser_volume<1, float><<<grid_for(n, 128), 128, 0, s>>>(M.n_cells, B, ls.cell_lo, M.cell_level, ls.level_h, M, ls.k, power, sp, (float*)f);
      else k_laser_volume<1, double><<<grid_for(n, 128), 128, 0, s>>>(M.n_cells, B, ls.cell_lo, M.cell_level, ls.level_h, M, ls.k, power, sp, (double*)f);
    } else {
      if (f32) k_laser_volume<2, float><<<grid_for(n, 128), 128, 0, s>>>(M.n_cells, B, ls.cell_lo, M.cell_level, ls.level_h, M, ls.k, power, sp, (float*)f);
      else k_laser_volume<2, double><<<grid_for(n, 128), 128, 0, s>>>(M.n_cells, B, ls.cell_lo, M.cell_level, ls.level_h, M, ls.k, power, sp, (double*)f);
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

cudaError_t launch_phase_init(bool f32, int nq, const DevMesh& M, void* rc, cudaStream_t s) {
  const int64_t n = (int64_t)nq * M.n_cells * M.batch;
  if (n == 0) return cudaSuccess;
  if (f32) k_phase_init<float><<<grid_for(n), kBS, 0, s>>>(n, M.n_cells, M.batch, M.cell_mat, (float*)rc);
  else k_phase_init<double><<<grid_for(n), kBS, 0, s>>>(n, M.n_cells, M.batch, M.cell_mat, (double*)rc);
  return cudaGetLastError();
}

cudaError_t launch_surface_loss(int degree, bool f32, const LaserSetup& ls, const DevMesh& M, const void* x,
                                double T_off, const LossK& q, void* f, cudaStream_t s) {
  const int B = M.batch;
  const int64_t n = (int64_t)ls.n_top * B;
  if (n == 0) return cudaSuccess;
  const unsigned grid = grid_for(n, 128);
  if (degree == 1) {
    if (f32) k_surface_loss<1, float><<<grid, 128, 0, s>>>(ls.n_top, B, ls.top_cell, ls.top_geo, M, (const float*)x, T_off, q, (float*)f);
    else k_surface_loss<1, double><<<grid, 128, 0, s>>>(ls.n_top, B, ls.top_cell, ls.top_geo, M, (const double*)x, T_off, q, (double*)f);
  } else {
    if (f32) k_surface_loss<2, float><<<grid, 128, 0, s>>>(ls.n_top, B, ls.top_cell, ls.top_geo, M, (const float*)x, T_off, q, (float*)f);
    else k_surface_loss<2, double><<<grid, 128, 0, s>>>(ls.n_top, B, ls.top_cell, ls.top_geo, M, (const double*)x, T_off, q, (double*)f);
  }
  return cudaGetLastError();
}

cudaError_t launch_surface_loss_adjoint(int degree, bool f32, const LaserSetup& ls, const DevMesh& M, const void* x,
                                        double T_off, const void* v, const LossK& q, void* g, cudaStream_t s) {
  const int64_t n = (int64_t)ls.n_top * M.batch;
  if (n == 0) return cudaSuccess;
  const unsigned grid = grid_for(n, 128);
  if (degree == 1) {
    if (f32)
      k_surface_loss_adjoint<1, float><<<grid, 128, 0, s>>>(ls.n_top, M.batch, ls.top_cell, ls.top_geo, M,
                                                            (const float*)x, T_off, (const float*)v, q, (float*)g);
    else
      k_surface_loss_adjoint<1, double><<<grid, 128, 0, s>>>(ls.n_top, M.batch, ls.top_cell, ls.top_geo, M,
                                                             (const double*)x, T_off, (const double*)v, q, (double*)g);
  } else {
    if (f32)
      k_surface_loss_adjoint<2, float><<<grid, 128, 0, s>>>(ls.n_top, M.batch, ls.top_cell, ls.top_geo, M,
                                                            (const float*)x, T_off, (const float*)v, q, (float*)g);
    else
      k_surface_loss_adjoint<2, double><<<grid, 128, 0, s>>>(ls.n_top, M.batch, ls.top_cell, ls.top_geo, M,
                                                             (const double*)x, T_off, (const double*)v, q, (double*)g);
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

cudaError_t launch_reciprocal(int64_t n, const double* c, double* inv_d, float* inv_f, float* inv_fx,
                              const uint8_t* dirichlet, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (inv_fx && !dirichlet) return cudaErrorInvalidValue;
  k_reciprocal<<<grid_for(n), kBS, 0, s>>>(n, c, inv_d, inv_f, inv_fx, dirichlet);
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

cudaError_t launch_axpy2(int64_t n, double alpha, const double* p, const double* Ap, double* x, double* r,
                         cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_axpy2<<<grid_for(n), kBS, 0, s>>>(n, alpha, p, Ap, x, r);
  return cudaGetLastError();
}
cudaError_t launch_axpy2_dev(int64_t n, const double* num, const double* den, const double* p, const double* Ap,
                             double* x, double* r, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_axpy2_dev<<<grid_for(n), kBS, 0, s>>>(n, num, den, p, Ap, x, r);
  return cudaGetLastError();
}
cudaError_t launch_xpby_dev(int64_t n, const double* z, const double* num, const double* den, double* p,
                            cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_xpby_dev<<<grid_for(n), kBS, 0, s>>>(n, z, num, den, p);
  return cudaGetLastError();
}
cudaError_t launch_xpby(int64_t n, const double* z, double beta, double* p, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_xpby<<<grid_for(n), kBS, 0, s>>>(n, z, beta, p);
  return cudaGetLastError();
}
cudaError_t launch_cheb_init(int64_t n, const double* r, const double* diag, double inv_theta, double* res, double* d,
                             double* z, const uint8_t* mask, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_cheb_init<<<grid_for(n), kBS, 0, s>>>(n, r, diag, inv_theta, res, d, z, mask);
  return cudaGetLastError();
}
cudaError_t launch_cheb_update(int64_t n, const double* Ad, double* res, double* d, double* z, const double* diag,
                               double a, double b, const uint8_t* mask, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_cheb_update<<<grid_for(n), kBS, 0, s>>>(n, Ad, res, d, z, diag, a, b, mask);
  return cudaGetLastError();
}
cudaError_t launch_jacobi(int64_t n, const double* r, const double* diag, double* z, const uint8_t* mask,
                          cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_jacobi<<<grid_for(n), kBS, 0, s>>>(n, r, diag, z, mask);
  return cudaGetLastError();
}
cudaError_t launch_neg_masked(int64_t n, double* y, const uint8_t* mask, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_neg_masked<<<grid_for(n), kBS, 0, s>>>(n, y, mask);
  return cudaGetLastError();
}
cudaError_t launch_add(int64_t n, double* T, const double* x, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_add<<<grid_for(n), kBS, 0, s>>>(n, T, x);
  return cudaGetLastError();
}

cudaError_t launch_adj_prepare(int n, int B, const double* lam, const double* fd, const double* fv, const double* fre,
                               const double* Cm, const uint8_t* dir, double* v, double* mu, double* q1, double* q2,
                               cudaStream_t s) {
  if (n * B == 0) return cudaSuccess;
  k_adj_prepare<<<grid_for((int64_t)n * B), kBS, 0, s>>>(n, B, lam, fd, fv, fre, Cm, dir, v, mu, q1, q2);
  return cudaGetLastError();
}

cudaError_t launch_objective(int ns, int B, const int32_t* sidx, const double* sw, const double* T, double W, double p,
                             double Tt, double invN, int accumulate, double* part, double* J, double* coef,
                             cudaStream_t s) {
  const int ip = (p == (double)(int)p && p >= 1 && p <= 64) ? (int)p : 0;
  k_pnorm_partial<<<kRedBlocks, kBS, 0, s>>>(ns, B, sidx, sw, T, p, ip, part);
  k_objective<<<(B + 63) / 64, 64, 0, s>>>(B, kRedBlocks, part, W, p, Tt, invN, accumulate, J, coef);
  return cudaGetLastError();
}

cudaError_t launch_lambda_objective(int ns, int B, const int32_t* sidx, const double* sw, const double* T, double p,
                                    const double* coef, const uint8_t* dir, double* lam, cudaStream_t s) {
  if (ns * B == 0) return cudaSuccess;
  const int ip = (p == (double)(int)p && p >= 1 && p <= 64) ? (int)p : 0;
  k_lambda_objective<<<grid_for((int64_t)ns * B), kBS, 0, s>>>(ns, B, sidx, sw, T, p, ip, coef, dir, lam);
  return cudaGetLastError();
}

cudaError_t launch_lambda_update(bool f32, bool nodal, int n, int B, double* lam, void* g, const double* mu,
                                 const double* C0, const double* T, const NodalCap& nc, const uint8_t* dir, double dt,
                                 cudaStream_t s) {
  if (n * B == 0) return cudaSuccess;
  const unsigned gr = grid_for((int64_t)n * B);
  if (f32) {
    if (nodal) k_lambda_update<float, true><<<gr, kBS, 0, s>>>(n, B, lam, (float*)g, mu, C0, T, nc, dir, dt);
    else k_lambda_update<float, false><<<gr, kBS, 0, s>>>(n, B, lam, (float*)g, mu, C0, T, nc, dir, dt);
  } else {
    if (nodal) k_lambda_update<double, true><<<gr, kBS, 0, s>>>(n, B, lam, (double*)g, mu, C0, T, nc, dir, dt);
    else k_lambda_update<double, false><<<gr, kBS, 0, s>>>(n, B, lam, (double*)g, mu, C0, T, nc, dir, dt);
  }
  return cudaGetLastError();
}

cudaError_t launch_grad_accum(int B, int nseg, int seg, const double* d1, const double* d2, const double* sc,
                              const double* power, double dt, double* grad, cudaStream_t s) {
  k_grad_accum<<<(B + 63) / 64, 64, 0, s>>>(B, nseg, seg, d1, d2, sc, power, dt, grad);
  return cudaGetLastError();
}

cudaError_t launch_surface_weights(int degree, int n_top, const int32_t* top_cell, const double* top_geo,
                                   const DevMesh& M, double* w, cudaStream_t s) {
  if (n_top == 0) return cudaSuccess;
  if (degree == 1) k_surface_weights<1><<<grid_for(n_top, 128), 128, 0, s>>>(n_top, top_cell, top_geo, M, w);
  else k_surface_weights<2><<<grid_for(n_top, 128), 128, 0, s>>>(n_top, top_cell, top_geo, M, w);
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
