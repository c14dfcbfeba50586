// Internal device structures and kernel launchers of the library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace pbf {

constexpr int kMaxLevels = 13;
constexpr int kMaxSeg = 64;
constexpr double kPi = 3.14159265358979323846;

// 1D tables on [0,1] for Q_P with P+1 Gauss-Legendre points x_q:
//   S(q,i) = N_i(x_q), nodal Lagrange basis (nodes i/P) at the Gauss points
//   D(q,j) = L_j'(x_q), derivative of the Lagrange polynomial through the Gauss points
//            (collocation derivative: gradients at the points from values at the points)
//   W(q)   = Gauss weight, X(q) = Gauss point
template <int P>
struct Basis;

template <>
struct Basis<1> {
  static constexpr int N = 2;
  __host__ __device__ static constexpr double X(int q) { return q == 0 ? 0.21132486540518711 : 0.78867513459481287; }
  __host__ __device__ static constexpr double W(int) { return 0.5; }
  __host__ __device__ static constexpr double S(int q, int i) {
    return (q == i) ? 0.78867513459481287 : 0.21132486540518711;
  }
  __host__ __device__ static constexpr double D(int, int j) {
    return j == 0 ? -1.7320508075688772 : 1.7320508075688772;
  }
};

template <>
struct Basis<2> {
  static constexpr int N = 3;
  __host__ __device__ static constexpr double X(int q) {
    return q == 0 ? 0.11270166537925831 : (q == 1 ? 0.5 : 0.8872983346207417);
  }
  __host__ __device__ static constexpr double W(int q) {
    return q == 1 ? 0.44444444444444442 : 0.27777777777777779;
  }
  __host__ __device__ static constexpr double S(int q, int i) {
    return q == 1 ? (i == 1 ? 1.0 : 0.0)
                  : (i == 1 ? 0.40000000000000002 : ((q == i) ? 0.68729833462074164 : -0.087298334620741685));
  }
  __host__ __device__ static constexpr double D(int q, int j) {
    return q == 0 ? (j == 0 ? -3.872983346207417 : (j == 1 ? 5.1639777949432224 : -1.2909944487358056))
         : q == 1 ? (j == 0 ? -1.2909944487358056 : (j == 1 ? 0.0 : 1.2909944487358056))
                  : (j == 0 ? 1.2909944487358056 : (j == 1 ? -5.1639777949432224 : 3.872983346207417));
  }
};

// Exact IEEE-754 conversions by integer operations. On this GPU the FP64 and the
// FP64<->FP32 conversion pipes run at about 1/60 of the FP32 rate, so the FP32-operator path
// converts with a handful of 32-bit integer instructions instead.
//
// d2f_rn: binary64 -> binary32, round to nearest, ties to even. Values whose magnitude is
// below the smallest normal binary32 (2^-126) flush to a signed zero; inputs must be finite
// with magnitude below 2^128 (temperatures and their increments are).
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned lo = (unsigned)__double2loint(x), hi = (unsigned)__double2hiint(x);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;  // rebias 1023 -> 127
  if (e <= 0) return __uint_as_float(sign);
  const unsigned mf = ((hi & 0xFFFFFu) << 3) | (lo >> 29);  // top 23 of 52 mantissa bits
  const unsigned rem = lo & 0x1FFFFFFFu;                    // 29 discarded bits
  unsigned out = sign | ((unsigned)e << 23) | mf;
  out += (rem > 0x10000000u) | ((rem == 0x10000000u) & (mf & 1u));  // carry may bump e
  return __uint_as_float(out);
}

// f2d: binary32 -> binary64, exact (subnormal inputs flush to a signed zero).
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  if (e == 0xFFu) return (double)f;  // inf / nan keep their meaning
  if (e == 0u) return __hiloint2double((int)sign, 0);
  return __hiloint2double((int)(sign | ((e + 896u) << 20) | (m >> 3)), (int)(m << 29));
}

// Mesh tables on the device (one copy shared by all instances of a batch).
struct DevMesh {
  int n_cells = 0, npc = 0, n_dofs = 0, n_hang = 0, batch = 1;
  const int32_t* cell_dofs = nullptr;  // [npc][n_cells], dof or -1-row
  const uint8_t* cell_level = nullptr;
  const uint8_t* cell_mat = nullptr;
  const int32_t* con_ptr = nullptr;
  const int32_t* con_idx = nullptr;
  const double* con_w = nullptr;
  const float* con_wf = nullptr;
  const uint8_t* dirichlet = nullptr;
  const uint8_t* cell_top = nullptr;  // 1 when the cell has an active top face
  const double* cell_lo = nullptr;    // [n_cells][3] lower corner
  const float* cell_lof = nullptr;    // the same in FP32
};

// Per-level geometry of axis-aligned cells (diagonal Jacobian J = diag(h)), precomputed on
// the host in the kernel's precision.
template <typename R>
struct GeoR {
  R detJ[kMaxLevels];
  R ih2[kMaxLevels][3];  // 1 / h_d^2
  R h[kMaxLevels][3];    // h_d
};

// Surface laser evaluated inside the cell kernel on top faces (spot from the host per step).
struct LaserInline {
  int on = 0;
  int seg = -1;
  double sx = 0.0, sy = 0.0;     // spot position
  double amp = 0.0;              // 2 eta / (pi r^2) (times the segment power per instance)
  double ir2 = 0.0;              // 2 / r^2
  double cut2 = 0.0;             // faces farther than sqrt(cut2) from the spot are skipped
  const double* power = nullptr; // [batch][kMaxSeg]
  const float* powerf = nullptr; // the same in FP32
};

// Material constants precomputed on the host in the kernel's precision.
template <typename R>
struct MatR {
  R rho, c, lat_norm, tm_off, inv_sigma;  // c_app = c + lat_norm exp(-((v + tm_off) inv_sigma)^2/2)
  R k0, dk, tk_off, inv_dT;               // k = k0 + dk clamp((v + tk_off) inv_dT, 0, 1)
  R powder_scale;
  R m_impl;                               // rho c / dt of the implicit operator
};

// Phase-dependent conductivity with history (Sec. 2, Eqs. liquid_fraction ..
// material_parameter_interp) in the kernel's precision: g = clamp((v + t_off) inv_dT, 0, 1)
// with v = T - T_ref, r_c = max(stored r_c, g), k = k_p + r_c dks + g dkm
// (dks = k_s - k_p, dkm = k_m - k_s).
template <typename R>
struct PhaseR {
  R t_off, inv_dT, kp, dks, dkm;
};

struct LaserK {
  int n_seg = 0;
  int volumetric = 0;
  double seg[kMaxSeg][6];
  double eta, radius, h_powder, z_top;
};

// Spot of the laser at one time: position and active segment (-1: no segment active).
struct Spot {
  double x = 0.0, y = 0.0;
  int seg = -1;
};

// The spot at time t: the first segment with t0 <= t < t1, moving linearly from (x0, y0) to
// (x1, y1). Host and device evaluate it with the same correctly rounded FP64 operations.
__host__ __device__ inline Spot spot_at(const LaserK& k, double t) {
  Spot sp;
  for (int i = 0; i < k.n_seg; ++i) {
    const double* g = k.seg[i];
    if (t >= g[4] && t < g[5]) {
#ifdef __CUDA_ARCH__
      const double a = __ddiv_rn(__dsub_rn(t, g[4]), __dsub_rn(g[5], g[4]));
      sp.x = __dadd_rn(g[0], __dmul_rn(__dsub_rn(g[2], g[0]), a));
      sp.y = __dadd_rn(g[1], __dmul_rn(__dsub_rn(g[3], g[1]), a));
#else
      const double a = (t - g[4]) / (g[5] - g[4]);
      sp.x = g[0] + (g[2] - g[0]) * a;
      sp.y = g[1] + (g[3] - g[1]) * a;
#endif
      sp.seg = i;
      return sp;
    }
  }
  return sp;
}

// ---- launchers (kernels_cell.cu) --------------------------------------------------------
enum CellMode {
  MODE_RESIDUAL = 0,  // f += f_diff(T), C += lumped capacity (when C != null)
  MODE_CAPACITY = 1,  // C += lumped capacity only
  MODE_STIFF = 2,     // f += K x (linear k0, positive), x without offset
  MODE_IMPLICIT = 3,  // f += (C_consistent/dt + K) x, linear material
};

struct CellLaunch {
  DevMesh mesh;
  GeoR<float> gf;
  GeoR<double> gd;
  MatR<float> mf;
  MatR<double> md;
  int nonlin_k = 0, latent = 0;
  double offset = 0.0;              // subtracted from x before rounding (T_ref or 0)
  const float* k_scale_f = nullptr;  // [batch]
  const double* k_scale_d = nullptr; // [batch]
  const double* x = nullptr;        // input field [n_dofs][batch] (FP64 operator)
  const double* xh = nullptr;       // its values at hanging nodes [n_hang][batch]
  const float* xf = nullptr;        // input field rounded to FP32 (FP32 operator)
  const float* xfh = nullptr;       // FP32 values at hanging nodes
  // adjoint: v = lambda / C~ and mu = lambda f / C~^2 (quadrature-point capacity only)
  const double* v = nullptr;
  const double* vh = nullptr;
  const float* vf = nullptr;
  const float* vfh = nullptr;
  const double* mu = nullptr;
  const double* muh = nullptr;
  const float* muf = nullptr;
  const float* mufh = nullptr;
  int degree = 1;
  int f32 = 0;
  int variant = 0;  // launch shape of the FP32 residual kernel (see kCellVariants)
  LaserInline las;
  // phase-dependent conductivity (residual mode): r_c per quadrature point, [q][n_cells][batch]
  // in the context's precision (rc_f32: FP32 elements, else FP64; a launch's arithmetic may
  // differ, as in the FP64 Newton residual of an FP32 context), read from rc_in and stored to
  // rc_out (null: read only); kernels access it through rc_load / rc_store only
  int phase = 0;
  int rc_f32 = 0;
  PhaseR<float> phf;
  PhaseR<double> phd;
  const void* rc_in = nullptr;
  void* rc_out = nullptr;
  // adjoint sweep with the phase model: the history's adjoint divided by dt, [q][n_cells][batch]
  // in the operator precision, read and replaced by the adjoint kernel
  void* sig = nullptr;
};

// Element j of the phase model's history, in the element type the context keeps it in.
template <typename R>
__device__ __forceinline__ R rc_load(const CellLaunch& L, int64_t j) {
  return L.rc_f32 ? R(static_cast<const float*>(L.rc_in)[j]) : R(static_cast<const double*>(L.rc_in)[j]);
}
template <typename R>
__device__ __forceinline__ void rc_store(const CellLaunch& L, int64_t j, R v) {
  if (L.rc_f32) static_cast<float*>(L.rc_out)[j] = float(v);
  else static_cast<double*>(L.rc_out)[j] = double(v);
}

// Explicit-step shapes the autotuner chooses from for the FP32 operator. 0-3: the per-cell
// residual kernel {threads per block, minimum resident blocks per SM} = {128, 1}, {128, 5},
// {128, 6}, {64, 10} (the second bounds registers per thread), followed by the update kernel;
// 4: the fused step kernel (one instance, constant or nodal capacity), 5: the same launched
// with programmatic dependent launch, 6: all steps in one persistent cooperative launch,
// 7-9: the lean fused step kernel (tables through L1) compiled for 14, 12 and 10 resident
// blocks per SM. Residual-only launches of shapes 4-9 use shape 1.
constexpr int kCellVariants = 10;

template <typename R>
__host__ __device__ inline const GeoR<R>& geo_of(const CellLaunch& L);
template <>
__host__ __device__ inline const GeoR<float>& geo_of<float>(const CellLaunch& L) { return L.gf; }
template <>
__host__ __device__ inline const GeoR<double>& geo_of<double>(const CellLaunch& L) { return L.gd; }
template <typename R>
__host__ __device__ inline const MatR<R>& mat_of(const CellLaunch& L);
template <>
__host__ __device__ inline const MatR<float>& mat_of<float>(const CellLaunch& L) { return L.mf; }
template <>
__host__ __device__ inline const MatR<double>& mat_of<double>(const CellLaunch& L) { return L.md; }
template <typename R>
__host__ __device__ inline const R* kscale_of(const CellLaunch& L);
template <>
__host__ __device__ inline const float* kscale_of<float>(const CellLaunch& L) { return L.k_scale_f; }
template <>
__host__ __device__ inline const double* kscale_of<double>(const CellLaunch& L) { return L.k_scale_d; }

// f/C: accumulators over dofs; fh/Ch: accumulators over hanging nodes (distributed to their
// masters afterwards by launch_hang_distribute). C/Ch may be null.
cudaError_t launch_cell(const CellLaunch& L, void* f, void* fh, void* C, void* Ch, int mode, cudaStream_t s);

// implicit-operator diagonal: diag += diag(P^T A_e P) over cells (FP64 output)
cudaError_t launch_diag(const CellLaunch& L, double* diag, cudaStream_t s);

// adjoint cell kernel at state x: g += (df_diff/dT)^T v - (dC~/dT)^T mu, the capacity term only
// for the quadrature-point capacity (qp_capacity); g/gh accumulate over dofs / hanging nodes
cudaError_t launch_adjoint(const CellLaunch& L, bool qp_capacity, void* g, void* gh, cudaStream_t s);

}  // namespace pbf
