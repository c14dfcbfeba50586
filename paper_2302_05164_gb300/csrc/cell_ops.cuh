// Device building blocks of the sum-factorised cell operator (paper Sec. 4.2): 1D
// interpolation / collocation-derivative contractions with compile-time Gauss tables, the
// quadrature weights, the branch-free material helpers and the surface laser on top faces.
// Shared by the per-cell kernels (kernels_cell.cu) and the fused step kernel (kernels_step.cu).
#pragma once

#include "internal.cuh"

namespace pbf {

template <int N>
__device__ __forceinline__ constexpr int lin(int dir, int a, int b, int i) {
  return dir == 0 ? i + N * (a + N * b) : (dir == 1 ? a + N * (i + N * b) : a + N * (b + N * i));
}

template <int P, int WHICH>
__device__ __forceinline__ constexpr double coef(int q, int i) {
  return WHICH == 0 ? Basis<P>::S(q, i) : Basis<P>::D(q, i);
}

// out[line, q] (+)= sum_i M(q, i) in[line, i]   along direction DIR; TR uses M(i, q).
template <int P, int WHICH, int DIR, bool TR, bool ADD, typename R>
__device__ __forceinline__ void apply1d(const R* in, R* out) {
  constexpr int N = P + 1;
#pragma unroll
  for (int b = 0; b < N; ++b)
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
      for (int q = 0; q < N; ++q) {
        R s = ADD ? out[lin<N>(DIR, a, b, q)] : R(0);
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const double m = TR ? coef<P, WHICH>(i, q) : coef<P, WHICH>(q, i);
          if (m != 0.0) s = s + R(m) * in[lin<N>(DIR, a, b, i)];
        }
        out[lin<N>(DIR, a, b, q)] = s;
      }
}

template <int P, typename R>
__device__ __forceinline__ void values_at_qp(const R* u, R* v) {
  constexpr int NP = (P + 1) * (P + 1) * (P + 1);
  R t[NP], w[NP];
  apply1d<P, 0, 0, false, false>(u, t);
  apply1d<P, 0, 1, false, false>(t, w);
  apply1d<P, 0, 2, false, false>(w, v);
}

template <int P, typename R>
__device__ __forceinline__ void integrate_values(const R* r, R* fe) {
  constexpr int NP = (P + 1) * (P + 1) * (P + 1);
  R t[NP], w[NP];
  apply1d<P, 0, 0, true, false>(r, t);
  apply1d<P, 0, 1, true, false>(t, w);
  apply1d<P, 0, 2, true, false>(w, fe);
}

__device__ __forceinline__ float clamp01(float x) { return __saturatef(x); }
__device__ __forceinline__ double clamp01(double x) { return fmin(fmax(x, 0.0), 1.0); }
__device__ __forceinline__ float expo(float x) { return __expf(x); }
__device__ __forceinline__ double expo(double x) { return exp(x); }

template <int P>
__device__ __forceinline__ constexpr double wq3(int q) {
  return Basis<P>::W(q % (P + 1)) * Basis<P>::W((q / (P + 1)) % (P + 1)) * Basis<P>::W(q / ((P + 1) * (P + 1)));
}

// Surface Gaussian 2 eta P/(pi r^2) exp(-2 d^2/r^2) on the cell's top face, (P+1)^2 Gauss
// points, added to the top-face nodes of fe; skipped when the face lies farther than 6 r from
// the spot (the integrand is below e^-72 there). Offsets from the spot in FP64, the rest in R.
template <int P, typename R>
__device__ __forceinline__ void add_laser(const CellLaunch& L, const LaserInline& las, int cell, int inst, int lev,
                                          R* fe) {
  constexpr int N = P + 1;
  const GeoR<R>& geo = geo_of<R>(L);
  R ox, oy, amp;
  if (sizeof(R) == 4) {  // FP32 operator: positions and powers in FP32 too
    ox = R(L.mesh.cell_lof[3 * cell] - float(las.sx));
    oy = R(L.mesh.cell_lof[3 * cell + 1] - float(las.sy));
    amp = R(float(las.amp) * las.powerf[inst * kMaxSeg + las.seg]);
  } else {
    ox = R(L.mesh.cell_lo[3 * cell] - las.sx);
    oy = R(L.mesh.cell_lo[3 * cell + 1] - las.sy);
    amp = R(las.amp * las.power[inst * kMaxSeg + las.seg]);
  }
  const R hx = geo.h[lev][0], hy = geo.h[lev][1];
  const R gx = max(R(0), max(ox, -(ox + hx))), gy = max(R(0), max(oy, -(oy + hy)));
  if (gx * gx + gy * gy > R(las.cut2)) return;
  const R ir2 = R(las.ir2);
#pragma unroll
  for (int qy = 0; qy < N; ++qy)
#pragma unroll
    for (int qx = 0; qx < N; ++qx) {
      const R x = ox + R(Basis<P>::X(qx)) * hx, y = oy + R(Basis<P>::X(qy)) * hy;
      const R q = amp * expo(-(x * x + y * y) * ir2) * R(Basis<P>::W(qx) * Basis<P>::W(qy)) * hx * hy;
#pragma unroll
      for (int j = 0; j < N; ++j)
#pragma unroll
        for (int k = 0; k < N; ++k) fe[k + N * (j + N * P)] += q * R(Basis<P>::S(qy, j) * Basis<P>::S(qx, k));
    }
}

}  // namespace pbf
