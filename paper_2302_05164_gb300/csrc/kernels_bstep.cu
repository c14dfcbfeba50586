// Fused explicit step for a batch of instances (FP32 operator; Eq. forward_euler with the
// matrix-free operator of Sec. 4.2): one launch per step advances every instance. Threads are
// (cell, instance) pairs with the instance fastest, so each gather and each atomic addition of
// a warp touches consecutive values of one dof, and the mesh tables are read once per cell
// for all instances of a warp. Per thread:
//  1. gather the cell's 27 (Q2) node values, completing the previous step on the fly,
//     T_n = T_{n-1} + dt f_{n-1} / C~ (the cell that owns a dof stores its T_n and clears
//     the accumulator of step n+1); hanging nodes are interpolated from their masters'
//     updated values (T_e = P G_e T);
//  2. the sum-factorised diffusion operator with k(T), and the surface laser, whose spot the
//     block computes on the device from the call's start time and the step index (so a chunk
//     of steps can be replayed as one CUDA graph);
//  3. add the cell vector to the dofs and, through the constraint rows, to the masters of
//     hanging nodes (G_e^T P^T), with atomics contiguous over the instances.
// The state is T - T_ref as an unevaluated FP32 pair per dof and instance, as in the
// single-instance fused step.
#include "cell_ops.cuh"
#include "step.cuh"

namespace pbf {
namespace {

// value of one dof and instance at step n: the previous state completed by its update. The
// previous state and accumulator are written by earlier launches only (this launch writes the
// other buffers), so they are read through the read-only path, where the re-reads of a dof by
// its other adjacent cells can hit L1.
template <int CAP>
__device__ __forceinline__ float2 staged(const BStepArgs& A, int d, int idx) {
  if (A.first) {
    const double v = __ldg(&A.T0[idx]) - A.off;
    const float hi = d2f_rn(v);
    return make_float2(hi, d2f_rn(v - f2d(hi)));
  }
  return euler_ff<CAP>(__ldg(&A.x_in[idx]), __ldg(&A.f_in[idx]), __ldg(&A.invC0x[d]), A.nc, A.x_dir, A.dt);
}

template <int P, bool NLK, int CAP>
__global__ void __launch_bounds__(128) k_bstep(const CellLaunch L, const BStepArgs A) {
  constexpr int N = P + 1, NP = N * N * N;
  (void)N;
  const DevMesh& M = L.mesh;
  const int B = M.batch;
  __shared__ LaserInline s_las;
  if (threadIdx.x == 0) {
    LaserInline las = L.las;
    las.on = 0;
    if (A.laser) {
      const Spot sp = spot_at(*A.laser, __dadd_rn(*A.t0, __dmul_rn((double)A.step, A.dt64)));
      las.on = sp.seg >= 0 && A.laser->n_seg > 0 && !A.laser->volumetric;
      las.seg = sp.seg;
      las.sx = sp.x;
      las.sy = sp.y;
    }
    s_las = las;
  }
  __syncthreads();
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= M.n_cells * B) return;
  const int cell = tid / B, inst = tid - cell * B;
  const uint32_t own = __ldg(&A.own[cell]);
  float u[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    const int d = __ldg(&M.cell_dofs[a * M.n_cells + cell]);
    if (d >= 0) {
      const int idx = d * B + inst;
      const float2 x = staged<CAP>(A, d, idx);
      u[a] = x.x;
      if ((own >> a) & 1u) {
        A.x_out[idx] = x;
        A.f_clear[idx] = 0.f;
      }
    } else {
      const int row = -1 - d;
      float val = 0.f;
      for (int e = __ldg(&M.con_ptr[row]); e < __ldg(&M.con_ptr[row + 1]); ++e) {
        const int m = __ldg(&M.con_idx[e]);
        val += __ldg(&M.con_wf[e]) * staged<CAP>(A, m, m * B + inst).x;
      }
      u[a] = val;
    }
  }
  float v[NP];
  values_at_qp<P, float>(u, v);
  const int lev = M.cell_level[cell];
  const MatR<float>& mt = L.mf;
  const GeoR<float>& geo = L.gf;
  const float detJ = geo.detJ[lev];
  const float scale = (M.cell_mat[cell] == 1 ? mt.powder_scale : 1.f) * (L.k_scale_f ? L.k_scale_f[inst] : 1.f);
  const float k0 = mt.k0 * scale, dk = mt.dk * scale;
  float kw[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    float k = k0;
    if (NLK) k = k0 + dk * clamp01((v[q] + mt.tk_off) * mt.inv_dT);
    kw[q] = -k * (float(wq3<P>(q)) * detJ);
  }
  float r[NP], g[NP];
  {
    const float cd = geo.ih2[lev][0];
    apply1d<P, 1, 0, false, false>(v, g);
#pragma unroll
    for (int q = 0; q < NP; ++q) g[q] *= kw[q] * cd;
    apply1d<P, 1, 0, true, false>(g, r);
  }
  {
    const float cd = geo.ih2[lev][1];
    apply1d<P, 1, 1, false, false>(v, g);
#pragma unroll
    for (int q = 0; q < NP; ++q) g[q] *= kw[q] * cd;
    apply1d<P, 1, 1, true, true>(g, r);
  }
  {
    const float cd = geo.ih2[lev][2];
    apply1d<P, 1, 2, false, false>(v, g);
#pragma unroll
    for (int q = 0; q < NP; ++q) g[q] *= kw[q] * cd;
    apply1d<P, 1, 2, true, true>(g, r);
  }
  float fe[NP];
  integrate_values<P, float>(r, fe);
  if (s_las.on && M.cell_top[cell]) add_laser<P, float>(L, s_las, cell, inst, lev, fe);
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    const int d = __ldg(&M.cell_dofs[a * M.n_cells + cell]);
    if (d >= 0) {
      atomicAdd(&A.f_acc[d * B + inst], fe[a]);
    } else {
      const int row = -1 - d;
      for (int e = __ldg(&M.con_ptr[row]); e < __ldg(&M.con_ptr[row + 1]); ++e)
        atomicAdd(&A.f_acc[__ldg(&M.con_idx[e]) * B + inst], __ldg(&M.con_wf[e]) * fe[a]);
    }
  }
}

// the last update of a sequence: T = T_ref + x_{N-1} + dt f_{N-1} / C~ (FP64 out) for every
// dof and instance, clearing f_in and f_other (nullable)
template <int CAP>
__global__ void k_bstep_final(int64_t n, int B, const float2* __restrict__ x_in, float* __restrict__ f_in,
                              float* __restrict__ f_other, const float* __restrict__ invC0x, const NodalCap nc,
                              float2 x_dir, float dt, double off, double* __restrict__ T) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float2 t = euler_ff<CAP>(x_in[i], f_in[i], invC0x[i / B], nc, x_dir, dt);
  T[i] = off + (f2d(t.x) + f2d(t.y));
  f_in[i] = 0.f;
  if (f_other) f_other[i] = 0.f;
}

template <int P, bool NLK, int CAP>
cudaError_t go_bstep(const CellLaunch& L, const BStepArgs& A, cudaStream_t s) {
  const int bs = 128;
  const int64_t nt = (int64_t)L.mesh.n_cells * L.mesh.batch;
  k_bstep<P, NLK, CAP><<<(unsigned)((nt + bs - 1) / bs), bs, 0, s>>>(L, A);
  return cudaGetLastError();
}

template <int P>
cudaError_t dispatch_bstep(const CellLaunch& L, const BStepArgs& A, int cap, cudaStream_t s) {
  const bool nl = L.nonlin_k != 0;
  if (cap == CAP_NODAL) return nl ? go_bstep<P, true, CAP_NODAL>(L, A, s) : go_bstep<P, false, CAP_NODAL>(L, A, s);
  return nl ? go_bstep<P, true, CAP_CONST>(L, A, s) : go_bstep<P, false, CAP_CONST>(L, A, s);
}

}  // namespace

cudaError_t launch_bstep(const CellLaunch& L, const BStepArgs& A, int cap, cudaStream_t s) {
  if (!L.f32 || !(cap == CAP_CONST || cap == CAP_NODAL) || !A.own || !A.x_out || !A.f_acc || !A.f_clear ||
      !A.invC0x || !A.t0 || (!A.first && (!A.x_in || !A.f_in)) || (A.first && !A.T0) || A.f_acc == A.f_clear ||
      A.x_in == A.x_out)
    return cudaErrorInvalidValue;
  if (L.mesh.n_cells == 0) return cudaSuccess;
  if ((int64_t)L.mesh.n_cells * L.mesh.batch >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
  if (L.degree == 1) return dispatch_bstep<1>(L, A, cap, s);
  if (L.degree == 2) return dispatch_bstep<2>(L, A, cap, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_bstep_final(int cap, int64_t n_dofs, int B, const float2* x_in, float* f_in, float* f_other,
                               const float* invC0x, const NodalCap& nc, float2 x_dir, float dt, double off, double* T,
                               cudaStream_t s) {
  const int64_t n = n_dofs * B;
  if (n == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((n + 255) / 256);
  if (cap == CAP_NODAL)
    k_bstep_final<CAP_NODAL><<<grid, 256, 0, s>>>(n, B, x_in, f_in, f_other, invC0x, nc, x_dir, dt, off, T);
  else if (cap == CAP_CONST)
    k_bstep_final<CAP_CONST><<<grid, 256, 0, s>>>(n, B, x_in, f_in, f_other, invC0x, nc, x_dir, dt, off, T);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace pbf
