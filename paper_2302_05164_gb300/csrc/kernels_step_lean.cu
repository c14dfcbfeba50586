// Fused explicit step, lean form (FP32 operator, one instance): the step of kernels_step.cu
// (Eq. forward_euler with the matrix-free operator of Sec. 4.2; the previous step completed
// while staging, hanging nodes resolved in shared memory, one global addition per dof slot)
// with the patch tables kept in global memory and read through L1 instead of shared memory.
#include <algorithm>

#include "cell_ops.cuh"
#include "step.cuh"

namespace pbf {
namespace {

// ---- lean form: the same step with fewer registers and less shared memory ----------------
//
// The patch tables stay in global memory and are read through L1 (prefetched into L1 before
// the wait on the previous step), so that shared memory holds only the staged values and
// their sums (8 bytes per slot); the cell operator recomputes the conductivity in each of the
// three gradient passes instead of keeping it per quadrature point (the fused
// multiply-add with saturation makes that as cheap as the stored form) and folds the
// quadrature weights into the transposed derivative coefficients. Fewer live registers and
// less shared memory per block let more patches run at once on an SM.

constexpr int kLeanUnroll = 8;  // dof slots each thread has in flight while staging

// The gradient part of the cell operator on the values v at the quadrature points:
// r = sum_d D_d^T (W k(T) detJ / h_d^2 * D_d v) with k = scale (k0 + dk clamp((v + tk_off) /
// dT, 0, 1)) recomputed in each direction d; W the tensor Gauss weights, folded into the
// transposed derivative coefficients. Sign: the residual's -k.
template <int P, bool NLK>
__device__ __forceinline__ void cell_gradient_lean(const float* v, float* r, const MatR<float>& mt, float scale,
                                                   const GeoR<float>& geo, int lev) {
  constexpr int N = P + 1;
  const float detJ = geo.detJ[lev];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float sd = detJ * geo.ih2[lev][d] * scale;
    const float k0s = -mt.k0 * sd, dks = -mt.dk * sd;
    // the ramp's constants pass through an opaque move in each direction, so that the
    // compiler evaluates k(T) where it is used instead of keeping it per point across the
    // three directions (which is what the recomputation avoids)
    float inv, zo;
    asm volatile("mov.b32 %0, %1;" : "=f"(inv) : "f"(mt.inv_dT));
    asm volatile("mov.b32 %0, %1;" : "=f"(zo) : "f"(mt.tk_off * mt.inv_dT));
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
      for (int a = 0; a < N; ++a) {
        float g[N];
#pragma unroll
        for (int q = 0; q < N; ++q) {
          float s = 0.f;
#pragma unroll
          for (int i = 0; i < N; ++i) {
            const double m = Basis<P>::D(q, i);
            if (m != 0.0) s = s + float(m) * v[lin<N>(d, a, b, i)];
          }
          float kq = k0s;
          if (NLK) kq = fmaf(dks, __saturatef(fmaf(v[lin<N>(d, a, b, q)], inv, zo)), k0s);
          g[q] = s * kq;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
          float acc = d == 0 ? 0.f : r[lin<N>(d, a, b, i)];
#pragma unroll
          for (int q = 0; q < N; ++q) {
            const double c = Basis<P>::D(q, i) * Basis<P>::W(q) * Basis<P>::W(a) * Basis<P>::W(b);
            if (c != 0.0) acc = acc + float(c) * g[q];
          }
          r[lin<N>(d, a, b, i)] = acc;
        }
      }
  }
}

// MINB: resident blocks per SM the register budget is chosen for (14: 72 registers per
// thread, 12: 80, 10: 96).
template <int P, bool NLK, int CAP, int MINB>
__global__ void __launch_bounds__(kStepCells, MINB)
    k_step_lean(const CellLaunch L, const StepTables T, const StepState S) {
  constexpr int N = P + 1, NP = N * N * N, KP = kStepCells, U = kLeanUnroll;
  (void)N;
  extern __shared__ __align__(16) unsigned char smem[];
  float* sv = reinterpret_cast<float*>(smem);  // [max_nu32] staged values, swizzled
  float* sf = sv + T.max_nu32;                   // [max_nu32] accumulated contributions
  const DevMesh& M = L.mesh;
  const int tid = threadIdx.x, p = blockIdx.x;
  grid_dependency_trigger();  // the next step may be scheduled once every block of this one started
  // independent of the previous step: tables and cell data, prefetched before the wait
  const int p0 = __ldg(&T.ptr[p]);
  const int4 cn = __ldg(&T.cnt[p]);
  const int nfree = cn.x, nu = cn.y, hb = cn.z;
  const int cell = __ldg(&T.cell[p * KP + tid]);
  const uint16_t* loc = T.loc + (size_t)p * NP * KP + tid;
  int lev = 0, mat = 0, top = 0;
  if (cell >= 0) {
    lev = __ldg(&M.cell_level[cell]);
    mat = __ldg(&M.cell_mat[cell]);
    top = __ldg(&M.cell_top[cell]);
  }
  {
    // one L1 prefetch per 128-byte line of the patch's slot list, cell-node positions and
    // hanging table
    const char* sb = reinterpret_cast<const char*>(T.slot + p0);
    const char* lb = reinterpret_cast<const char*>(T.loc + (size_t)p * NP * KP);
    const int ns = (nu * 4 + 127) >> 7, nl = (NP * KP * 2 + 127) >> 7;
    for (int i = tid; i < ns + nl; i += KP) {
      // the line of byte min(128 i, end - 4): every address lies inside the tables
      const char* a = i < ns ? sb + min(i << 7, (nu - 1) * 4) : lb + ((i - ns) << 7);
      asm volatile("prefetch.global.L1 [%0];" ::"l"(a));
    }
  }
  grid_dependency_wait();  // the previous step's state and accumulators are complete
  // 2a. dof slots (the previous step's update applied on the fly; the owner stores it)
  for (int j0 = 0; j0 < nfree; j0 += KP * U) {
    int sl[U];
    float2 x[U];
    float fi[U], ic[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u * KP + tid;
      sl[u] = j < nfree ? __ldg(&T.slot[p0 + j]) : 0;
    }
    if (S.first) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const double vv = __ldg(&S.T0[sl[u] & 0x7fffffff]) - S.off;
        const float hi = d2f_rn(vv);
        x[u] = make_float2(hi, d2f_rn(vv - f2d(hi)));
      }
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int dd = sl[u] & 0x7fffffff;
        x[u] = __ldg(&S.x_in[dd]);
        fi[u] = __ldg(&S.f_in[dd]);
        ic[u] = __ldg(&S.invC0x[dd]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) x[u] = euler_ff<CAP>(x[u], fi[u], ic[u], S.nc, S.x_dir, S.dt);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u * KP + tid;
      if (j < nfree) {
        const int q = step_swizzle(j);
        sv[q] = x[u].x;
        sf[q] = 0.f;
        if (sl[u] < 0) {
          const int dd = sl[u] & 0x7fffffff;
          S.x_out[dd] = x[u];
          S.f_clear[dd] = 0.f;
        }
      }
    }
  }
  __syncthreads();
  // 2b. hanging slots from their masters: x_h = sum_m w_m x_m
  for (int j = nfree + tid; j < nu; j += KP) {
    const int h = __ldg(&T.slot[p0 + j]), e0 = hb + (h >> 5), ne = h & 31;
    float val = 0.f;
    for (int e = e0; e < e0 + ne; ++e) val += __ldg(&T.hw[e]) * sv[__ldg(&T.hloc[e])];
    const int q = step_swizzle(j);
    sv[q] = val;
    sf[q] = 0.f;
  }
  __syncthreads();
  // 3. the cells
  if (cell >= 0) {
    float r[NP];
    {
      float v[NP];
      {
        float u[NP];
#pragma unroll
        for (int a = 0; a < NP; ++a) u[a] = sv[__ldg(&loc[a * KP])];
        values_at_qp<P, float>(u, v);
      }
      const float scale = (mat == 1 ? L.mf.powder_scale : 1.f) * (L.k_scale_f ? L.k_scale_f[0] : 1.f);
      cell_gradient_lean<P, NLK>(v, r, L.mf, scale, L.gf, lev);
    }
    float fe[NP];
    integrate_values<P, float>(r, fe);
    if (L.las.on && top) add_laser<P, float>(L, L.las, cell, 0, lev, fe);
#pragma unroll
    for (int a = 0; a < NP; ++a) atomicAdd(&sf[__ldg(&loc[a * KP])], fe[a]);
  }
  __syncthreads();
  // 4a. hanging contributions to their masters
  for (int j = nfree + tid; j < nu; j += KP) {
    const int h = __ldg(&T.slot[p0 + j]), e0 = hb + (h >> 5), ne = h & 31;
    const float val = sf[step_swizzle(j)];
    if (val != 0.f)
      for (int e = e0; e < e0 + ne; ++e) atomicAdd(&sf[__ldg(&T.hloc[e])], __ldg(&T.hw[e]) * val);
  }
  __syncthreads();
  // 4b. one global addition per dof slot
  for (int j = tid; j < nfree; j += KP) {
    const float val = sf[step_swizzle(j)];
    if (val != 0.f) atomicAdd(&S.f_acc[__ldg(&T.slot[p0 + j]) & 0x7fffffff], val);
  }
}

template <int P, bool NLK, int CAP, int MINB>
cudaError_t go_lean(const CellLaunch& L, const StepTables& t, const StepState& st, cudaStream_t s) {
  auto kern = k_step_lean<P, NLK, CAP, MINB>;
  const size_t smem = (size_t)t.max_nu32 * 8;
  cudaError_t e = cudaSuccess;
  if (smem > 48 * 1024) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // shared memory for MINB blocks, the rest of the unified L1 / shared storage left to L1,
  // which holds the patch tables
  const int pct = (int)std::min<size_t>(100, (smem * MINB * 100 + 228 * 1024 - 1) / (228 * 1024) + 2);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
  if (e != cudaSuccess) return e;
  return launch_ex(kern, (unsigned)t.n_patches, kStepCells, smem, 1, s, L, t, st);
}

template <int P, int MINB>
cudaError_t dispatch_lean(const CellLaunch& L, const StepTables& t, const StepState& st, int cap, cudaStream_t s) {
  const bool nl = L.nonlin_k != 0;
  if (cap == CAP_NODAL) return nl ? go_lean<P, true, CAP_NODAL, MINB>(L, t, st, s) : go_lean<P, false, CAP_NODAL, MINB>(L, t, st, s);
  return nl ? go_lean<P, true, CAP_CONST, MINB>(L, t, st, s) : go_lean<P, false, CAP_CONST, MINB>(L, t, st, s);
}

template <int P>
cudaError_t dispatch_lean_form(const CellLaunch& L, const StepTables& t, const StepState& st, int cap, int form,
                               cudaStream_t s) {
  switch (form) {
    case 0: return dispatch_lean<P, kLeanForms[0]>(L, t, st, cap, s);
    case 1: return dispatch_lean<P, kLeanForms[1]>(L, t, st, cap, s);
    case 2: return dispatch_lean<P, kLeanForms[2]>(L, t, st, cap, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_step_lean(const CellLaunch& L, const StepTables& t, const StepState& st, int cap, int form,
                             cudaStream_t s) {
  if (!L.f32 || L.mesh.batch != 1 || !(cap == CAP_CONST || cap == CAP_NODAL) || !t.ptr || !t.cnt || !t.slot ||
      !t.cell || !t.hloc || !t.hw || !t.loc || !st.x_in || !st.x_out || !st.f_in || !st.f_acc || !st.f_clear ||
      !st.invC0x || st.x_in == st.x_out || st.f_in == st.f_acc || st.f_in == st.f_clear || st.f_acc == st.f_clear ||
      L.phase || st.has_loss)  // the model options run in the fused step kernel
    return cudaErrorInvalidValue;
  if (t.n_patches == 0) return cudaSuccess;
  if (L.degree == 1) return dispatch_lean_form<1>(L, t, st, cap, form, s);
  if (L.degree == 2) return dispatch_lean_form<2>(L, t, st, cap, form, s);
  return cudaErrorInvalidValue;
}

}  // namespace pbf
