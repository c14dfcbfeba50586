// Fused explicit step (FP32 operator, one instance): one launch per forward-Euler step of
// Eq. forward_euler with the matrix-free operator of Sec. 4.2.
//
// Each block takes a patch of kStepCells consecutive Z-order cells and
//  1. loads its patch tables (independent of the previous step, so under programmatic
//     dependent launch this overlaps the previous kernel's tail);
//  2. stages the patch's unique node values in shared memory, completing the previous step
//     on the fly, T_n = T_{n-1} + dt f_{n-1} / C~, at every dof slot (the patch that owns
//     the dof stores T_n), then interpolates its hanging nodes from their masters, which the
//     patch lists too (T_e = P G_e T);
//  3. evaluates the sum-factorised diffusion operator and the surface laser of its cells,
//     one thread per cell, gathering from and accumulating into shared memory;
//  4. pushes hanging-node sums to their masters in shared memory (G_e^T P^T) and adds each
//     dof slot's sum to global memory once, in ascending dof order.
// Compared with a per-cell gather / atomic scatter plus a separate update kernel, a dof's
// value is read about 1.4 times instead of once per adjacent cell (up to 8 for Q2 vertices),
// its contributions are added with one global atomic per patch instead of one per cell, and
// the update costs no launch of its own.
#include <utility>

#include "cell_ops.cuh"
#include "step.cuh"

namespace pbf {
namespace {

__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependency_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

constexpr int kStepMinBlocks = 10;  // 64-thread blocks: at most 102 registers per thread
constexpr int kStageUnroll = 8;     // dof slots each thread has in flight while staging

template <int P, bool NLK, int CAP>
__global__ void __launch_bounds__(kStepCells, kStepMinBlocks)
    k_step(const CellLaunch L, const StepTables T, const StepState S) {
  constexpr int N = P + 1, NP = N * N * N, KP = kStepCells, U = kStageUnroll;
  (void)N;
  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t* sloc = reinterpret_cast<uint16_t*>(smem);                // [NP][KP]
  int32_t* sslot = reinterpret_cast<int32_t*>(smem + NP * KP * 2);   // [max_nu32]
  float* sv = reinterpret_cast<float*>(sslot + T.max_nu32);          // staged values (swizzled)
  float* sf = sv + T.max_nu32;                                       // contributions (swizzled)
  float* shw = sf + T.max_nu32;                                      // [max_hent8] weights
  uint16_t* shl = reinterpret_cast<uint16_t*>(shw + T.max_hent8);    // [max_hent8] master positions
  const DevMesh& M = L.mesh;
  const int p = blockIdx.x, tid = threadIdx.x;
  const int p0 = __ldg(&T.ptr[p]);
  const int4 cn = __ldg(&T.cnt[p]);
  const int nfree = cn.x, nu = cn.y, hb = cn.z, nh = cn.w - cn.z;

  // 1. tables (16-byte loads; the loc table of a patch is NP * KP * 2 bytes, a multiple of 16)
  {
    const uint4* src = reinterpret_cast<const uint4*>(T.loc + (size_t)p * NP * KP);
    uint4* dst = reinterpret_cast<uint4*>(sloc);
#pragma unroll 4
    for (int i = tid; i < NP * KP / 8; i += KP) dst[i] = __ldg(&src[i]);
    const int4* s4 = reinterpret_cast<const int4*>(T.slot + p0);
    int4* d4 = reinterpret_cast<int4*>(sslot);
    const int n4 = (nu + 3) >> 2;
    for (int i = tid; i < n4; i += KP) d4[i] = __ldg(&s4[i]);
    for (int i = tid; i < nh; i += KP) {
      shl[i] = __ldg(&T.hloc[hb + i]);
      shw[i] = __ldg(&T.hw[hb + i]);
    }
  }
  const int c0 = p * KP, ncell = min(KP, M.n_cells - c0);
  const int cell = c0 + tid;
  const bool active = tid < ncell;
  int lev = 0, mat = 0, top = 0;
  if (active) {
    lev = __ldg(&M.cell_level[cell]);
    mat = __ldg(&M.cell_mat[cell]);
    top = __ldg(&M.cell_top[cell]);
  }
  grid_dependency_wait();  // the previous step's state and accumulators are complete
  __syncthreads();

  // 2a. dof slots: U independent slots in flight per thread
  for (int j0 = 0; j0 < nfree; j0 += KP * U) {
    int g[U];
    float2 x[U];
    float fi[U], ic[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u * KP + tid;
      g[u] = j < nfree ? (sslot[j] & 0x7fffffff) : -1;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int d = g[u] < 0 ? 0 : g[u];
      x[u] = __ldg(&S.x_in[d]);
      fi[u] = __ldg(&S.f_in[d]);
      ic[u] = __ldg(&S.invC0x[d]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u * KP + tid;
      if (g[u] >= 0) {
        const float2 t = S.first ? x[u] : euler_ff<CAP>(x[u], fi[u], ic[u], S.nc, S.x_dir, S.dt);
        const int q = step_swizzle(j);
        sv[q] = t.x;
        sf[q] = 0.f;
        if (sslot[j] < 0) {
          S.x_out[g[u]] = t;
          S.f_clear[g[u]] = 0.f;
        }
      }
    }
  }
  __syncthreads();
  // 2b. hanging slots from their masters in shared memory: x_h = sum_m w_m x_m
  for (int j = nfree + tid; j < nu; j += KP) {
    const int h = sslot[j], e0 = h >> 5, ne = h & 31;
    float val = 0.f;
    for (int e = e0; e < e0 + ne; ++e) val += shw[e] * sv[shl[e]];
    const int q = step_swizzle(j);
    sv[q] = val;
    sf[q] = 0.f;
  }
  __syncthreads();

  // 3. the cells: f_e = -int k(T_h) grad N . grad T_h (+ the surface laser)
  if (active) {
    const MatR<float>& mt = L.mf;
    const GeoR<float>& geo = L.gf;
    float u[NP], v[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) u[a] = sv[sloc[a * KP + tid]];
    values_at_qp<P, float>(u, v);
    const float detJ = geo.detJ[lev];
    const float scale = (mat == 1 ? mt.powder_scale : 1.f) * (L.k_scale_f ? L.k_scale_f[0] : 1.f);
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
    if (L.las.on && top) add_laser<P, float>(L, cell, 0, lev, fe);
#pragma unroll
    for (int a = 0; a < NP; ++a) atomicAdd(&sf[sloc[a * KP + tid]], fe[a]);
  }
  __syncthreads();
  grid_dependency_trigger();  // the next step may start loading its tables
  // 4a. hanging contributions to their masters (P_h^T f_h), in shared memory
  for (int j = nfree + tid; j < nu; j += KP) {
    const int h = sslot[j], e0 = h >> 5, ne = h & 31;
    const float val = sf[step_swizzle(j)];
    if (val != 0.f)
      for (int e = e0; e < e0 + ne; ++e) atomicAdd(&sf[shl[e]], shw[e] * val);
  }
  __syncthreads();
  // 4b. one global addition per dof slot
  for (int j = tid; j < nfree; j += KP) {
    const float val = sf[step_swizzle(j)];
    if (val != 0.f) atomicAdd(&S.f_acc[sslot[j] & 0x7fffffff], val);
  }
}

template <int CAP>
__global__ void k_step_final(int n, const float2* __restrict__ x_in, float* __restrict__ f_in,
                             float* __restrict__ f_other, const float* __restrict__ invC0x, const NodalCap nc,
                             float2 x_dir, float dt, double off, double* __restrict__ T) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float2 t = euler_ff<CAP>(x_in[i], f_in[i], invC0x[i], nc, x_dir, dt);
  T[i] = off + (f2d(t.x) + f2d(t.y));
  f_in[i] = 0.f;
  if (f_other) f_other[i] = 0.f;
}

// x = T - off as hi + lo: the FP64 difference is exact to 53 bits, hi its FP32 rounding and
// lo = (T - off - hi) rounded (the FP64 subtraction is exact)
__global__ void k_step_prepare(int n, const double* __restrict__ T, double off, float2* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = T[i] - off;
  const float hi = d2f_rn(v);
  x[i] = make_float2(hi, d2f_rn(v - f2d(hi)));
}

template <typename... KArgs, typename... Args>
cudaError_t launch_ex(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, bool pdl, cudaStream_t s,
                      Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? attr : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <int P, bool NLK, int CAP>
cudaError_t go_step(const CellLaunch& L, const StepTables& t, const StepState& st, bool pdl, cudaStream_t s) {
  auto kern = k_step<P, NLK, CAP>;
  if (t.smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, t.smem);
    if (e != cudaSuccess) return e;
  }
  return launch_ex(kern, (unsigned)t.n_patches, kStepCells, (size_t)t.smem, pdl, s, L, t, st);
}

template <int P>
cudaError_t dispatch_step(const CellLaunch& L, const StepTables& t, const StepState& st, int cap, bool pdl,
                          cudaStream_t s) {
  const bool nl = L.nonlin_k != 0;
  if (cap == CAP_NODAL) return nl ? go_step<P, true, CAP_NODAL>(L, t, st, pdl, s) : go_step<P, false, CAP_NODAL>(L, t, st, pdl, s);
  return nl ? go_step<P, true, CAP_CONST>(L, t, st, pdl, s) : go_step<P, false, CAP_CONST>(L, t, st, pdl, s);
}

}  // namespace

cudaError_t launch_step(const CellLaunch& L, const StepTables& t, const StepState& st, int cap, bool pdl,
                        cudaStream_t s) {
  // the fused form covers one instance of the FP32 operator with the constant or nodal capacity
  if (!L.f32 || L.mesh.batch != 1 || !(cap == CAP_CONST || cap == CAP_NODAL) || !t.ptr || !t.cnt || !t.slot || !t.hloc || !t.hw ||
      !t.loc || !st.x_in || !st.x_out || !st.f_in || !st.f_acc || !st.f_clear || !st.invC0x ||
      st.x_in == st.x_out || st.f_in == st.f_acc || st.f_in == st.f_clear || st.f_acc == st.f_clear)
    return cudaErrorInvalidValue;
  if (t.n_patches == 0) return cudaSuccess;
  if (L.degree == 1) return dispatch_step<1>(L, t, st, cap, pdl, s);
  if (L.degree == 2) return dispatch_step<2>(L, t, st, cap, pdl, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_step_prepare(int64_t n_dofs, const double* T, double off, float2* x, cudaStream_t s) {
  if (n_dofs == 0) return cudaSuccess;
  const int bs = 256;
  k_step_prepare<<<(unsigned)((n_dofs + bs - 1) / bs), bs, 0, s>>>((int)n_dofs, T, off, x);
  return cudaGetLastError();
}

cudaError_t launch_step_final(int cap, int64_t n_dofs, const float2* x_in, float* f_in, float* f_other,
                              const float* invC0x, const NodalCap& nc, float2 x_dir, float dt, double off, double* T,
                              cudaStream_t s) {
  if (n_dofs == 0) return cudaSuccess;
  const int bs = 256;
  const unsigned grid = (unsigned)((n_dofs + bs - 1) / bs);
  if (cap == CAP_NODAL)
    k_step_final<CAP_NODAL><<<grid, bs, 0, s>>>((int)n_dofs, x_in, f_in, f_other, invC0x, nc, x_dir, dt, off, T);
  else if (cap == CAP_CONST)
    k_step_final<CAP_CONST><<<grid, bs, 0, s>>>((int)n_dofs, x_in, f_in, f_other, invC0x, nc, x_dir, dt, off, T);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace pbf
