// Fused explicit step (FP32 operator, one instance): one launch per forward-Euler step of
// Eq. forward_euler with the matrix-free operator of Sec. 4.2.
//
// Each block takes a patch of kStepCells cells (consecutive in the global Morton order) and
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
// value is read about 1.5 times instead of once per adjacent cell (up to 8 for Q2 vertices),
// its contributions are added with one global atomic per patch instead of one per cell, and
// the update costs no launch of its own.
#include <algorithm>
#include <utility>

#include "cell_ops.cuh"
#include "step.cuh"

namespace pbf {
namespace {

constexpr int kStepMinBlocks = 10;  // 64-thread blocks: at most 102 registers per thread
constexpr int kStageUnroll = 14;    // dof slots each thread has in flight while staging

// Loads of data that changes between steps: through the read-only path when each step is its
// own launch, through L2 only (coherent with other blocks' stores) inside a persistent launch.
template <bool COHERENT, typename V>
__device__ __forceinline__ V ld_step(const V* p) {
  if (COHERENT) return __ldcg(p);
  return __ldg(p);
}

// Shared-memory layout of one block (dynamic shared memory, sized by step_smem_bytes).
template <int NP>
struct StepSmem {
  uint16_t* loc;   // [NP][kStepCells] shared position of each cell node
  int32_t* slot;   // [max_nu32] the patch's slot list
  float* v;        // [max_nu32] staged values, swizzled
  float* f;        // [max_nu32] accumulated contributions, swizzled
  float* hw;       // [max_hent8] hanging-table weights
  uint16_t* hl;    // [max_hent8] hanging-table master positions
  __device__ StepSmem(unsigned char* base, const StepTables& T) {
    loc = reinterpret_cast<uint16_t*>(base);
    slot = reinterpret_cast<int32_t*>(base + NP * kStepCells * 2);
    v = reinterpret_cast<float*>(slot + T.max_nu32);
    f = v + T.max_nu32;
    hw = f + T.max_nu32;
    hl = reinterpret_cast<uint16_t*>(hw + T.max_hent8);
  }
};

// Patch tables into shared memory (they never change: read-only path).
template <int NP>
__device__ __forceinline__ void load_patch_tables(const StepTables& T, const StepSmem<NP>& sm, int p, int4& cn) {
  constexpr int KP = kStepCells;
  const int tid = threadIdx.x;
  const int p0 = __ldg(&T.ptr[p]);
  cn = __ldg(&T.cnt[p]);
  const uint4* src = reinterpret_cast<const uint4*>(T.loc + (size_t)p * NP * KP);
  uint4* dst = reinterpret_cast<uint4*>(sm.loc);
#pragma unroll 4
  for (int i = tid; i < NP * KP / 8; i += KP) dst[i] = __ldg(&src[i]);
  const int4* s4 = reinterpret_cast<const int4*>(T.slot + p0);
  int4* d4 = reinterpret_cast<int4*>(sm.slot);
  const int n4 = (cn.y + 3) >> 2;
  for (int i = tid; i < n4; i += KP) d4[i] = __ldg(&s4[i]);
  const int hb = cn.z, nh = cn.w - cn.z;
  for (int i = tid; i < nh; i += KP) {
    sm.hl[i] = __ldg(&T.hloc[hb + i]);
    sm.hw[i] = __ldg(&T.hw[hb + i]);
  }
}

// Steps 2-4 of one patch (tables already in shared memory, a barrier after loading them):
// staging with the previous step's update, hanging values, the cells, the push of hanging
// sums and the scatter of the dof sums into S.f_acc. OPT: model options (kStepPhase,
// kStepLoss).
template <int P, bool NLK, int CAP, bool COHERENT, int OPT = 0>
__device__ __forceinline__ void step_patch(const CellLaunch& L, const LaserInline& las, const StepState& S,
                                           const StepTables& T, const StepSmem<(P + 1) * (P + 1) * (P + 1)>& sm,
                                           int p, int4 cn) {
  constexpr int N = P + 1, NP = N * N * N, KP = kStepCells, U = kStageUnroll;
  (void)N;
  const DevMesh& M = L.mesh;
  const int tid = threadIdx.x;
  const int nfree = cn.x, nu = cn.y;
  const int cell = __ldg(&T.cell[p * KP + tid]);
  const bool active = cell >= 0;
  int lev = 0, mat = 0, top = 0;
  if (active) {
    lev = __ldg(&M.cell_level[cell]);
    mat = __ldg(&M.cell_mat[cell]);
    top = __ldg(&M.cell_top[cell]);
  }
  // 2a. dof slots, U independent slots in flight per thread. Step 0 takes the state as given
  // (T - T_ref split into hi + lo); later steps complete the previous step first.
  for (int j0 = 0; j0 < nfree; j0 += KP * U) {
    int g[U];
    float2 x[U];
    float fi[U], ic[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u * KP + tid;
      g[u] = j < nfree ? (sm.slot[j] & 0x7fffffff) : -1;
    }
    if (S.first) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const double v = __ldg(&S.T0[g[u] < 0 ? 0 : g[u]]) - S.off;
        const float hi = d2f_rn(v);
        x[u] = make_float2(hi, d2f_rn(v - f2d(hi)));
      }
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int d = g[u] < 0 ? 0 : g[u];
        x[u] = ld_step<COHERENT>(&S.x_in[d]);
        fi[u] = ld_step<COHERENT>(&S.f_in[d]);
        ic[u] = __ldg(&S.invC0x[d]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) x[u] = euler_ff<CAP>(x[u], fi[u], ic[u], S.nc, S.x_dir, S.dt);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u * KP + tid;
      if (g[u] >= 0) {
        const int q = step_swizzle(j);
        sm.v[q] = x[u].x;
        sm.f[q] = 0.f;
        if (sm.slot[j] < 0) {
          S.x_out[g[u]] = x[u];
          S.f_clear[g[u]] = 0.f;
        }
      }
    }
  }
  __syncthreads();
  // 2b. hanging slots from their masters in shared memory: x_h = sum_m w_m x_m
  for (int j = nfree + tid; j < nu; j += KP) {
    const int h = sm.slot[j], e0 = h >> 5, ne = h & 31;
    float val = 0.f;
    for (int e = e0; e < e0 + ne; ++e) val += sm.hw[e] * sm.v[sm.hl[e]];
    const int q = step_swizzle(j);
    sm.v[q] = val;
    sm.f[q] = 0.f;
  }
  __syncthreads();

  // 3. the cells: f_e = -int k(T_h) grad N . grad T_h (+ the surface laser)
  if (active) {
    const MatR<float>& mt = L.mf;
    const GeoR<float>& geo = L.gf;
    float u[NP], v[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) u[a] = sm.v[sm.loc[a * KP + tid]];
    values_at_qp<P, float>(u, v);
    const float detJ = geo.detJ[lev];
    float kw[NP];
    if (OPT & kStepPhase) {
      // k(T, r_c) with r_c = max(stored r_c, g(T)) per quadrature point (Sec. 2, Eqs.
      // liquid_fraction .. material_parameter_interp); the history is stored where it grows
      const PhaseR<float>& ph = L.phf;
      const float is = L.k_scale_f ? L.k_scale_f[0] : 1.f;
      const float* rc_in = static_cast<const float*>(L.rc_in);
      float* rc_out = static_cast<float*>(L.rc_out);
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        const float g = clamp01((v[q] + ph.t_off) * ph.inv_dT);
        const int j = q * M.n_cells + cell;
        const float r0 = rc_in[j];
        const float rc = r0 > g ? r0 : g;
        if (rc_out && rc > r0) rc_out[j] = rc;
        kw[q] = -((ph.kp + rc * ph.dks + g * ph.dkm) * is) * (float(wq3<P>(q)) * detJ);
      }
    } else {
      const float scale = (mat == 1 ? mt.powder_scale : 1.f) * (L.k_scale_f ? L.k_scale_f[0] : 1.f);
      const float k0 = mt.k0 * scale, dk = mt.dk * scale;
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        float k = k0;
        if (NLK) k = k0 + dk * clamp01((v[q] + mt.tk_off) * mt.inv_dT);
        kw[q] = -k * (float(wq3<P>(q)) * detJ);
      }
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
    if (las.on && top) add_laser<P, float>(L, las, cell, 0, lev, fe);
    if ((OPT & kStepLoss) && top) {
      // radiation / evaporation at T_n on the top face (nodes (k, j, P), re-read from shared
      // memory), in the precision of the per-cell form's face kernel
      constexpr int NF = (P + 1) * (P + 1);
      float Tf[NF];
#pragma unroll
      for (int a = 0; a < NF; ++a) Tf[a] = sm.v[sm.loc[(NP - NF + a) * KP + tid]] + float(S.off);
      add_surface_loss<P, float>(S.loss, Tf, geo.h[lev][0], geo.h[lev][1], fe + (NP - NF));
    }
#pragma unroll
    for (int a = 0; a < NP; ++a) atomicAdd(&sm.f[sm.loc[a * KP + tid]], fe[a]);
  }
  __syncthreads();
  // 4a. hanging contributions to their masters (P_h^T f_h), in shared memory
  for (int j = nfree + tid; j < nu; j += KP) {
    const int h = sm.slot[j], e0 = h >> 5, ne = h & 31;
    const float val = sm.f[step_swizzle(j)];
    if (val != 0.f)
      for (int e = e0; e < e0 + ne; ++e) atomicAdd(&sm.f[sm.hl[e]], sm.hw[e] * val);
  }
  __syncthreads();
  // 4b. one global addition per dof slot
  for (int j = tid; j < nfree; j += KP) {
    const float val = sm.f[step_swizzle(j)];
    if (val != 0.f) atomicAdd(&S.f_acc[sm.slot[j] & 0x7fffffff], val);
  }
}

// One launch per step: block p takes patch p.
template <int P, bool NLK, int CAP, int OPT>
__global__ void __launch_bounds__(kStepCells, kStepMinBlocks)
    k_step(const CellLaunch L, const StepTables T, const StepState S) {
  constexpr int NP = (P + 1) * (P + 1) * (P + 1);
  extern __shared__ __align__(16) unsigned char smem[];
  const StepSmem<NP> sm(smem, T);
  // the next step may be scheduled once every block of this one has started: its blocks then
  // fill the SM slots that this step's last blocks free, load their tables and wait
  grid_dependency_trigger();
  int4 cn;
  load_patch_tables<NP>(T, sm, blockIdx.x, cn);
  grid_dependency_wait();  // the previous step's state and accumulators are complete
  __syncthreads();
  step_patch<P, NLK, CAP, false, OPT>(L, L.las, S, T, sm, blockIdx.x, cn);
}

// ---- persistent form: all steps of a sequence in one cooperative launch -----------------

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch (all blocks resident), in two levels so that no
// counter takes more than a few dozen atomics: block b arrives at the counter of its group
// b % kBarrierGroups; the last block of a group resets that counter and arrives at the top
// counter; the last group resets it and advances the generation, which every block waits
// for. A wait longer than kBarrierTimeoutNs, or an error flagged by another block, makes
// every block return false; the caller then leaves the kernel, so no block waits twice.
constexpr unsigned long long kBarrierTimeoutNs = 1000000000ull;
__device__ bool grid_sync(GridBarrier* gb, unsigned nblocks, unsigned& gen) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned G = nblocks < kBarrierGroups ? nblocks : kBarrierGroups;
    const unsigned g = blockIdx.x % G;
    const unsigned in_group = nblocks / G + (g < nblocks % G ? 1u : 0u);
    __threadfence();
    bool last = false;
    if (atomicAdd(&gb->group[g].count, 1u) == in_group - 1) {
      atomicExch(&gb->group[g].count, 0u);
      __threadfence();
      if (atomicAdd(&gb->count, 1u) == G - 1) {
        atomicExch(&gb->count, 0u);
        __threadfence();
        atomicAdd(&gb->gen, 1u);
        last = true;
      }
    }
    if (!last) {
      const unsigned long long t0 = global_ns();
      while (ld_acquire_gpu(&gb->gen) == gen) {
        if (ld_acquire_gpu(&gb->err) != 0u) {
          ok = 0;
          break;
        }
        if (global_ns() - t0 > kBarrierTimeoutNs) {
          atomicExch(&gb->err, 1u);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    gen += 1;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <int P, bool NLK, int CAP>
__global__ void __launch_bounds__(kStepCells, kStepMinBlocks)
    k_steps(const CellLaunch L, const StepTables T, const PersistState A) {
  constexpr int NP = (P + 1) * (P + 1) * (P + 1);
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ LaserInline s_las;
  __shared__ Spot s_spot[32];  // spots of steps 32 k .. 32 k + 31, computed by warp 0 in parallel
  __shared__ unsigned s_gen0;
  const StepSmem<NP> sm(smem, T);
  if (threadIdx.x == 0) s_gen0 = ld_acquire_gpu(&A.bar->gen);  // no barrier completes before all blocks arrive
  unsigned gen = 0;
  __syncthreads();
  gen = s_gen0;
  StepState S = A.st;
  // with a block for every patch the patch tables stay in shared memory for all steps
  const bool resident = (int)gridDim.x >= T.n_patches;
  int4 cn0 = make_int4(0, 0, 0, 0);
  if (resident) load_patch_tables<NP>(T, sm, blockIdx.x, cn0);
  for (int n = 0; n < A.nsteps; ++n) {
    S.x_in = A.x[n & 1];
    S.x_out = A.x[(n + 1) & 1];
    S.f_in = A.f[(n + 2) % 3];
    S.f_acc = A.f[n % 3];
    S.f_clear = A.f[(n + 1) % 3];
    S.first = n == 0;
    if ((n & 31) == 0 && threadIdx.x < 32) {
      // the time as the host forms it for the per-launch form: t0 + n dt, each rounded
      s_spot[threadIdx.x] = spot_at(A.laser, __dadd_rn(A.t0, __dmul_rn((double)(n + (int)threadIdx.x), A.dt64)));
      __syncwarp();
    }
    if (threadIdx.x == 0) {
      LaserInline las = A.las;
      const Spot sp = s_spot[n & 31];
      las.on = A.las.on && sp.seg >= 0;
      las.seg = sp.seg;
      las.sx = sp.x;
      las.sy = sp.y;
      s_las = las;
    }
    for (int p = blockIdx.x; p < T.n_patches; p += gridDim.x) {
      __syncthreads();  // the previous patch is done with shared memory; s_las is set
      int4 cn = cn0;
      if (!resident) {
        load_patch_tables<NP>(T, sm, p, cn);
        __syncthreads();
      }
      step_patch<P, NLK, CAP, true>(L, s_las, S, T, sm, p, cn);
    }
    if (!grid_sync(A.bar, gridDim.x + A.extra_arrivals, gen)) return;
  }
  // the last update: T = T_ref + x_{N-1} + dt f_{N-1} / C~ on owned dofs; clear f_{N-1}, f_{N-2}
  const float2* x_last = A.x[A.nsteps & 1];
  float* f_last = A.f[(A.nsteps - 1) % 3];
  float* f_prev = A.nsteps >= 2 ? A.f[(A.nsteps - 2) % 3] : nullptr;
  for (int p = blockIdx.x; p < T.n_patches; p += gridDim.x) {
    const int p0 = __ldg(&T.ptr[p]);
    const int nfree = __ldg(&T.cnt[p]).x;
    for (int j = threadIdx.x; j < nfree; j += kStepCells) {
      const int s = __ldg(&T.slot[p0 + j]);
      if (s >= 0) continue;
      const int d = s & 0x7fffffff;
      const float2 t = euler_ff<CAP>(__ldcg(&x_last[d]), __ldcg(&f_last[d]), __ldg(&A.st.invC0x[d]), A.st.nc,
                                     A.st.x_dir, A.st.dt);
      A.T[d] = A.st.off + (f2d(t.x) + f2d(t.y));
      f_last[d] = 0.f;
      if (f_prev) f_prev[d] = 0.f;
    }
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

template <int P, bool NLK, int CAP, int OPT = 0>
cudaError_t go_step(const CellLaunch& L, const StepTables& t, const StepState& st, bool pdl, cudaStream_t s) {
  auto kern = k_step<P, NLK, CAP, OPT>;
  if (t.smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, t.smem);
    if (e != cudaSuccess) return e;
  }
  return launch_ex(kern, (unsigned)t.n_patches, kStepCells, (size_t)t.smem, pdl ? 1 : 0, s, L, t, st);
}

// the model options: with the phase model the conductivity ramp of the material is not used
template <int P, int CAP>
cudaError_t dispatch_step_opt(const CellLaunch& L, const StepTables& t, const StepState& st, bool pdl,
                              cudaStream_t s) {
  const bool nl = L.nonlin_k != 0, loss = st.has_loss != 0;
  if (L.phase)
    return loss ? go_step<P, false, CAP, kStepPhase | kStepLoss>(L, t, st, pdl, s)
                : go_step<P, false, CAP, kStepPhase>(L, t, st, pdl, s);
  if (loss) return nl ? go_step<P, true, CAP, kStepLoss>(L, t, st, pdl, s) : go_step<P, false, CAP, kStepLoss>(L, t, st, pdl, s);
  return nl ? go_step<P, true, CAP>(L, t, st, pdl, s) : go_step<P, false, CAP>(L, t, st, pdl, s);
}

template <int P>
cudaError_t dispatch_step(const CellLaunch& L, const StepTables& t, const StepState& st, int cap, bool pdl,
                          cudaStream_t s) {
  if (cap == CAP_NODAL) return dispatch_step_opt<P, CAP_NODAL>(L, t, st, pdl, s);
  return dispatch_step_opt<P, CAP_CONST>(L, t, st, pdl, s);
}

template <int P, bool NLK, int CAP>
cudaError_t go_steps(const CellLaunch& L, const StepTables& t, const PersistState& ps, int* blocks, cudaStream_t s) {
  auto kern = k_steps<P, NLK, CAP>;
  cudaError_t e = cudaSuccess;
  if (t.smem > 48 * 1024) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, t.smem);
  int dev = 0, nsm = 0, per_sm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kStepCells, (size_t)t.smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = std::min(t.n_patches, nsm * per_sm);
  if (blocks) *blocks = grid;
  return launch_ex(kern, (unsigned)grid, kStepCells, (size_t)t.smem, 2, s, L, t, ps);
}

template <int P>
cudaError_t dispatch_steps(const CellLaunch& L, const StepTables& t, const PersistState& ps, int cap, int* blocks,
                           cudaStream_t s) {
  const bool nl = L.nonlin_k != 0;
  if (cap == CAP_NODAL)
    return nl ? go_steps<P, true, CAP_NODAL>(L, t, ps, blocks, s) : go_steps<P, false, CAP_NODAL>(L, t, ps, blocks, s);
  return nl ? go_steps<P, true, CAP_CONST>(L, t, ps, blocks, s) : go_steps<P, false, CAP_CONST>(L, t, ps, blocks, s);
}

}  // namespace

cudaError_t launch_steps_persistent(const CellLaunch& L, const StepTables& t, const PersistState& ps, int cap,
                                    int* blocks, cudaStream_t s) {
  const StepState& st = ps.st;
  if (!L.f32 || L.mesh.batch != 1 || !(cap == CAP_CONST || cap == CAP_NODAL) || !t.ptr || !t.cnt || !t.slot ||
      !t.cell || !t.loc || !t.hloc || !t.hw || !ps.x[0] || !ps.x[1] || !ps.f[0] || !ps.f[1] || !ps.f[2] || !ps.T ||
      !st.T0 || !st.invC0x || !ps.bar || ps.nsteps < 1 || ps.laser.volumetric || L.phase || st.has_loss)
    return cudaErrorInvalidValue;
  if (t.n_patches == 0) return cudaSuccess;
  if (L.degree == 1) return dispatch_steps<1>(L, t, ps, cap, blocks, s);
  if (L.degree == 2) return dispatch_steps<2>(L, t, ps, cap, blocks, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_step(const CellLaunch& L, const StepTables& t, const StepState& st, int cap, bool pdl,
                        cudaStream_t s) {
  // the fused form covers one instance of the FP32 operator with the constant or nodal
  // capacity, with or without the phase model and the surface loss
  if (!L.f32 || L.mesh.batch != 1 || !(cap == CAP_CONST || cap == CAP_NODAL) || !t.ptr || !t.cnt || !t.slot ||
      !t.cell || !t.hloc || !t.hw || !t.loc || !st.x_in || !st.x_out || !st.f_in || !st.f_acc || !st.f_clear ||
      !st.invC0x || st.x_in == st.x_out || st.f_in == st.f_acc || st.f_in == st.f_clear || st.f_acc == st.f_clear ||
      (L.phase && (!L.rc_in || !L.rc_f32)))  // the fused step reads and stores an FP32 history
    return cudaErrorInvalidValue;
  if (t.n_patches == 0) return cudaSuccess;
  if (L.degree == 1) return dispatch_step<1>(L, t, st, cap, pdl, s);
  if (L.degree == 2) return dispatch_step<2>(L, t, st, cap, pdl, s);
  return cudaErrorInvalidValue;
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
