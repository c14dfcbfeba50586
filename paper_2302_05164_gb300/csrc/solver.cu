// Implicit cool-down solver (paper Sec. 3.2, backward Euler; linear case) and the adjoint
// sweep of the explicit stepper. Host orchestration of the kernels in kernels_cell.cu and
// vec_kernels.cu; FP64 vectors and deterministic FP64 reductions throughout.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <cstdio>
#include <string>
#include <vector>

#include "newton.cuh"
#include "pbf.h"
#include "solver.hpp"

using namespace pbf;

struct pbf_ctx : public CtxBase {};

namespace {

pbf_status err(pbf_status s, const std::string& m) { return set_error(s, m.c_str()); }

struct Implicit {
  pbf_ctx* c;
  cudaStream_t s;
  double dt;
  int64_t n;
  CellLaunch L;
  cudaError_t e = cudaSuccess;

  Implicit(pbf_ctx* ctx, double dt_, cudaStream_t st) : c(ctx), s(st), dt(dt_), n(ctx->n_dofs) {
    L = ctx->base;
    L.mesh.batch = 1;
    L.offset = 0.0;
    L.nonlin_k = 0;
    L.latent = 0;
    L.md.m_impl = ctx->mat.rho * ctx->mat.c / dt;
    L.mf.m_impl = (float)L.md.m_impl;
  }

  // y = A x = (C/dt + K) x on free rows; x is zero on Dirichlet rows, y_D = 0
  void apply(const double* x, double* y) {
    if (e != cudaSuccess) return;
    CellLaunch La = L;
    if (c->f32) {
      e = launch_round_f32(n, x, c->Tf, s);
      La.xf = c->Tf;
      if (e == cudaSuccess) e = c->apply_cell(La, c->f, nullptr, MODE_IMPLICIT, s);
      if (e == cudaSuccess) e = launch_f32_to_f64(n, (const float*)c->f, y, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(c->f, 0, (size_t)n * 4, s);
      c->launches += 2;
    } else {
      e = cudaMemsetAsync(y, 0, (size_t)n * 8, s);
      La.x = x;
      if (e == cudaSuccess) e = c->apply_cell(La, y, nullptr, MODE_IMPLICIT, s);
    }
    if (e == cudaSuccess) e = launch_zero_masked(n, y, c->dirichlet, s);
    ++c->launches;
  }

  double dot(const double* a, const double* b) {
    double h = 0.0;
    if (e != cudaSuccess) return 0.0;
    e = launch_dot(n, 1, a, b, nullptr, nullptr, c->part, c->scal, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, c->scal, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    c->launches += 2;
    return h;
  }

  // diag(P^T A P) once per dt (Dirichlet rows 1)
  void diagonal() {
    if (e != cudaSuccess || c->diag_dt == dt) return;
    if (!c->diag) {
      e = c->dalloc_raw(&c->diag, (size_t)n);
      if (e != cudaSuccess) return;
    }
    e = cudaMemsetAsync(c->diag, 0, (size_t)std::max<int64_t>(1, n) * 8, s);
    CellLaunch Ld = L;
    Ld.f32 = 0;
    if (e == cudaSuccess) e = launch_diag(Ld, c->diag, s);
    if (e == cudaSuccess) e = launch_set_masked(n, c->diag, c->dirichlet, 1.0, s);
    c->launches += 2;
    if (e == cudaSuccess) c->diag_dt = dt;
  }

  // z = p(D^-1 A) D^-1 r: Chebyshev iteration (Saad, Iterative Methods, Alg. 12.1) from a zero
  // start with `deg` applications of A (polynomial of degree deg in D^-1 A)
  void chebyshev(const double* r, double* z, int deg, double lmin, double lmax, double* res, double* d, double* Ad) {
    if (e != cudaSuccess) return;
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
    const double sigma = theta / delta;
    double rho = 1.0 / sigma;
    e = launch_cheb_init(n, r, c->diag, 1.0 / theta, res, d, z, c->dirichlet, s);
    ++c->launches;
    for (int k = 1; k <= deg && e == cudaSuccess; ++k) {
      apply(d, Ad);
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      if (e == cudaSuccess)
        e = launch_cheb_update(n, Ad, res, d, z, c->diag, rho_new * rho, 2.0 * rho_new / delta, c->dirichlet, s);
      ++c->launches;
      rho = rho_new;
    }
  }

  // Replays the launch sequence that `body` enqueues as one CUDA graph. For a fixed key the
  // sequence is fixed, and at the sizes of an interlayer cool-down its small launches cost
  // more in launch latency than in work; it is captured once on the context's private stream
  // (the caller's stream may be the legacy default stream, which cannot be captured) and
  // replayed on the caller's stream.
  template <typename F>
  void replay(pbf_ctx::GraphSlot& g, const double* key, F body) {
    if (e != cudaSuccess) return;
    if (!g.exec || std::memcmp(key, g.key, sizeof g.key) != 0) {
      if (g.exec) {
        e = cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
        if (e != cudaSuccess) return;
      }
      if (!c->cap_stream) {
        e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return;
      }
      const long long l0 = c->launches;
      const bool timing = c->timing;
      c->timing = false;  // no event records inside a graph
      cudaStream_t user = s;
      e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        c->timing = timing;
        return;
      }
      s = c->cap_stream;
      body();
      s = user;
      cudaGraph_t graph = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(c->cap_stream, &graph);
      c->timing = timing;
      if (e == cudaSuccess) e = ec;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) return;
      g.launches = c->launches - l0;
      c->launches = l0;
      std::memcpy(g.key, key, sizeof g.key);
    }
    e = cudaGraphLaunch(g.exec, s);
    c->launches += g.launches;
  }

  // the key of the implicit solve's graphs: dt, bounds, degree and every buffer they touch
  void graph_key(double* key, int deg, double lmin, double lmax, const double* const* vecs, int nv) {
    for (int i = 0; i < CtxBase::kGraphKey; ++i) key[i] = 0.0;
    key[0] = dt;
    key[1] = lmin;
    key[2] = lmax;
    key[3] = (double)deg;
    key[4] = (double)(uintptr_t)c->diag;
    key[5] = (double)(uintptr_t)c->Tf;
    key[6] = (double)(uintptr_t)c->f;
    key[7] = (double)(uintptr_t)c->scal;
    for (int i = 0; i < nv && 8 + i < 16; ++i) key[8 + i] = (double)(uintptr_t)vecs[i];
    key[16] = (double)c->base.variant;  // the launch shape of the captured cell kernels
  }

  // z = p(D^-1 A) D^-1 r as one graph launch
  void precondition(const double* r, double* z, int deg, double lmin, double lmax, double* res, double* d,
                    double* Ad) {
    double key[CtxBase::kGraphKey];
    const double* v[] = {r, z, res, d, Ad};
    graph_key(key, deg, lmin, lmax, v, 5);
    replay(c->cheb_graph, key, [&] { chebyshev(r, z, deg, lmin, lmax, res, d, Ad); });
  }
};

// Eigenvalues of the symmetric tridiagonal matrix (diag a, off-diagonal b): the smallest
// and largest, by Sturm-sequence counts and bisection on the Gershgorin interval.
void tridiagonal_extremes(const std::vector<double>& a, const std::vector<double>& b, double* lo_out, double* hi_out) {
  const size_t k = a.size();
  double glo = a[0], ghi = a[0];
  for (size_t i = 0; i < k; ++i) {
    const double rad = (i ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(b[i]) : 0.0);
    glo = std::min(glo, a[i] - rad);
    ghi = std::max(ghi, a[i] + rad);
  }
  auto below = [&](double x) {  // number of eigenvalues < x
    int neg = 0;
    double q = a[0] - x;
    if (q < 0) ++neg;
    for (size_t i = 1; i < k; ++i) {
      if (q == 0.0) q = 1e-300;
      q = a[i] - x - b[i - 1] * b[i - 1] / q;
      if (q < 0) ++neg;
    }
    return neg;
  };
  auto kth = [&](int target) {  // eigenvalue with index target (ascending)
    double lo = glo, hi = ghi;
    for (int it = 0; it < 300 && hi - lo > 1e-15 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
      const double mid = 0.5 * (lo + hi);
      if (below(mid) > target) hi = mid;
      else lo = mid;
    }
    return 0.5 * (lo + hi);
  };
  *lo_out = kth(0);
  *hi_out = kth((int)k - 1);
}

void splitmix_vector(std::vector<double>& v, uint64_t seed) {
  // SplitMix64 (Steele, Lea, Flood 2014), mapped to [-1, 1)
  uint64_t x = seed;
  for (double& o : v) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    o = (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  }
}

// The implicit solvers run one instance without the surface loss or the phase model; the
// capacity of the backward-Euler residual is the consistent one with the plain c (the
// apparent capacity of the latent heat is not part of it). A T-dependent conductivity is
// solved by Newton's method.
pbf_status check_implicit(pbf_ctx* c) {
  if (c->batch != 1) return err(PBF_EINVAL, "the implicit solve runs one instance (batch 1)");
  return PBF_OK;
}

// Lanczos estimate from n_iter Jacobi-PCG steps on A x = b, x0 = 0 (vectors v[0..4]).
pbf_status lanczos(pbf_ctx* c, Implicit& I, const double* b_dev, int n_iter, double* out) {
  const int64_t n = I.n;
  double *r = c->vec[0], *z = c->vec[1], *p = c->vec[2], *Ap = c->vec[3], *x = c->vec[4];
  if (b_dev) {
    I.e = cudaMemcpyAsync(r, b_dev, (size_t)n * 8, cudaMemcpyDeviceToDevice, I.s);
  } else {
    std::vector<double> h((size_t)n);
    splitmix_vector(h, 0xC0FFEEull);
    I.e = cudaMemcpyAsync(r, h.data(), (size_t)n * 8, cudaMemcpyHostToDevice, I.s);
    if (I.e == cudaSuccess) I.e = cudaStreamSynchronize(I.s);
  }
  if (I.e == cudaSuccess) I.e = launch_zero_masked(n, r, c->dirichlet, I.s);
  if (I.e == cudaSuccess) I.e = cudaMemsetAsync(x, 0, (size_t)n * 8, I.s);
  I.diagonal();
  if (I.e == cudaSuccess) I.e = launch_jacobi(n, r, c->diag, z, c->dirichlet, I.s);
  if (I.e == cudaSuccess) I.e = cudaMemcpyAsync(p, z, (size_t)n * 8, cudaMemcpyDeviceToDevice, I.s);
  double rz = I.dot(r, z);
  std::vector<double> alphas, betas;
  for (int k = 0; k < n_iter && I.e == cudaSuccess && rz > 0.0; ++k) {
    I.apply(p, Ap);
    const double pAp = I.dot(p, Ap);
    const double alpha = rz / pAp;
    if (I.e == cudaSuccess) I.e = launch_axpy2(n, alpha, p, Ap, x, r, I.s);
    if (I.e == cudaSuccess) I.e = launch_jacobi(n, r, c->diag, z, c->dirichlet, I.s);
    const double rz_new = I.dot(r, z);
    const double beta = rz_new / rz;
    alphas.push_back(alpha);
    betas.push_back(beta);
    rz = rz_new;
    if (I.e == cudaSuccess) I.e = launch_xpby(n, z, beta, p, I.s);
    c->launches += 3;
  }
  if (I.e != cudaSuccess) return c->cuda(I.e, "chebyshev bounds");
  if (alphas.empty()) return err(PBF_EINVAL, "start vector vanishes on the free dofs");
  const size_t k = alphas.size();
  std::vector<double> a(k), o(k > 1 ? k - 1 : 1, 0.0);
  for (size_t i = 0; i < k; ++i) {
    a[i] = 1.0 / alphas[i] + (i ? betas[i - 1] / alphas[i - 1] : 0.0);
    if (i + 1 < k) o[i] = std::sqrt(betas[i]) / alphas[i];
  }
  tridiagonal_extremes(a, o, &out[0], &out[1]);
  return PBF_OK;
}

}  // namespace

extern "C" pbf_status pbf_cheb_bounds(pbf_ctx* ctx, double dt, const double* b_dev, int n_iter, double* out,
                                      pbf_stream stream) {
  if (!ctx || !out) return err(PBF_EINVAL, "null argument");
  if (!(dt > 0) || n_iter < 1) return err(PBF_EINVAL, "need dt > 0 and n_iter >= 1");
  pbf_status st = ctx->check_usable();
  if (st) return st;
  if ((st = check_implicit(ctx))) return st;
  if ((st = ctx->ensure_vectors(5))) return st;
  Implicit I(ctx, dt, (cudaStream_t)stream);
  return lanczos(ctx, I, b_dev, n_iter, out);
}

extern "C" pbf_status pbf_implicit_solve(pbf_ctx* ctx, double* T_dev, double dt, int nsteps, double rtol, int max_it,
                                         int cheb_degree, const double* cheb_bounds, int* iters_out,
                                         pbf_stream stream) {
  if (!ctx || !T_dev) return err(PBF_EINVAL, "null argument");
  if (!(dt > 0) || nsteps < 0 || !(rtol > 0) || max_it < 1 || cheb_degree < 0 || cheb_degree > 64)
    return err(PBF_EINVAL, "bad solver parameters");
  pbf_status st = ctx->check_usable();
  if (st) return st;
  if ((st = check_implicit(ctx))) return st;
  if (ctx->nonlin || ctx->has_phase || ctx->has_loss)  // Newton's method (iters_out: BiCGStab iterations)
    return pbf_implicit_newton(ctx, T_dev, dt, nsteps, rtol, 50, 1e-4, max_it, cheb_degree, cheb_bounds, nullptr,
                               iters_out, nullptr, stream);
  if ((st = ctx->ensure_vectors(8))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  Implicit I(ctx, dt, s);
  double bounds[2];
  if (cheb_bounds) {
    bounds[0] = cheb_bounds[0];
    bounds[1] = cheb_bounds[1];
  } else {
    if ((st = lanczos(ctx, I, nullptr, 30, bounds))) return st;
    bounds[1] *= 1.1;
  }
  if (!(bounds[1] > bounds[0]) || !(bounds[0] > 0)) return err(PBF_EINVAL, "need 0 < lmin < lmax");
  I.diagonal();
  const int64_t n = ctx->n_dofs;
  double *r = ctx->vec[0], *z = ctx->vec[1], *p = ctx->vec[2], *Ap = ctx->vec[3], *x = ctx->vec[4];
  double *res = ctx->vec[5], *d = ctx->vec[6], *Ad = ctx->vec[7];
  // right-hand side f(T_n) = -K T_n in FP64 (no laser during the cool-down)
  CellLaunch Ls = ctx->base;
  Ls.mesh.batch = 1;
  Ls.f32 = 0;
  Ls.nonlin_k = 0;
  Ls.latent = 0;
  Ls.offset = 0.0;
  bool converged = true;
  for (int step = 0; step < nsteps && I.e == cudaSuccess; ++step) {
    I.e = cudaMemsetAsync(r, 0, (size_t)n * 8, s);
    Ls.x = T_dev;
    if (I.e == cudaSuccess) I.e = ctx->apply_cell(Ls, r, nullptr, MODE_STIFF, s);
    if (I.e == cudaSuccess) I.e = launch_neg_masked(n, r, ctx->dirichlet, s);
    if (I.e == cudaSuccess) I.e = cudaMemsetAsync(x, 0, (size_t)n * 8, s);
    ctx->launches += 1;
    const double r0 = std::sqrt(I.dot(r, r));
    double rn = r0;
    int it = 0;
    if (r0 > 0.0) {
      // the CG scalars stay on the device (rz in sc[4], the new r.z in sc[6], p.Ap in sc[5],
      // r.r in sc[0]); the host reads r.r once per iteration for the stopping test
      double* sc = ctx->scal;
      double* const rz = sc + 4;
      double* const rz_new = sc + 6;
      I.precondition(r, z, cheb_degree, bounds[0], bounds[1], res, d, Ad);
      if (I.e == cudaSuccess) I.e = cudaMemcpyAsync(p, z, (size_t)n * 8, cudaMemcpyDeviceToDevice, s);
      if (I.e == cudaSuccess) I.e = launch_dot(n, 1, r, z, nullptr, nullptr, ctx->part, rz, s);
      ctx->launches += 2;
      // first iteration with separate launches; the following ones, preconditioner and
      // search direction of iteration k followed by the update of iteration k + 1, as one
      // graph launch and one host round trip (r.r into page-locked memory)
      if (!ctx->pinned && I.e == cudaSuccess) I.e = cudaMallocHost(&ctx->pinned, sizeof(double));
      auto update = [&] {  // x += alpha p, r -= alpha Ap, alpha = rz / p.Ap; sc[0] = r.r
        I.apply(p, Ap);
        if (I.e == cudaSuccess) I.e = launch_dot(n, 1, p, Ap, nullptr, nullptr, ctx->part, sc + 5, I.s);
        if (I.e == cudaSuccess) I.e = launch_axpy2_dev(n, rz, sc + 5, p, Ap, x, r, I.s);
        if (I.e == cudaSuccess) I.e = launch_dot(n, 1, r, r, nullptr, nullptr, ctx->part, sc, I.s);
        if (I.e == cudaSuccess) I.e = cudaMemcpyAsync(ctx->pinned, sc, sizeof(double), cudaMemcpyDeviceToHost, I.s);
        ctx->launches += 5;
      };
      auto direction = [&] {  // z = M^-1 r, beta = r.z / rz, p = z + beta p, rz = r.z
        I.chebyshev(r, z, cheb_degree, bounds[0], bounds[1], res, d, Ad);
        if (I.e == cudaSuccess) I.e = launch_dot(n, 1, r, z, nullptr, nullptr, ctx->part, rz_new, I.s);
        if (I.e == cudaSuccess) I.e = launch_xpby_dev(n, z, rz_new, rz, p, I.s);
        if (I.e == cudaSuccess) I.e = cudaMemcpyAsync(rz, rz_new, sizeof(double), cudaMemcpyDeviceToDevice, I.s);
        ctx->launches += 3;
      };
      double key[CtxBase::kGraphKey];
      const double* kv[] = {r, z, p, Ap, x, res, d, Ad};
      I.graph_key(key, cheb_degree, bounds[0], bounds[1], kv, 8);
      bool first = true;
      while (rn > rtol * r0 && it < max_it && I.e == cudaSuccess) {
        if (first) {
          update();
          first = false;
        } else {
          I.replay(ctx->iter_graph, key, [&] {
            direction();
            update();
          });
        }
        if (I.e == cudaSuccess) I.e = cudaStreamSynchronize(s);
        if (I.e != cudaSuccess) break;
        ++it;
        rn = std::sqrt(*ctx->pinned);
      }
    }
    if (rn > rtol * r0) converged = false;
    if (iters_out) iters_out[step] = it;
    if (I.e == cudaSuccess) I.e = launch_add(n, T_dev, x, s);
    ++ctx->launches;
  }
  if (I.e != cudaSuccess) return ctx->cuda(I.e, "implicit_solve");
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ctx->cuda(e, "implicit_solve");
  return converged ? PBF_OK : err(PBF_ENOCONV, "CG missed the tolerance within max_it");
}

// ======================================================================================
// Nonlinear backward Euler by Newton-Raphson (Sec. 3.2, Eqs. backward_euler_nonlinear,
// Newton_1, Newton_2): from T^0 = T_n (Dirichlet dofs set to T_D), solve J(T^i) dT = -r(T^i)
// by BiCGStab preconditioned with the Chebyshev-Jacobi polynomial of the linear operator
// C/dt + K(k0), set T^{i+1} = T^i + dT, until ||r(T^i)||_2 <= newton_rtol ||r(T^0)||_2. The
// residual is always evaluated in FP64; the Jacobian in the context's operator precision, so
// that for an FP32-operator context the iteration is an FP64 iterative refinement of FP32
// linear solves and converges to the FP64 solution.
// ======================================================================================
namespace {

struct Newton {
  pbf_ctx* c;
  Implicit& I;
  int64_t n;
  CellLaunch Lr, Lj;  // residual (FP64) and Jacobian (operator precision) launches
  double* T = nullptr;
  double* diff = nullptr;
  double* fre = nullptr;  // f_RE(T_n), the surface loss at the previous state (null: none)

  Newton(pbf_ctx* ctx, Implicit& imp, double dt) : c(ctx), I(imp), n(ctx->n_dofs) {
    Lj = ctx->base;
    Lj.mesh.batch = 1;
    Lj.offset = ctx->mat.T_ref;
    Lj.nonlin_k = ctx->nonlin ? 1 : 0;
    Lj.latent = 0;
    Lj.md.m_impl = ctx->mat.rho * ctx->mat.c / dt;
    Lj.mf.m_impl = (float)Lj.md.m_impl;
    ctx->set_phase(Lj, false);  // the stored history is read, not changed, while iterating
    Lr = Lj;
    Lr.f32 = 0;
  }

  // fre = f_RE(Tn): the radiation / evaporation term at the previous state (Eq.
  // backward_euler_nonlinear evaluates it there)
  void surface_loss(const double* Tn) {
    if (I.e != cudaSuccess || !fre) return;
    I.e = cudaMemsetAsync(fre, 0, (size_t)n * 8, I.s);
    if (I.e == cudaSuccess)
      I.e = launch_surface_loss(c->degree, false, c->lsetup, Lr.mesh, Tn, 0.0, c->loss, fre, I.s);
    ++c->launches;
  }

  // R = r(T) on free dofs, 0 on Dirichlet dofs (Tn: the state of the previous step)
  void residual(const double* Tn, double* R) {
    if (I.e != cudaSuccess) return;
    I.e = launch_sub(n, T, Tn, diff, I.s);
    if (I.e == cudaSuccess) I.e = cudaMemsetAsync(R, 0, (size_t)n * 8, I.s);
    if (I.e == cudaSuccess) I.e = launch_newton(Lr, false, T, diff, R, I.s);
    if (I.e == cudaSuccess && fre) I.e = launch_sub(n, R, fre, R, I.s);
    if (I.e == cudaSuccess) I.e = launch_zero_masked(n, R, c->dirichlet, I.s);
    c->launches += fre ? 4 : 3;
  }

  // the history of the converged state: r_c = max(r_c, g(T)) at every quadrature point (a
  // residual pass that stores it; its vector goes to scratch)
  void store_history(const double* Tn, double* scratch) {
    if (I.e != cudaSuccess || !c->has_phase) return;
    CellLaunch Ls = Lr;
    c->set_phase(Ls, true);
    I.e = launch_sub(n, T, Tn, diff, I.s);
    if (I.e == cudaSuccess) I.e = cudaMemsetAsync(scratch, 0, (size_t)n * 8, I.s);
    if (I.e == cudaSuccess) I.e = launch_newton(Ls, false, T, diff, scratch, I.s);
    c->launches += 2;
  }

  // y = J(T) w, identity rows on Dirichlet dofs
  void jacobian(const double* w, double* y) {
    if (I.e != cudaSuccess) return;
    I.e = cudaMemsetAsync(y, 0, (size_t)n * 8, I.s);
    if (I.e == cudaSuccess) I.e = launch_newton(Lj, true, T, w, y, I.s);
    if (I.e == cudaSuccess) I.e = launch_copy_masked(n, y, w, c->dirichlet, I.s);
    c->launches += 2;
  }

  double host_scalar(const double* dev) {
    double h = 0.0;
    if (I.e == cudaSuccess) I.e = cudaMemcpyAsync(&h, dev, 8, cudaMemcpyDeviceToHost, I.s);
    if (I.e == cudaSuccess) I.e = cudaStreamSynchronize(I.s);
    return h;
  }

  // BiCGStab for J x = b from x = 0 (van der Vorst 1992, preconditioned form); the scalars
  // stay in device memory, the host reads s.s and r.r for the stopping tests. b is used as
  // the residual vector r and is overwritten. Returns the iterations used.
  int bicgstab(double* b, double* x, double rtol, int max_it, int deg, const double* bounds, double* const* w) {
    double *rh = w[0], *p = w[1], *v = w[2], *sv = w[3], *t = w[4], *y = w[5], *z = w[6];
    double *res = w[7], *d = w[8], *Ad = w[9];
    double* sc = c->scal;
    double* r = b;
    const double bn = std::sqrt(I.dot(r, r));
    if (I.e == cudaSuccess) I.e = cudaMemsetAsync(x, 0, (size_t)n * 8, I.s);
    if (!(bn > 0.0) || I.e != cudaSuccess) return 0;
    const double one[3] = {1.0, 1.0, 1.0};
    I.e = cudaMemcpyAsync(rh, r, (size_t)n * 8, cudaMemcpyDeviceToDevice, I.s);
    if (I.e == cudaSuccess) I.e = cudaMemsetAsync(p, 0, (size_t)n * 8, I.s);
    if (I.e == cudaSuccess) I.e = cudaMemsetAsync(v, 0, (size_t)n * 8, I.s);
    if (I.e == cudaSuccess) I.e = cudaMemcpyAsync(sc + kScRho, one, 8, cudaMemcpyHostToDevice, I.s);
    if (I.e == cudaSuccess) I.e = cudaMemcpyAsync(sc + kScAlpha, one + 1, 8, cudaMemcpyHostToDevice, I.s);
    if (I.e == cudaSuccess) I.e = cudaMemcpyAsync(sc + kScOmega, one + 2, 8, cudaMemcpyHostToDevice, I.s);
    int it = 0;
    while (it < max_it && I.e == cudaSuccess) {
      ++it;
      I.e = launch_dot(n, 1, rh, r, nullptr, nullptr, c->part, sc + kScRhoNew, I.s);
      if (I.e == cudaSuccess) I.e = launch_bicg_p(n, p, r, v, sc, I.s);
      I.chebyshev(p, y, deg, bounds[0], bounds[1], res, d, Ad);
      jacobian(y, v);
      if (I.e == cudaSuccess) I.e = launch_dot(n, 1, rh, v, nullptr, nullptr, c->part, sc + kScRhv, I.s);
      if (I.e == cudaSuccess) I.e = launch_bicg_s(n, sv, r, v, x, y, sc, I.s);
      if (I.e == cudaSuccess) I.e = launch_dot(n, 1, sv, sv, nullptr, nullptr, c->part, sc + kScSs, I.s);
      c->launches += 5;
      const double sn = std::sqrt(host_scalar(sc + kScSs));
      if (!(sn > rtol * bn)) break;  // converged (or not a number: the caller's test fails)
      I.chebyshev(sv, z, deg, bounds[0], bounds[1], res, d, Ad);
      jacobian(z, t);
      if (I.e == cudaSuccess) I.e = launch_dot(n, 1, t, sv, nullptr, nullptr, c->part, sc + kScTs, I.s);
      if (I.e == cudaSuccess) I.e = launch_dot(n, 1, t, t, nullptr, nullptr, c->part, sc + kScTt, I.s);
      if (I.e == cudaSuccess) I.e = launch_bicg_x(n, x, z, r, sv, t, sc, I.s);
      if (I.e == cudaSuccess) I.e = launch_dot(n, 1, r, r, nullptr, nullptr, c->part, sc + kScRr, I.s);
      c->launches += 7;
      const double rn = std::sqrt(host_scalar(sc + kScRr));
      if (!(rn > rtol * bn)) break;
    }
    return it;
  }
};

}  // namespace

extern "C" pbf_status pbf_implicit_newton(pbf_ctx* ctx, double* T_dev, double dt, int nsteps, double newton_rtol,
                                          int newton_max, double lin_rtol, int lin_max, int cheb_degree,
                                          const double* cheb_bounds, int* newton_iters_out, int* lin_iters_out,
                                          double* rel_residual_out, pbf_stream stream) {
  if (!ctx || !T_dev) return err(PBF_EINVAL, "null argument");
  if (!(dt > 0) || nsteps < 0 || !(newton_rtol > 0) || newton_max < 1 || !(lin_rtol > 0) || lin_max < 1 ||
      cheb_degree < 0 || cheb_degree > 64)
    return err(PBF_EINVAL, "bad solver parameters");
  pbf_status st = ctx->check_usable();
  if (st) return st;
  if ((st = check_implicit(ctx))) return st;
  if ((st = ctx->ensure_vectors(16))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  Implicit I(ctx, dt, s);
  double bounds[2];
  if (cheb_bounds) {
    bounds[0] = cheb_bounds[0];
    bounds[1] = cheb_bounds[1];
  } else {
    if ((st = lanczos(ctx, I, nullptr, 30, bounds))) return st;
    bounds[1] *= 1.1;
  }
  if (!(bounds[1] > bounds[0]) || !(bounds[0] > 0)) return err(PBF_EINVAL, "need 0 < lmin < lmax");
  I.diagonal();
  const int64_t n = ctx->n_dofs;
  double* const* v = ctx->vec.data();
  Newton N(ctx, I, dt);
  N.T = T_dev;
  N.diff = v[10];
  N.fre = ctx->has_loss ? v[15] : nullptr;
  double *Tn = v[11], *R = v[12], *b = v[13], *x = v[14];
  bool converged = true;
  double worst = 0.0;
  for (int step = 0; step < nsteps && I.e == cudaSuccess; ++step) {
    I.e = cudaMemcpyAsync(Tn, T_dev, (size_t)n * 8, cudaMemcpyDeviceToDevice, s);
    if (I.e == cudaSuccess) I.e = launch_set_masked(n, T_dev, ctx->dirichlet, ctx->mat.T_dirichlet, s);
    ctx->launches += 1;
    N.surface_loss(Tn);
    N.residual(Tn, R);
    const double r0 = std::sqrt(I.dot(R, R));
    double rn = r0;
    int it = 0, lin = 0;
    bool done = !(rn > newton_rtol * r0);
    while (!done && it < newton_max && I.e == cudaSuccess) {
      I.e = cudaMemcpyAsync(b, R, (size_t)n * 8, cudaMemcpyDeviceToDevice, s);
      if (I.e == cudaSuccess) I.e = launch_neg_masked(n, b, ctx->dirichlet, s);
      ctx->launches += 1;
      lin += N.bicgstab(b, x, lin_rtol, lin_max, cheb_degree, bounds, v);
      if (I.e == cudaSuccess) I.e = launch_add(n, T_dev, x, s);
      ++ctx->launches;
      ++it;
      N.residual(Tn, R);
      rn = std::sqrt(I.dot(R, R));
      // converged: the residual criterion, or a correction at the rounding level of T
      const double xn = std::sqrt(I.dot(x, x)), tn = std::sqrt(I.dot(T_dev, T_dev));
      done = !(rn > newton_rtol * r0) || xn <= 1e-13 * tn;
    }
    if (!done) converged = false;
    N.store_history(Tn, b);
    if (r0 > 0.0) worst = std::max(worst, rn / r0);
    if (!(rn == rn)) worst = rn;
    if (newton_iters_out) newton_iters_out[step] = it;
    if (lin_iters_out) lin_iters_out[step] = lin;
  }
  if (I.e != cudaSuccess) return ctx->cuda(I.e, "implicit_newton");
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ctx->cuda(e, "implicit_newton");
  if (rel_residual_out) *rel_residual_out = worst;
  return converged ? PBF_OK : err(PBF_ENOCONV, "Newton missed the tolerance within newton_max corrections");
}

// ======================================================================================
// Binomial checkpointing (Griewank and Walther, "revolve"): the fewest forward steps F(l, s)
// needed to reverse l steps from a stored state with s free snapshot slots, and the split
// that attains it: F(l, s) = min_m [ m + F(l - m, s - 1) + F(m, s) ], F(1, s) = 0,
// F(l, 0) = l (l - 1) / 2. With c stored states including the initial one, F(l, c - 1)
// equals the closed form r l - beta(c + 1, r - 1), beta(c, r) = C(c + r, c).
// ======================================================================================
namespace {

struct Revolve {
  int L = 0, S = 0;
  std::vector<long long> cost;  // [(S+1) x (L+1)]
  std::vector<int> split;
  long long F(int l, int s) const { return cost[(size_t)s * (L + 1) + l]; }
  int M(int l, int s) const { return split[(size_t)s * (L + 1) + l]; }
  void build(int l_max, int s_max) {
    L = l_max;
    S = s_max;
    cost.assign((size_t)(S + 1) * (L + 1), 0);
    split.assign((size_t)(S + 1) * (L + 1), 0);
    for (int l = 2; l <= L; ++l) cost[l] = (long long)l * (l - 1) / 2;
    for (int s = 1; s <= S; ++s)
      for (int l = 2; l <= L; ++l) {
        long long best = -1;
        int arg = 1;
        for (int m = 1; m < l; ++m) {
          const long long c = m + F(l - m, s - 1) + F(m, s);
          if (best < 0 || c < best) {
            best = c;
            arg = m;
          }
        }
        cost[(size_t)s * (L + 1) + l] = best;
        split[(size_t)s * (L + 1) + l] = arg;
      }
  }
};

struct Adjoint {
  pbf_ctx* c;
  cudaStream_t s;
  const pbf_laser* laser;
  double t0, dt, Tt, p;
  int N, B, n_seg;
  int64_t nv;
  Revolve rv;
  long long fwd = 0;
  cudaError_t e = cudaSuccess;
  // device buffers
  std::vector<double*> slots;
  double *lam = nullptr, *v = nullptr, *mu = nullptr, *q1 = nullptr, *q2 = nullptr, *fd = nullptr, *fv = nullptr,
         *Cm = nullptr, *work = nullptr, *J = nullptr, *coef = nullptr, *grad = nullptr, *scal = nullptr;
  double* fre = nullptr;  // the surface loss's part of f (with a surface loss)
  float *vf = nullptr, *muf = nullptr;
  void *vh = nullptr, *muh = nullptr;
  // phase model: the history at each snapshot (beside slots) and the history's adjoint
  bool ph = false;
  size_t hbytes = 0;
  std::vector<char*> hslots;
  char* sig = nullptr;
  std::vector<void*> owned;

  template <typename X>
  void alloc(X** ptr, size_t n) {
    if (e != cudaSuccess) return;
    void* q = nullptr;
    e = cudaMalloc(&q, std::max<size_t>(1, n) * sizeof(X));
    if (e == cudaSuccess) {
      owned.push_back(q);
      *ptr = (X*)q;
    }
  }
  ~Adjoint() {
    for (void* q : owned) cudaFree(q);
  }

  void copy(double* dst, const double* src) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, (size_t)nv * 8, cudaMemcpyDeviceToDevice, s);
  }
  // the context's live history to / from the snapshot kept beside `slot` (phase model)
  char* hist_of(const double* slot) {
    for (size_t i = 0; i < slots.size(); ++i)
      if (slots[i] == slot) return hslots[i];
    return nullptr;
  }
  void put_hist(const double* slot) {
    if (ph && e == cudaSuccess) e = cudaMemcpyAsync(hist_of(slot), c->rc, hbytes, cudaMemcpyDeviceToDevice, s);
  }
  void get_hist(const double* slot) {
    if (ph && e == cudaSuccess) e = cudaMemcpyAsync(c->rc, hist_of(slot), hbytes, cudaMemcpyDeviceToDevice, s);
  }
  // advance T from step k by m steps
  void advance(double* T, int k, int m) {
    if (e == cudaSuccess && m > 0) e = c->explicit_steps(T, t0 + k * dt, dt, m, s);
    fwd += m;
  }
  void objective(const double* T, int accumulate) {
    if (e == cudaSuccess)
      e = launch_objective(c->n_surf, B, c->surf_idx, c->surf_w, T, c->surf_W, p, Tt, 1.0 / N, accumulate, c->part, J,
                           coef, s);
    c->launches += 2;
  }
  void add_objective_gradient(const double* T) {
    objective(T, 0);
    if (e == cudaSuccess) e = launch_lambda_objective(c->n_surf, B, c->surf_idx, c->surf_w, T, p, coef, c->dirichlet, lam, s);
    ++c->launches;
  }
  // lambda_{k+1} -> lambda_k at the state T_k
  void adjoint_step(int k, const double* Tk) {
    if (e != cudaSuccess) return;
    const double t = t0 + k * dt;
    // f_vol without the surface loss (fre): the power gradients take the laser's part alone
    e = c->residual_f64(Tk, t, fd, fv, Cm, s, fre);
    if (e == cudaSuccess)
      e = launch_adj_prepare((int)c->n_dofs, B, lam, fd, fv, fre, Cm, c->dirichlet, v, mu, q1, q2, s);
    // parameter gradients with lambda_{k+1}
    if (e == cudaSuccess) e = launch_dot(c->n_dofs, B, lam, q1, nullptr, nullptr, c->part, scal, s);
    if (e == cudaSuccess) e = launch_dot(c->n_dofs, B, lam, q2, nullptr, nullptr, c->part, scal + B, s);
    const Spot sp = spot_at(c->lsetup.k, t);
    if (e == cudaSuccess) e = launch_grad_accum(B, n_seg, sp.seg, scal, scal + B, c->k_scale_d, c->power, dt, grad, s);
    // transposed linearisation (with the phase model: the history entering step k, read only,
    // and the history's adjoint)
    CellLaunch L = c->base;
    c->set_phase(L, false);
    L.sig = sig;
    const bool qpc = c->cap == CAP_QUADRATURE;
    if (c->f32) {
      if (e == cudaSuccess) e = launch_prepare_f32(nv, Tk, c->mat.T_ref, c->Tf, nullptr, s);
      if (e == cudaSuccess) e = launch_round_f32(nv, v, vf, s);
      if (e == cudaSuccess && qpc) e = launch_round_f32(nv, mu, muf, s);
      L.xf = c->Tf;
      L.vf = vf;
      L.muf = muf;
    } else {
      L.x = Tk;
      L.v = v;
      L.mu = mu;
    }
    const bool f32 = c->f32;
    if (e == cudaSuccess) e = launch_hang_values(f32, L.mesh, f32 ? (const void*)L.xf : (const void*)L.x, c->xh, s);
    if (e == cudaSuccess) e = launch_hang_values(f32, L.mesh, f32 ? (const void*)L.vf : (const void*)L.v, vh, s);
    if (e == cudaSuccess && qpc) e = launch_hang_values(f32, L.mesh, f32 ? (const void*)L.muf : (const void*)L.mu, muh, s);
    if (f32) {
      L.xfh = (const float*)c->xh;
      L.vfh = (const float*)vh;
      L.mufh = (const float*)muh;
    } else {
      L.xh = (const double*)c->xh;
      L.vh = (const double*)vh;
      L.muh = (const double*)muh;
    }
    if (e == cudaSuccess) e = launch_adjoint(L, qpc, c->f, c->fh, s);
    if (e == cudaSuccess) e = launch_hang_distribute(f32, L.mesh, c->fh, c->f, s);
    if (e == cudaSuccess && c->has_loss) {  // the loss's face term at the state T_k
      e = launch_surface_loss_adjoint(c->degree, f32, c->lsetup, L.mesh, f32 ? (const void*)c->Tf : (const void*)Tk,
                                      f32 ? c->mat.T_ref : 0.0, f32 ? (const void*)vf : (const void*)v, c->loss,
                                      c->f, s);
      ++c->launches;
    }
    if (e == cudaSuccess)
      e = launch_lambda_update(f32, c->cap == CAP_NODAL, (int)c->n_dofs, B, lam, c->f, mu, c->C0, Tk, c->nodal,
                               c->dirichlet, dt, s);
    c->launches += 12;
    if (k > 0) add_objective_gradient(Tk);
  }
  // reverse steps [a, b) with T_a in `slot` and `free` unused snapshot slots (free_base..)
  void reverse(int a, int b, double* slot, int free, int free_base) {
    if (e != cudaSuccess) return;
    const int l = b - a;
    if (l == 1) {
      get_hist(slot);
      adjoint_step(a, slot);
      return;
    }
    if (free == 0) {
      for (int k = b - 1; k >= a && e == cudaSuccess; --k) {
        copy(work, slot);
        get_hist(slot);
        advance(work, a, k - a);
        adjoint_step(k, work);
      }
      return;
    }
    const int m = rv.M(l, free);
    double* mid = slots[(size_t)free_base];
    copy(mid, slot);
    get_hist(slot);
    advance(mid, a, m);
    put_hist(mid);
    reverse(a + m, b, mid, free - 1, free_base + 1);
    reverse(a, a + m, slot, free, free_base);
  }
};

pbf_status ensure_surface(pbf_ctx* c, cudaStream_t s) {
  if (c->surf_idx) return PBF_OK;
  double* w = nullptr;
  cudaError_t e = c->dalloc_raw(&w, (size_t)c->n_dofs);
  if (e == cudaSuccess) e = cudaMemsetAsync(w, 0, (size_t)std::max<int64_t>(1, c->n_dofs) * 8, s);
  CellLaunch L = c->base;
  if (e == cudaSuccess) e = launch_surface_weights(c->degree, (int)c->n_top, c->top_cell, c->top_geo, L.mesh, w, s);
  std::vector<double> h((size_t)c->n_dofs);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), w, h.size() * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return c->cuda(e, "surface weights");
  std::vector<int32_t> idx;
  std::vector<double> sw;
  double W = 0.0;
  for (size_t i = 0; i < h.size(); ++i)
    if (h[i] != 0.0) {
      idx.push_back((int32_t)i);
      sw.push_back(h[i]);
      W += h[i];
    }
  if (idx.empty()) return err(PBF_EINVAL, "the mesh has no top surface");
  double* dw = nullptr;
  e = c->dalloc_raw(&dw, sw.size());
  void* di = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&di, idx.size() * 4);
  if (e == cudaSuccess) c->allocs.push_back(di);
  if (e == cudaSuccess) e = cudaMemcpy(dw, sw.data(), sw.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(di, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return c->cuda(e, "surface weights");
  c->surf_idx = (int32_t*)di;
  c->surf_w = dw;
  c->n_surf = (int)idx.size();
  c->surf_W = W;
  return PBF_OK;
}

}  // namespace

extern "C" pbf_status pbf_revolve_cost(int nsteps, int n_snaps, long long* forward_steps_out) {
  if (nsteps < 1 || n_snaps < 1 || !forward_steps_out) return err(PBF_EINVAL, "need nsteps >= 1, n_snaps >= 1");
  if ((long long)nsteps * nsteps * std::min(n_snaps, nsteps) > 4000000000LL) return err(PBF_EINVAL, "schedule too large");
  Revolve r;
  const int S = std::min(n_snaps - 1, nsteps);
  r.build(nsteps, S);
  *forward_steps_out = r.F(nsteps, S);
  return PBF_OK;
}

extern "C" pbf_status pbf_adjoint_sweep(pbf_ctx* ctx, const double* T0_dev, const pbf_laser* laser, double t0,
                                        double dt, int nsteps, int n_checkpoints, double T_target, double p_exp,
                                        double* J_out, double* grad_out, long long* forward_steps_out,
                                        pbf_stream stream) {
  if (!ctx || !T0_dev || !laser || !J_out || !grad_out) return err(PBF_EINVAL, "null argument");
  if (nsteps < 1 || n_checkpoints < 1 || !(dt > 0) || !(p_exp >= 1)) return err(PBF_EINVAL, "bad sweep parameters");
  if (laser->n_seg < 1) return err(PBF_EINVAL, "the adjoint needs a laser with at least one segment");
  pbf_status st = ctx->check_usable();
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = ctx->set_laser(laser, s))) return st;
  if ((st = ensure_surface(ctx, s))) return st;
  Adjoint A;
  A.c = ctx;
  A.s = s;
  A.laser = laser;
  A.t0 = t0;
  A.dt = dt;
  A.Tt = T_target;
  A.p = p_exp;
  A.N = nsteps;
  A.B = ctx->batch;
  A.n_seg = laser->n_seg;
  A.nv = ctx->n_dofs * ctx->batch;
  const int free_slots = std::min(n_checkpoints - 1, nsteps);
  A.rv.build(nsteps, free_slots);
  const size_t nv = (size_t)A.nv, nh = std::max<size_t>(1, (size_t)ctx->n_hang * ctx->batch);
  const size_t rsz = ctx->f32 ? 4 : 8;
  A.slots.resize((size_t)free_slots + 1);
  for (auto& sl : A.slots) A.alloc(&sl, nv);
  if (ctx->has_phase) {  // the history travels with every snapshot; its adjoint starts at zero
    const int p1 = ctx->degree + 1;
    A.ph = true;
    A.hbytes = (size_t)p1 * p1 * p1 * (size_t)ctx->n_cells * (size_t)ctx->batch * rsz;
    A.hslots.resize(A.slots.size());
    for (auto& hs : A.hslots) A.alloc(&hs, A.hbytes);
    A.alloc(&A.sig, A.hbytes);
    if (A.e == cudaSuccess) A.e = cudaMemsetAsync(A.sig, 0, A.hbytes, s);
  }
  A.alloc(&A.lam, nv);
  A.alloc(&A.v, nv);
  A.alloc(&A.mu, nv);
  A.alloc(&A.q1, nv);
  A.alloc(&A.q2, nv);
  A.alloc(&A.fd, nv);
  A.alloc(&A.fv, nv);
  A.alloc(&A.Cm, nv);
  A.alloc(&A.work, nv);
  if (ctx->has_loss) A.alloc(&A.fre, nv);
  A.alloc(&A.J, (size_t)A.B);
  A.alloc(&A.coef, (size_t)A.B);
  A.alloc(&A.grad, (size_t)A.B * (A.n_seg + 1));
  A.alloc(&A.scal, (size_t)A.B * 2);
  A.alloc(&A.vf, nv);
  A.alloc(&A.muf, nv);
  A.alloc((char**)&A.vh, nh * rsz);
  A.alloc((char**)&A.muh, nh * rsz);
  if (A.e != cudaSuccess) {
    cudaGetLastError();
    return err(A.e == cudaErrorMemoryAllocation ? PBF_ENOMEM : PBF_ECUDA, "adjoint work space");
  }
  if (A.e == cudaSuccess) A.e = cudaMemsetAsync(A.J, 0, (size_t)A.B * 8, s);
  if (A.e == cudaSuccess) A.e = cudaMemsetAsync(A.grad, 0, (size_t)A.B * (A.n_seg + 1) * 8, s);
  if (A.e == cudaSuccess) A.e = cudaMemsetAsync(A.lam, 0, nv * 8, s);
  // forward sweep along the right spine of the schedule: store its snapshots, accumulate J
  double* start = A.slots[0];
  A.copy(start, T0_dev);
  A.put_hist(start);  // the history at T0 (restored on return)
  struct Node { int a; double* slot; int free; int base; };
  std::vector<Node> spine;
  int a = 0, free = free_slots, base = 1;
  double* cur = start;
  A.copy(A.work, start);
  while (A.e == cudaSuccess && nsteps - a > 1 && free > 0) {
    spine.push_back({a, cur, free, base});
    const int m = A.rv.M(nsteps - a, free);
    double* nxt = A.slots[(size_t)base];
    for (int k = 0; k < m && A.e == cudaSuccess; ++k) {
      A.advance(A.work, a + k, 1);
      A.objective(A.work, 1);
    }
    A.copy(nxt, A.work);
    A.put_hist(nxt);
    a += m;
    cur = nxt;
    --free;
    ++base;
  }
  // rest of the sweep to T_N: objective terms and lambda_N
  for (int k = a; k < nsteps && A.e == cudaSuccess; ++k) {
    A.advance(A.work, k, 1);
    A.objective(A.work, 1);
  }
  A.add_objective_gradient(A.work);
  // reverse: the innermost spine segment first, then the left parts outward
  A.reverse(a, nsteps, cur, free, base);
  for (int i = (int)spine.size() - 1; i >= 0 && A.e == cudaSuccess; --i) {
    const int b = (i + 1 < (int)spine.size()) ? spine[(size_t)i + 1].a : a;
    A.reverse(spine[(size_t)i].a, b, spine[(size_t)i].slot, spine[(size_t)i].free, spine[(size_t)i].base);
  }
  A.get_hist(start);  // the context's history as it was on entry
  if (A.e == cudaSuccess) A.e = cudaMemcpyAsync(J_out, A.J, (size_t)A.B * 8, cudaMemcpyDeviceToHost, s);
  if (A.e == cudaSuccess)
    A.e = cudaMemcpyAsync(grad_out, A.grad, (size_t)A.B * (A.n_seg + 1) * 8, cudaMemcpyDeviceToHost, s);
  if (A.e == cudaSuccess) A.e = cudaStreamSynchronize(s);
  if (A.e != cudaSuccess) return ctx->cuda(A.e, "adjoint_sweep");
  if (forward_steps_out) *forward_steps_out = A.fwd;
  return PBF_OK;
}
