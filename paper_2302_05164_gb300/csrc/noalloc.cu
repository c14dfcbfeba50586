// pbf_estimate_dt_noalloc: the critical-time-step power iteration of pbf_estimate_dt for
// callers that must not allocate device memory during the call: applications that reserve
// almost all device memory up front for their own pool allocator (a cudaMalloc would fail or
// fragment that pool), and latency-bound loops where cudaMalloc / cudaFree would stall the
// device. The caller passes the vectors; the only scratch the iteration needs, the partial
// sums of its deterministic FP64 reductions, lives in a fixed file-scope device array.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "pbf.h"
#include "solver.hpp"

using namespace pbf;

struct pbf_ctx : public CtxBase {};

namespace {

constexpr int kChunk = 4096;                 // dofs reduced by one block, in a fixed order
constexpr int kMaxPartials = 32768;          // => at most 134,217,728 dofs
constexpr int kScalars = 64;
constexpr int kScratchDoubles = kMaxPartials + kScalars;  // 262,656 bytes per device

// Shared by every call on a device and kept until the process exits; the contents of the
// last call stay behind. Each call overwrites every partial and scalar it reads before
// reading it, so nothing has to start at zero. Calls whose work overlaps on the GPU (two
// streams, or two host threads) race on this array.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the array for the current device, looked up once per device. In host
// code the array's name only stands in for it and must never be handed to a kernel.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// part[b] = sum over dofs [b kChunk, (b+1) kChunk) of w x y (w may be null), fixed order
__global__ void k_chunk_dot(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                            const double* __restrict__ w, double* __restrict__ part) {
  __shared__ double sh[256];
  const int64_t lo = (int64_t)blockIdx.x * kChunk, hi = min(n, lo + kChunk);
  double s = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += w ? w[i] * x[i] * y[i] : x[i] * y[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_chunk_final(int nblk, const double* __restrict__ part, double* __restrict__ out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += part[k];
    *out = s;
  }
}

cudaError_t dot(int64_t n, const double* x, const double* y, const double* w, double* scratch, int slot,
                cudaStream_t s, double* host_out) {
  const int nblk = (int)((n + kChunk - 1) / kChunk);
  if (nblk > 0) k_chunk_dot<<<nblk, 256, 0, s>>>(n, x, y, w, scratch);
  k_chunk_final<<<1, 32, 0, s>>>(nblk, scratch, scratch + kMaxPartials + slot);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, scratch + kMaxPartials + slot, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

// The power iteration on the caller's vectors x and y with the static scratch (no
// allocation): the body of pbf_estimate_dt_noalloc, also run once by noalloc_prepare.
pbf_status run_noalloc(pbf_ctx* ctx, double* x_dev, double* y_dev, int max_iter, double rtol, double* lambda_out,
                       double* dt_crit_out, int* iters_out, cudaStream_t s) {
  const int64_t n = ctx->n_dofs;
  double* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return ctx->cuda(e, "estimate_dt_noalloc scratch set-up");
  CellLaunch L = ctx->base;
  L.f32 = 0;
  L.nonlin_k = 0;
  L.latent = 0;
  L.offset = 0.0;
  L.mesh.batch = 1;
  e = launch_zero_masked(n, x_dev, ctx->dirichlet, s);
  double lambda = 0.0;
  int it = 0;
  for (; it < max_iter && e == cudaSuccess; ++it) {
    double nx2 = 0.0;
    e = dot(n, x_dev, x_dev, ctx->C0, scratch, 0, s, &nx2);
    if (e != cudaSuccess) break;
    if (!(nx2 > 0)) return set_error(PBF_EINVAL, "start vector vanishes on the free dofs");
    const double inv = 1.0 / std::sqrt(nx2);
    e = cudaMemcpyAsync(scratch + kMaxPartials + 1, &inv, 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_scale_masked(n, x_dev, scratch + kMaxPartials + 1, nullptr, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(y_dev, 0, (size_t)n * 8, s);
    L.x = x_dev;
    if (e == cudaSuccess) e = ctx->apply_cell(L, y_dev, nullptr, MODE_STIFF, s);
    if (e == cudaSuccess) e = launch_zero_masked(n, y_dev, ctx->dirichlet, s);
    double lam = 0.0;
    if (e == cudaSuccess) e = dot(n, x_dev, y_dev, nullptr, scratch, 2, s, &lam);
    if (e == cudaSuccess) e = launch_div_masked(n, x_dev, y_dev, ctx->invC0_d, ctx->dirichlet, s);
    ctx->launches += 10;
    if (e != cudaSuccess) break;
    const bool done = it > 0 && std::fabs(lam - lambda) <= rtol * std::fabs(lam);
    lambda = lam;
    if (done) {
      ++it;
      break;
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ctx->cuda(e, "estimate_dt_noalloc");
  if (lambda_out) *lambda_out = lambda;
  if (dt_crit_out) *dt_crit_out = lambda > 0 ? 2.0 / lambda : INFINITY;
  if (iters_out) *iters_out = it;
  return PBF_OK;
}

}  // namespace

namespace pbf {

// Set-up of the allocation-free entry point for the current device, run by pbf_ctx_create
// (which may allocate): looks up the static array's device address and runs one iteration
// of the power iteration on temporary vectors, so that every kernel the entry point launches
// is loaded. The CUDA runtime loads kernels lazily, on their first launch, and loading one
// allocates device memory; after this set-up a call of the entry point allocates nothing.
pbf_status noalloc_prepare(CtxBase* base) {
  pbf_ctx* ctx = static_cast<pbf_ctx*>(base);
  const int64_t n = ctx->n_dofs;
  if (n == 0 || (n + kChunk - 1) / kChunk > kMaxPartials) return PBF_OK;  // the entry point rejects these
  double *x = nullptr, *y = nullptr;
  cudaError_t e = cudaMalloc(&x, (size_t)n * 8);
  if (e == cudaSuccess) e = cudaMalloc(&y, (size_t)n * 8);
  pbf_status st = PBF_OK;
  if (e == cudaSuccess) {
    std::vector<double> one((size_t)n, 1.0);
    e = cudaMemcpy(x, one.data(), (size_t)n * 8, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) {
    st = run_noalloc(ctx, x, y, 1, 0.0, nullptr, nullptr, nullptr, 0);
    if (st == PBF_EINVAL) st = PBF_OK;  // every dof is a Dirichlet dof: the kernels loaded all the same
  }
  if (x) cudaFree(x);
  if (y) cudaFree(y);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(e == cudaErrorMemoryAllocation ? PBF_ENOMEM : PBF_ECUDA, cudaGetErrorString(e));
  }
  return st;
}

}  // namespace pbf

extern "C" pbf_status pbf_estimate_dt_noalloc(pbf_ctx* ctx, double* x_dev, double* y_dev, int max_iter, double rtol,
                                              double* lambda_out, double* dt_crit_out, int* iters_out,
                                              pbf_stream stream) {
  if (!ctx || !x_dev || !y_dev) return set_error(PBF_EINVAL, "null argument");
  if (max_iter < 1) return set_error(PBF_EINVAL, "max_iter must be positive");
  pbf_status st = ctx->check_usable();
  if (st) return st;
  const int64_t n = ctx->n_dofs;
  if ((n + kChunk - 1) / kChunk > kMaxPartials)
    return set_error(PBF_EINVAL, "pbf_estimate_dt_noalloc handles at most 134,217,728 dofs "
                                 "(its fixed reduction scratch holds 32,768 partial sums)");
  const uintptr_t xa = (uintptr_t)x_dev, ya = (uintptr_t)y_dev, nb = (uintptr_t)n * 8;
  if (xa < ya + nb && ya < xa + nb) return set_error(PBF_EINVAL, "x_dev and y_dev overlap");
  return run_noalloc(ctx, x_dev, y_dev, max_iter, rtol, lambda_out, dt_crit_out, iters_out, (cudaStream_t)stream);
}
