// The consolidated-fraction history r_c of the phase model (Sec. 2, Eq. consolidated_fraction)
// across mesh changes (Sec. 4.1): the smallest r_c of each cell (the coarsening restriction's
// input), the gather of r_c onto a changed mesh through the host-built history map, and
// copies to and from FP64 arrays. Layout of r_c: [q][n_cells][batch] in the operator
// precision; of the map: [cell][q], old cell * nq + old point, or -1 (start at 0) / -2 (1).
#include "vec_kernels.cuh"

namespace pbf {
namespace {

template <typename R>
__global__ void k_history_min(int nq, int n_cells, int B, const R* __restrict__ rc, double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  double m = 1e300;
  for (int q = 0; q < nq; ++q)
    for (int b = 0; b < B; ++b) m = fmin(m, (double)rc[((int64_t)q * n_cells + c) * B + b]);
  out[c] = m;
}

template <typename R>
__global__ void k_history_gather(int nq, int n_new, int n_old, int B, const int32_t* __restrict__ map,
                                 const R* __restrict__ rc_old, R* __restrict__ rc_new) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // (q, cell, b) of the new array
  const int64_t n = (int64_t)nq * n_new * B;
  if (i >= n) return;
  const int b = (int)(i % B);
  const int c = (int)((i / B) % n_new);
  const int q = (int)(i / ((int64_t)B * n_new));
  const int32_t e = map[(int64_t)c * nq + q];
  R v;
  if (e >= 0) {
    const int oc = e / nq, oq = e - oc * nq;
    v = rc_old[((int64_t)oq * n_old + oc) * B + b];
  } else {
    v = e == -1 ? R(0) : R(1);
  }
  rc_new[i] = v;
}

template <typename A, typename Bt>
__global__ void k_convert(int64_t n, const A* __restrict__ in, Bt* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (Bt)in[i];
}

unsigned grid256(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

cudaError_t launch_history_min(bool f32, int nq, int n_cells, int B, const void* rc, double* out, cudaStream_t s) {
  if (n_cells == 0) return cudaSuccess;
  if (f32) k_history_min<float><<<grid256(n_cells), 256, 0, s>>>(nq, n_cells, B, (const float*)rc, out);
  else k_history_min<double><<<grid256(n_cells), 256, 0, s>>>(nq, n_cells, B, (const double*)rc, out);
  return cudaGetLastError();
}

cudaError_t launch_history_gather(bool f32, int nq, int n_new, int n_old, int B, const int32_t* map, const void* rc_old,
                                  void* rc_new, cudaStream_t s) {
  const int64_t n = (int64_t)nq * n_new * B;
  if (n == 0) return cudaSuccess;
  if (f32)
    k_history_gather<float><<<grid256(n), 256, 0, s>>>(nq, n_new, n_old, B, map, (const float*)rc_old, (float*)rc_new);
  else
    k_history_gather<double><<<grid256(n), 256, 0, s>>>(nq, n_new, n_old, B, map, (const double*)rc_old,
                                                        (double*)rc_new);
  return cudaGetLastError();
}

cudaError_t launch_history_copy(bool f32, bool to_f64, int64_t n, const void* in, void* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (!f32) return cudaMemcpyAsync(out, in, (size_t)n * 8, cudaMemcpyDeviceToDevice, s);
  if (to_f64) k_convert<float, double><<<grid256(n), 256, 0, s>>>(n, (const float*)in, (double*)out);
  else k_convert<double, float><<<grid256(n), 256, 0, s>>>(n, (const double*)in, (float*)out);
  return cudaGetLastError();
}

}  // namespace pbf
