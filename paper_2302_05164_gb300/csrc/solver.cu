// Implicit cool-down solver and adjoint sweep of the library.
#include <cuda_runtime.h>

#include "pbf.h"
#include "solver.hpp"

using namespace pbf;

struct pbf_ctx : public CtxBase {};

extern "C" pbf_status pbf_cheb_bounds(pbf_ctx*, double, const double*, int, double*, pbf_stream) {
  return set_error(PBF_EINVAL, "not available yet");
}

extern "C" pbf_status pbf_implicit_solve(pbf_ctx*, double*, double, int, double, int, int, const double*, int*,
                                         pbf_stream) {
  return set_error(PBF_EINVAL, "not available yet");
}

extern "C" pbf_status pbf_adjoint_sweep(pbf_ctx*, const double*, const pbf_laser*, double, double, int, int, double,
                                        double, double*, double*, long long*, pbf_stream) {
  return set_error(PBF_EINVAL, "not available yet");
}

extern "C" pbf_status pbf_revolve_cost(int, int, long long*) { return set_error(PBF_EINVAL, "not available yet"); }
