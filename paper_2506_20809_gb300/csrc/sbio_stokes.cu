// Stokes single layer through the Laplace-to-Stokes identity (Sec. 4.3).
#include "sbio_internal.cuh"

namespace sbio {

int launch_stokes(sbio_geom* g, const double* f, double* u, cudaStream_t st) {
  (void)g; (void)f; (void)u; (void)st;
  return set_error(SBIO_ENOTSUP, "Stokes single layer not built yet");
}

}  // namespace sbio
