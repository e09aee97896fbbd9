// Stokes velocity + pressure near kernels at points for p in {1, ..., 12}.
#include "sbio_stokes_points.cuh"

namespace sbio {

stokes_point_near_launcher stokes_point_near_lookup_a(int p) {
  return StokesPointNearTable<1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12>::get(p);
}

}  // namespace sbio
