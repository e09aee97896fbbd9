// Stokes velocity + pressure near kernels at points for p in {17, ..., 20}.
#include "sbio_stokes_points.cuh"

namespace sbio {

stokes_point_near_launcher stokes_point_near_lookup_c(int p) { return StokesPointNearTable<17, 18, 19, 20>::get(p); }

}  // namespace sbio
