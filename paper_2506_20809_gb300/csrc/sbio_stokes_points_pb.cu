// Stokes velocity + pressure near kernels at points for p in {13, ..., 16}.
#include "sbio_stokes_points.cuh"

namespace sbio {

stokes_point_near_launcher stokes_point_near_lookup_b(int p) { return StokesPointNearTable<13, 14, 15, 16>::get(p); }

}  // namespace sbio
