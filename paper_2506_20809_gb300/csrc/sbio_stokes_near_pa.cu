// Stokes near-field kernels for p in {1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12} (expansions carried to order p+1).
#include "sbio_stokes_near.cuh"

namespace sbio {

stokes_near_launcher stokes_near_lookup_a(int p) { return StokesNearTable<1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12>::get(p); }

}  // namespace sbio
