// Stokes near-field kernels for p in {13, 14, 15, 16} (expansions carried to order p+1).
#include "sbio_stokes_near.cuh"

namespace sbio {

stokes_near_launcher stokes_near_lookup_b(int p) { return StokesNearTable<13, 14, 15, 16>::get(p); }

}  // namespace sbio
