// Stokes near-field kernels for p in {17, 18, 19, 20} (expansions carried to order p+1).
#include "sbio_stokes_near.cuh"

namespace sbio {

stokes_near_launcher stokes_near_lookup_c(int p) { return StokesNearTable<17, 18, 19, 20>::get(p); }

}  // namespace sbio
