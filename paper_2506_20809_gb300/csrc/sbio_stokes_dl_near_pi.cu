// Stokes double-layer near kernels for p = 19 (expansions to order p+1);
// one translation unit per range so that the unrolled variants compile in parallel.
#include "sbio_stokes_dl_near.cuh"

namespace sbio {

stokes_dl_near_launcher stokes_dl_near_lookup_i(int p) { return StokesDLNearTable<19>::get(p); }

}  // namespace sbio
