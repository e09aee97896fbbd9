// Stokes double-layer near kernels for p in {1, ..., 8} (expansions to order p+1);
// one translation unit per range so that the unrolled variants compile in parallel.
#include "sbio_stokes_dl_near.cuh"

namespace sbio {

stokes_dl_near_launcher stokes_dl_near_lookup_a(int p) { return StokesDLNearTable<1, 2, 3, 4, 5, 6, 7, 8>::get(p); }

}  // namespace sbio
