// Stokes double-layer near kernels for p = 16 (expansions to order p+1);
// one translation unit per range so that the unrolled variants compile in parallel.
#include "sbio_stokes_dl_near.cuh"

namespace sbio {

stokes_dl_near_launcher stokes_dl_near_lookup_f(int p) { return StokesDLNearTable<16>::get(p); }

}  // namespace sbio
