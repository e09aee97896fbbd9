// Stokes double-layer near kernels for p in {1, ..., 12} (expansions to order p+1).
#include "sbio_stokes_dl_near.cuh"

namespace sbio {

stokes_dl_near_launcher stokes_dl_near_lookup_a(int p) { return StokesDLNearTable<1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12>::get(p); }

}  // namespace sbio
