// Stokes double-layer near kernels for p in {13, ..., 20} (expansions to order p+1).
#include "sbio_stokes_dl_near.cuh"

namespace sbio {

stokes_dl_near_launcher stokes_dl_near_lookup_b(int p) { return StokesDLNearTable<13, 14, 15, 16, 17, 18, 19, 20>::get(p); }

}  // namespace sbio
