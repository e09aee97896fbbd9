// S' / D' near-field kernels for p in {1, ..., 12}.
#include "sbio_deriv_near.cuh"

namespace sbio {

deriv_near_launcher deriv_near_lookup_a(int p) { return DerivNearTable<1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12>::get(p); }

}  // namespace sbio
