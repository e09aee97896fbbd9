// S' / D' near-field kernels for p in {13, ..., 20}.
#include "sbio_deriv_near.cuh"

namespace sbio {

deriv_near_launcher deriv_near_lookup_b(int p) { return DerivNearTable<13, 14, 15, 16, 17, 18, 19, 20>::get(p); }

}  // namespace sbio
