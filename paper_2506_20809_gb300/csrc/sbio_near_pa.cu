// Near-field kernels for p in {1, 2, 3, 4, 5, 6, 7, 8}.
#include "sbio_near_kernels.cuh"

namespace sbio {

near_launcher near_lookup_a(int p) { return NearTable<1, 2, 3, 4, 5, 6, 7, 8>::get(p); }

}  // namespace sbio
