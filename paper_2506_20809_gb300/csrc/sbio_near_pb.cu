// Near-field kernels for p in {9, 10, 11, 12, 13}.
#include "sbio_near_kernels.cuh"

namespace sbio {

near_launcher near_lookup_b(int p) { return NearTable<9, 10, 11, 12, 13>::get(p); }

}  // namespace sbio
