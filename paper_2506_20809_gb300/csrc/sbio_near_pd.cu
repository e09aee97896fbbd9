// Near-field kernels for p in {19, 20, 21, 22, 23, 24}.
#include "sbio_near_kernels.cuh"

namespace sbio {

near_launcher near_lookup_d(int p) { return NearTable<19, 20, 21, 22, 23, 24>::get(p); }

}  // namespace sbio
