// Near-field kernels for p in {14, 15, 16, 17, 18}.
#include "sbio_near_kernels.cuh"

namespace sbio {

near_launcher near_lookup_c(int p) { return NearTable<14, 15, 16, 17, 18>::get(p); }

}  // namespace sbio
