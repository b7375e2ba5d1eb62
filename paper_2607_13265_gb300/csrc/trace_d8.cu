// Kernels of the depth-8 cache bucket (paths of at most 8 vertices).
#include "wavefront.cuh"

namespace dppt {
DPPT_TRACE_BUCKET(8)
DPPT_SWEEP_BUCKET(8)
}  // namespace dppt
