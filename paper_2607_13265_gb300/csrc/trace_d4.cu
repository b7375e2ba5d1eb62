// Kernels of the depth-4 cache bucket (paths of at most 4 vertices).
#include "wavefront.cuh"

namespace dppt {
DPPT_TRACE_BUCKET(4)
DPPT_SWEEP_BUCKET(4)
}  // namespace dppt
