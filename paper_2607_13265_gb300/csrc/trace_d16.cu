// Kernels of the depth-16 cache bucket (paths of at most 16 vertices).
#include "wavefront.cuh"

namespace dppt {
DPPT_TRACE_BUCKET(16)
DPPT_SWEEP_BUCKET(16)
}  // namespace dppt
