// Kernels of the depth-64 cache bucket (paths of at most 64 vertices).
#include "wavefront.cuh"

namespace dppt {
DPPT_TRACE_BUCKET(64)
DPPT_SWEEP_BUCKET(64)
}  // namespace dppt
