// Kernels of the depth-32 cache bucket (paths of at most 32 vertices).
#include "wavefront.cuh"

namespace dppt {
DPPT_TRACE_BUCKET(32)
DPPT_SWEEP_BUCKET(32)
}  // namespace dppt
