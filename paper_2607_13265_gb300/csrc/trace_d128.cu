// Kernels of the depth-128 cache bucket (paths of at most 128 vertices).
#include "wavefront.cuh"

namespace dppt {
DPPT_TRACE_BUCKET(128)
DPPT_SWEEP_BUCKET(128)
}  // namespace dppt
