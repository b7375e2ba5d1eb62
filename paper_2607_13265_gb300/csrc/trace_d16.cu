// Kernels of the depth-16 cache bucket (paths of at most 16 vertices).
#include "trace.cuh"

namespace dppt {
DPPT_TRACE_BUCKET(16)
}  // namespace dppt
