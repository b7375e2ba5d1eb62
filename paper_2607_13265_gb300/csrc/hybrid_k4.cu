// Hybrid cached replay kernels with checkpoint interval 4 (every depth bucket).
#include "hybrid.cuh"

namespace dppt {
DPPT_HYBRID_INTERVAL(4)
}  // namespace dppt
