// Hybrid cached replay kernels with checkpoint interval 8 (every depth bucket).
#include "hybrid.cuh"

namespace dppt {
DPPT_HYBRID_INTERVAL(8)
}  // namespace dppt
