// Hybrid cached replay kernels with checkpoint interval 16 (every depth bucket).
#include "hybrid.cuh"

namespace dppt {
DPPT_HYBRID_INTERVAL(16)
}  // namespace dppt
