// Instantiation of the flux kernel for 32x12 cell tiles.
#include "cgks_stage.cuh"

namespace cgks {
CGKS_STAGE_INSTANCE(32, 12)
}  // namespace cgks
