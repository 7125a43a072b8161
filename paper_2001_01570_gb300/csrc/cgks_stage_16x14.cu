// Instantiation of the flux kernel for 16x14 cell tiles.
#include "cgks_stage.cuh"

namespace cgks {
CGKS_STAGE_INSTANCE(16, 14)
}  // namespace cgks
