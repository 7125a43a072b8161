// Instantiation of the flux kernel for 18x12 cell tiles.
#include "cgks_stage.cuh"

namespace cgks {
CGKS_STAGE_INSTANCE(18, 12)
}  // namespace cgks
