// Instantiation of the flux kernel for 20x12 cell tiles.
#include "cgks_stage.cuh"

namespace cgks {
CGKS_STAGE_INSTANCE(20, 12)
}  // namespace cgks
