// Instantiation of the flux kernel for 64x1 cell tiles.
#include "cgks_stage.cuh"

namespace cgks {
CGKS_STAGE_INSTANCE(64, 1)
}  // namespace cgks
