// Instantiation of the flux kernel for 24x8 cell tiles.
#include "cgks_stage.cuh"

namespace cgks {
CGKS_STAGE_INSTANCE(24, 8)
}  // namespace cgks
