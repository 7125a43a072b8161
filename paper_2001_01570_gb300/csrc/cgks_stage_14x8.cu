// Instantiation of the flux kernel for 14x8 cell tiles.
#include "cgks_stage.cuh"

namespace cgks {
CGKS_STAGE_INSTANCE(14, 8)
}  // namespace cgks
