// Instantiation of the flux kernel for 16x7 cell tiles.
#include "cgks_stage.cuh"

namespace cgks {
CGKS_STAGE_INSTANCE(16, 7)
}  // namespace cgks
