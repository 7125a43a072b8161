// Instantiation of the flux kernel for 16x16 cell tiles.
#include "cgks_stage.cuh"

namespace cgks {
CGKS_STAGE_INSTANCE(16, 16)
}  // namespace cgks
