// Instantiation of the flux kernel for 24x16 cell tiles.
#include "cgks_stage.cuh"

namespace cgks {
CGKS_STAGE_INSTANCE(24, 16)
}  // namespace cgks
