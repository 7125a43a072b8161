// Instantiation of the flux kernel for 17x14 cell tiles.
#include "cgks_stage.cuh"

namespace cgks {
CGKS_STAGE_INSTANCE(17, 14)
}  // namespace cgks
