// Instantiation of the flux kernel for 8x16 cell tiles.
#include "cgks_stage.cuh"

namespace cgks {
CGKS_STAGE_INSTANCE(8, 16)
}  // namespace cgks
