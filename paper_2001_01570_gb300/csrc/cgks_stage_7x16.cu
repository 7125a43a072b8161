// Instantiation of the flux kernel for 7x16 cell tiles.
#include "cgks_stage.cuh"

namespace cgks {
CGKS_STAGE_INSTANCE(7, 16)
}  // namespace cgks
