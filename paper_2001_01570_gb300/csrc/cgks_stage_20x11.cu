// Instantiation of the flux kernel for 20x11 cell tiles.
#include "cgks_stage.cuh"

namespace cgks {
CGKS_STAGE_INSTANCE(20, 11)
}  // namespace cgks
