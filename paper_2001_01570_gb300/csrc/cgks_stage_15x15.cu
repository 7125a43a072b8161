// Instantiation of the flux kernel for 15x15 cell tiles.
#include "cgks_stage.cuh"

namespace cgks {
CGKS_STAGE_INSTANCE(15, 15)
}  // namespace cgks
