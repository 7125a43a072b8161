// Instantiation of the flux kernel for 15x16 cell tiles.
#include "cgks_stage.cuh"

namespace cgks {
CGKS_STAGE_INSTANCE(15, 16)
}  // namespace cgks
