// Instantiation of the flux kernel for 22x10 cell tiles.
#include "cgks_stage.cuh"

namespace cgks {
CGKS_STAGE_INSTANCE(22, 10)
}  // namespace cgks
