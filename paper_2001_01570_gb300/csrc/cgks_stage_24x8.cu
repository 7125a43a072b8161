// Instantiation of the fused stage kernel for 24x8 cell tiles (one
// translation unit per tile shape so they compile in parallel).
#include "cgks_stage.cuh"

namespace cgks {
cudaError_t launch_stage_24x8(int stage, const GridDev* grids, const TileRef* tiles, int ntiles, int nblocks,
                               cudaStream_t st)
{
    return stage == 1 ? launch_stage_t<24, 8, 1>(grids, tiles, ntiles, nblocks, st)
                      : launch_stage_t<24, 8, 2>(grids, tiles, ntiles, nblocks, st);
}
size_t smem_24x8(int stage)
{
    return stage == 1 ? StageLayout<24, 8, 1>::bytes : StageLayout<24, 8, 2>::bytes;
}
}  // namespace cgks
