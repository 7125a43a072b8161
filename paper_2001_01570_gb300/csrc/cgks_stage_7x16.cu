// Instantiation of the fused stage kernel for 7x16 cell tiles (one
// translation unit per tile shape so they compile in parallel).
#include "cgks_stage.cuh"

namespace cgks {
cudaError_t launch_stage_7x16(int stage, const GridDev* grids, const TileRef* tiles, int ntiles, int nblocks,
                               cudaStream_t st)
{
    return stage == 1 ? launch_stage_t<7, 16, 1>(grids, tiles, ntiles, nblocks, st)
                      : launch_stage_t<7, 16, 2>(grids, tiles, ntiles, nblocks, st);
}
size_t smem_7x16(int stage)
{
    return stage == 1 ? StageLayout<7, 16, 1>::bytes : StageLayout<7, 16, 2>::bytes;
}
}  // namespace cgks
