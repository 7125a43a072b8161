// Instantiation of the fused stage kernel for 64x1 cell tiles (one
// translation unit per tile shape so they compile in parallel).
#include "cgks_stage.cuh"

namespace cgks {
cudaError_t launch_stage_64x1(int stage, const GridDev* grids, const TileRef* tiles, int ntiles, int nblocks,
                               cudaStream_t st)
{
    return stage == 1 ? launch_stage_t<64, 1, 1>(grids, tiles, ntiles, nblocks, st)
                      : launch_stage_t<64, 1, 2>(grids, tiles, ntiles, nblocks, st);
}
size_t smem_64x1(int stage)
{
    return stage == 1 ? StageLayout<64, 1, 1>::bytes : StageLayout<64, 1, 2>::bytes;
}
}  // namespace cgks
