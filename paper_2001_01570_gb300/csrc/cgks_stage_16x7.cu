// Instantiation of the fused stage kernel for 16x7 cell tiles (one
// translation unit per tile shape so they compile in parallel).
#include "cgks_stage.cuh"

namespace cgks {
cudaError_t launch_stage_16x7(int stage, const GridDev* grids, const TileRef* tiles, int ntiles, int nblocks,
                               cudaStream_t st)
{
    return stage == 1 ? launch_stage_t<16, 7, 1>(grids, tiles, ntiles, nblocks, st)
                      : launch_stage_t<16, 7, 2>(grids, tiles, ntiles, nblocks, st);
}
size_t smem_16x7(int stage)
{
    return stage == 1 ? StageLayout<16, 7, 1>::bytes : StageLayout<16, 7, 2>::bytes;
}
}  // namespace cgks
