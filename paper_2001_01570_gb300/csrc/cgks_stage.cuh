// cgks_stage.cuh -- the per-stage flux kernel of the two-stage fourth-order
// compact GKS (Sec. 2.2, Eq. step-hyper-1).  It runs after the record kernel
// (cgks_records.cu), which did the normal reconstruction of every face row of
// the grid once, and before the update kernel (cgks_update.cu), which applies
// the face results to the cells.
//
// One CTA owns a TX x TY tile of cells of one grid and runs, in shared memory:
//   phase 1  stage the face-row records the tile needs (its faces on its rows
//            and two rows either side) with asynchronous copies
//   phase 2  per face segment the tile owns (the x- and y-faces on the low side
//            of its cells, plus the grid's last face where the tile ends on the
//            grid's edge, so every face is evaluated once), at two Gauss points:
//            WENO-Z point values along the face over rows j-2..j+2
//            (equilibrium) and j-1..j+1 (non-equilibrium states, with their
//            tangential slopes); tangential derivatives of the equilibrium state
//            and normal derivatives from the quartic / quadratic through the same
//            line averages (their Gauss-point-independent parts once per
//            segment); the gas-kinetic evaluation at each point; the Gauss
//            average, weighted by the stage's time factors, written to the face
//            results (stage 1: the W* and R flux combinations and the interface
//            states W(dt/2), W(dt); stage 2: dt^2/3 F_t and dt^2/3 W_tt)
// Coefficients (fixed, and the tile's grid and dt) come from the shared-memory
// table of cgks_flux.cuh; all arithmetic is in the register-only DFMA forms.
// The kernel is persistent: CTAs stride over a flattened tile queue that may
// span many grids of different sizes (each with its own dt in its Ctrl).
#pragma once
#include "cgks_segment.cuh"
#include "../../include/cgks.h"

#include <mutex>

namespace cgks {

static __constant__ FluxFixed kFluxFixed = make_flux_fixed();

template <int TX, int TY, int STAGE>
__global__ void __launch_bounds__(kThreads, kStageCtasPerSm)
stage_kernel(const GridDev* __restrict__ grids, const TileRef* __restrict__ tiles, int ntiles,
             const int* __restrict__ dcount)
{
    using L = StageLayout<TX, TY, STAGE>;
    constexpr int NF = L::NF;
    extern __shared__ double smem[];
    double* rx = smem;                  // x-face records, RecGroups<TY, TX+1>
    double* ry = rx + L::n_rx;          // y-face records, RecGroups<TX, TY+1>
    double* dc = ry + L::n_ry + threadIdx.x;   // [32][kThreads] when L::share
    __shared__ double s_fk[FK_N];       // coefficient table (fixed part, then the tile's grid and dt)
    __shared__ int s_skip;
    // the queue length (a kernel argument, or in device memory for a server's patched queue) is
    // kept in shared memory: at 255 registers a loop bound in a register costs spills
    const int tid = threadIdx.x;

    for (int i = tid; i < FK_NFIX; i += kThreads) s_fk[i] = kFluxFixed.v[i];
    if (tid < 32) s_fk[FK_EXP2 + tid] = exp2((double)tid * (1.0 / 32.0));
    __syncthreads();
    const RegK r{s_fk, ((volatile const double*)s_fk)[FK_ONE], ((volatile const double*)s_fk)[FK_NZERO]};

    // the queue length: the kernel argument, or the int in device memory behind dcount (a server's
    // queue, patched between replays), read at each tile -- at 255 registers a bound kept in a
    // register through the loop costs spills (5 % of the stage-1 kernel's time)
    for (int tile = blockIdx.x; tile < (dcount ? *(volatile const int*)dcount : ntiles); tile += gridDim.x) {
        __syncthreads();
        const TileRef tr = tiles[tile];
        const GridDev& G = grids[tr.grid];
        if (tid == 0) {
            const Ctrl* C = G.ctrl;
            s_skip = C->done;
            if (!C->done) flux_table_tile(s_fk, G, C->dt);
        }
        __syncthreads();
        if (s_skip) continue;
        const int nx = G.nx, ny = G.ny, x0 = tr.x0, y0 = tr.y0;
        const bool dim1 = (G.dim == 1);

        // ---------------- phase 1: the tile's face-row records (the record kernel
        // wrote them for every face row of the grid): x-faces x0..x0+TX on rows
        // y0-2..y0+TY+1, y-faces y0..y0+TY on columns x0-2..x0+TX+1, each field on
        // the rows it is read on; rows beyond the grid's last ghost row are zero
        // and unused.  Asynchronous 8-byte copies, zero-filled where invalid.
        {
            const size_t sx = (size_t)(ny + 4) * (nx + 1), sy = (size_t)(nx + 4) * (ny + 1);
            const unsigned sbx = (unsigned)__cvta_generic_to_shared(rx), sby = (unsigned)__cvta_generic_to_shared(ry);
            // group g of one orientation: plane p of the group is global plane p0 + p, its
            // local row q is record row base + q (records carry two ghost rows first)
            auto stage = [&](unsigned sbase, int sofs, int np, int plane, int F, int p0, const double* g, size_t gs,
                             int gfaces, int row0, int face0, int nface_max, int row_max, bool on, int nsmem) {
                const int n = np * plane;
                for (int idx = tid; idx < n; idx += kThreads) {
                    const int p = idx / plane, rem = idx - p * plane;
                    const int q = rem / F, fc = rem - q * F;
                    bool valid = on && (face0 + fc <= nface_max) && (row0 + q <= row_max);
                    if (!CGKS_IN_BOUNDS(sofs + idx < nsmem, G.ctrl)) continue;
                    if (valid)
                        valid = CGKS_IN_BOUNDS(row0 + q >= 0 && face0 + fc >= 0 &&
                                                   (size_t)(p0 + p) * gs + (size_t)(row0 + q) * gfaces + face0 + fc <
                                                       28 * gs,
                                               G.ctrl);
                    const double* src = valid ? g + (size_t)(p0 + p) * gs + (size_t)(row0 + q) * gfaces + face0 + fc
                                              : G.recx;
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(sbase + 8u * (unsigned)(sofs + idx)),
                                 "l"(src), "r"(valid ? 8 : 0) : "memory");
                }
            };
            using RX = RecGroups<TY, TX + 1>;
            using RY = RecGroups<TX, TY + 1>;
            // x-faces: record rows y0 + 2 + (own row); group A starts two rows earlier, B one
            stage(sbx, 0, 8, RX::pa, TX + 1, 0, G.recx, sx, nx + 1, y0, x0, nx, ny + 3, true, RX::n);
            stage(sbx, 8 * RX::pa, 16, RX::pb, TX + 1, 4 * RL, G.recx, sx, nx + 1, y0 + 1, x0, nx, ny + 3, true, RX::n);
            stage(sbx, 8 * RX::pa + 16 * RX::pb, 4, RX::pc, TX + 1, 4 * RNN, G.recx, sx, nx + 1, y0 + 2, x0, nx, ny + 3,
                  true, RX::n);
            stage(sby, 0, 8, RY::pa, TY + 1, 0, G.recy, sy, ny + 1, x0, y0, ny, nx + 3, !dim1, RY::n);
            stage(sby, 8 * RY::pa, 16, RY::pb, TY + 1, 4 * RL, G.recy, sy, ny + 1, x0 + 1, y0, ny, nx + 3, !dim1,
                  RY::n);
            stage(sby, 8 * RY::pa + 16 * RY::pb, 4, RY::pc, TY + 1, 4 * RNN, G.recy, sy, ny + 1, x0 + 2, y0, ny, nx + 3,
                  !dim1, RY::n);
            asm volatile("cp.async.wait_all;" ::: "memory");
        }
        __syncthreads();

        // ---------------- phase 2: face segments, two Gauss points each
        bool bad = false;
        // the tile's own faces: x-faces x0..x0+TX-1 and y-faces y0..y0+TY-1 of its
        // cells, plus the last face of the grid where the tile ends on the grid's
        // edge; every face is evaluated by exactly one tile
        const int xe = (x0 + TX == nx) ? TY : 0, ye = (!dim1 && y0 + TY == ny) ? TX : 0;
        const int nseg = (dim1 ? TX * TY : 2 * TX * TY) + xe + ye;
        const size_t nfx = (size_t)ny * (nx + 1), nfy = (size_t)(ny + 1) * nx;
        for (int item = tid; item < nseg; item += kThreads) {
            int fl, jl, il, gl;
            bool xo;
            if (item < TX * TY) { xo = true; fl = item % TX; jl = item / TX; }
            else if (!dim1 && item < 2 * TX * TY) { xo = false; const int it = item - TX * TY; il = it % TX; gl = it / TX; }
            else {
                const int it = item - (dim1 ? TX * TY : 2 * TX * TY);
                if (it < xe) { xo = true; fl = TX; jl = it; }
                else { xo = false; il = it - xe; gl = TY; }
            }
            const double* rec;
            int pa, pb, pc, r0, rstride;
            double* out;
            size_t ostride, oidx;
            if (xo) {
                if (!((x0 + fl <= nx) && (y0 + jl < ny))) continue;
                rec = rx; pa = RecGroups<TY, TX + 1>::pa; pb = RecGroups<TY, TX + 1>::pb; pc = RecGroups<TY, TX + 1>::pc;
                r0 = jl * (TX + 1) + fl; rstride = TX + 1;
                out = G.facex; ostride = nfx; oidx = (size_t)(y0 + jl) * (nx + 1) + x0 + fl;
            } else {
                if (!((y0 + gl <= ny) && (x0 + il < nx))) continue;
                rec = ry; pa = RecGroups<TX, TY + 1>::pa; pb = RecGroups<TX, TY + 1>::pb; pc = RecGroups<TX, TY + 1>::pc;
                r0 = il * (TY + 1) + gl; rstride = TY + 1;
                out = G.facey; ostride = nfy; oidx = (size_t)(y0 + gl) * nx + x0 + il;
            }
            // the segment's record window (rows -2..2 of group A, -1..1 of group B, 0 of group C)
            // and its output index
            if (!CGKS_IN_BOUNDS(r0 >= 0 && r0 + 4 * rstride < pa && r0 + 2 * rstride < pb && r0 < pc &&
                                    oidx < ostride,
                                G.ctrl))
                continue;
            const double iht = r.k(xo ? FK_IDY : FK_IDX);
            double acc[NF];
            // stage 2 parks the first Gauss point's sums in the output slots: its register
            // allocation then spills nothing (measured: 26.3 -> 25.5 ms on 2048^2); stage 1
            // runs faster with them in registers
            bad |= !segment_results<STAGE, L::share, STAGE == 2>(r, rec, pa, pb, pc, r0, rstride, iht, dc, acc,
                                                                  out + oidx, ostride);
            // back to the physical frame (y-faces: swap momentum components)
#pragma unroll
            for (int q = 0; q < NF; q += 4) {
                const int k1 = xo ? 1 : 2, k2 = xo ? 2 : 1;
                out[(q + 0) * ostride + oidx] = acc[q + 0];
                out[(q + k1) * ostride + oidx] = acc[q + 1];
                out[(q + k2) * ostride + oidx] = acc[q + 2];
                out[(q + 3) * ostride + oidx] = acc[q + 3];
            }
        }
        if (bad) atomicOr(&G.ctrl->status, (int)CGKS_E_NONPHYSICAL);
    }
}

// The kernel's attributes (more than 48 KB of dynamic shared memory, the
// largest carveout) belong to one device's context: they are set once per
// device, thread-safely, before the first launch on that device.
template <int TX, int TY, int STAGE>
cudaError_t configure_stage_t()
{
    using L = StageLayout<TX, TY, STAGE>;
    static std::once_flag once[kMaxDevices];
    static cudaError_t status[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(once[dev], [dev] {
        cudaError_t r = cudaFuncSetAttribute(stage_kernel<TX, TY, STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)L::bytes);
        // the largest shared-memory carveout, so that two CTAs fit where the shape allows
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(stage_kernel<TX, TY, STAGE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        status[dev] = r;
    });
    return status[dev];
}

template <int TX, int TY, int STAGE>
cudaError_t launch_stage_t(const GridDev* grids, const TileRef* tiles, int ntiles, int nblocks, cudaStream_t st,
                           const int* dcount)
{
    using L = StageLayout<TX, TY, STAGE>;
    cudaError_t e = configure_stage_t<TX, TY, STAGE>();
    if (e != cudaSuccess) return e;
    if (ntiles <= 0 || nblocks <= 0) return cudaSuccess;
    stage_kernel<TX, TY, STAGE><<<nblocks, kThreads, L::bytes, st>>>(grids, tiles, ntiles, dcount);
    return cudaGetLastError();
}

// The launcher and shared-memory size of one tile shape (one translation unit
// per shape, so the shapes compile in parallel).
#define CGKS_STAGE_INSTANCE(TX, TY)                                                                         \
    static_assert(StageLayout<TX, TY, 1>::bytes + 64 <= 227 * 1024, "stage-1 tile exceeds shared memory");  \
    cudaError_t launch_stage_##TX##x##TY(int stage, const GridDev* grids, const TileRef* tiles, int ntiles,  \
                                         int nblocks, cudaStream_t st, const int* dcount)                   \
    {                                                                                                       \
        return stage == 1 ? launch_stage_t<TX, TY, 1>(grids, tiles, ntiles, nblocks, st, dcount)            \
                          : launch_stage_t<TX, TY, 2>(grids, tiles, ntiles, nblocks, st, dcount);           \
    }                                                                                                       \
    size_t smem_##TX##x##TY(int stage)                                                                      \
    {                                                                                                       \
        return stage == 1 ? StageLayout<TX, TY, 1>::bytes : StageLayout<TX, TY, 2>::bytes;                  \
    }

}  // namespace cgks
