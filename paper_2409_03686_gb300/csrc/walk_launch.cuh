// walk_launch.cuh -- launch planning of the persistent walk kernel, shared by
// every entry point that launches it (grid, block, shared memory, tiles).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "walk_kernel.cuh"
#include "wos.h"

namespace wos {

struct WalkPlan {
    const void *kfn;   // kernel entry
    int block, grid, nslot;
    size_t smem;       // dynamic shared memory per block
    uint32_t tile_w, tiles_per_point;
    uint64_t n_tiles;
};

template <typename Real, int DIM, int KIND>
const void *walk_kernel_ptr()
{
    return reinterpret_cast<const void *>(&walk_kernel<Real, DIM, KIND>);
}

template <typename Real, int DIM>
const void *pick_walk_kernel(int kind)
{
    if (kind == kSphereOnly) return walk_kernel_ptr<Real, DIM, kSphereOnly>();
    if (kind == kBoxOnly) return walk_kernel_ptr<Real, DIM, kBoxOnly>();
    if (kind == kSphereHoles) return walk_kernel_ptr<Real, DIM, kSphereHoles>();
    return walk_kernel_ptr<Real, DIM, kGeneric>();
}

// Kernel kind: specialised distance for a plain disc / ball or box.
inline int walk_kind(const wos_domain &d, const wos_partition &part)
{
    if (part.voronoi_n <= 0 && d.outer_kind == WOS_OUTER_SPHERE)
        return d.n_holes == 0 ? kSphereOnly : kSphereHoles;
    if (part.voronoi_n <= 0 && d.n_holes == 0 && d.outer_kind == WOS_OUTER_BOX)
        return kBoxOnly;
    return kGeneric;
}

// Plans a launch: block size, shared-memory histogram slots per warp (2 when
// they fit next to the exit queues in ~56 KiB per block, so that four blocks
// share an SM; else 1; else none), grid = SMs x resident blocks, and the tile
// size (about 16 tiles per warp, 64..16384 walks, a multiple of 32, at most
// the walks of one point).
template <typename Real, int DIM>
wos_status plan_walk(int kind, int32_t M_tot, const wos_opts &o, int sm_count,
                     int max_smem_optin, uint64_t per_point, int32_t M_D, WalkPlan *P)
{
    P->kfn = pick_walk_kernel<Real, DIM>(kind);
    P->block = o.block_size > 0 ? o.block_size : 256;
    const int warps = P->block / 32;
    const size_t qbytes = size_t(warps) * queue_bytes<Real, DIM>();
    const size_t slot_bytes = size_t(warps) * size_t((M_tot + 1) / 2) * 4;
    const size_t budget = 56 * 1024;
    int nslot = o.hist_slots;
    if (nslot == 0) {
        if (qbytes + 2 * slot_bytes <= budget) nslot = 2;
        else if (qbytes + slot_bytes <= 2 * budget) nslot = 1;
        else nslot = -1;
    }
    if (nslot < 0) nslot = 0;
    P->nslot = nslot;
    P->smem = qbytes + size_t(nslot) * slot_bytes;
    if (P->smem > size_t(max_smem_optin))
        return WOS_INVALID_ARG;
    cudaError_t e = cudaFuncSetAttribute(P->kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(P->smem));
    if (e != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? WOS_OOM : WOS_CUDA_ERROR;
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, P->kfn, P->block, P->smem);
    if (e != cudaSuccess)
        return WOS_CUDA_ERROR;
    if (bps < 1)
        return WOS_INVALID_ARG;
    if (o.blocks_per_sm > 0)
        bps = std::min(bps, o.blocks_per_sm);
    P->grid = sm_count * bps;
    const uint64_t total = per_point * uint64_t(M_D);
    uint64_t tw = o.tile_walks > 0 ? uint64_t(o.tile_walks)
                                   : total / (16ull * uint64_t(P->grid) * warps);
    tw = std::max<uint64_t>(tw, 64);
    tw = std::min<uint64_t>(tw, 16384);
    tw = (tw + 31) / 32 * 32;
    tw = std::min<uint64_t>(tw, per_point);
    if (tw == 0) tw = 1;
    P->tile_w = uint32_t(tw);
    P->tiles_per_point = uint32_t((per_point + tw - 1) / tw);
    P->n_tiles = uint64_t(P->tiles_per_point) * uint64_t(M_D);
    return WOS_OK;
}

template <typename Real>
wos_status plan_walk_any(int dim, int kind, int32_t M_tot, const wos_opts &o, int sm_count,
                         int max_smem_optin, uint64_t per_point, int32_t M_D, WalkPlan *P)
{
    if (dim == 2)
        return plan_walk<Real, 2>(kind, M_tot, o, sm_count, max_smem_optin, per_point, M_D, P);
    return plan_walk<Real, 3>(kind, M_tot, o, sm_count, max_smem_optin, per_point, M_D, P);
}

}  // namespace wos
