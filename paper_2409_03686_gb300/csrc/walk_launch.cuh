// walk_launch.cuh -- host-side set-up and launch planning of the persistent
// walk kernel, shared by every entry point that launches it: the instance
// record, the kernel variant, block / grid / shared memory and tile sizes.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "walk_kernel.cuh"
#include "wos.h"
#include "wos_internal.h"

namespace wos {

struct WalkPlan {
    const void *kfn;   // kernel entry
    int block, grid, nslot;
    size_t smem;       // dynamic shared memory per block
    uint32_t tile_w;   // walks per tile (single instance)
    uint32_t tiles_per_point;
    uint64_t n_tiles;
};

template <typename Real, int DIM, int KIND, bool MULTI>
const void *walk_kernel_ptr()
{
    return reinterpret_cast<const void *>(&walk_kernel<Real, DIM, KIND, MULTI>);
}

template <typename Real, int DIM, bool MULTI>
const void *pick_walk_kernel(int kind)
{
    if (kind == kSphereOnly) return walk_kernel_ptr<Real, DIM, kSphereOnly, MULTI>();
    if (kind == kBoxOnly) return walk_kernel_ptr<Real, DIM, kBoxOnly, MULTI>();
    if (kind == kSphereHoles) return walk_kernel_ptr<Real, DIM, kSphereHoles, MULTI>();
    if (kind == kAnnulus) return walk_kernel_ptr<Real, DIM, kAnnulus, MULTI>();
    if (kind == kMapped) return walk_kernel_ptr<Real, DIM, kMapped, MULTI>();
    if (kind == kCubeOnly) return walk_kernel_ptr<Real, DIM, kCubeOnly, MULTI>();
    if (kind == kQuadric) return walk_kernel_ptr<Real, DIM, kQuadric, MULTI>();
    if (kind == kQuadricConc) return walk_kernel_ptr<Real, DIM, kQuadricConc, MULTI>();
    return walk_kernel_ptr<Real, DIM, kGeneric, MULTI>();
}

// Kernel kind: specialised distance for a plain disc / ball, a box (a square
// / cube when its half-extents are equal), a disc / ball with holes, or a
// disc / ball with one hole of the same centre.
inline int walk_kind(const wos_domain &d, const wos_partition &part, bool mapped = false)
{
    if (mapped && d.outer_kind == WOS_OUTER_SPHERE) {
        bool concentric = d.n_holes == 1;
        for (int a = 0; a < d.dim; ++a)
            concentric = concentric && d.hole_center[0][a] == d.center[a];
        return concentric ? kQuadricConc : kQuadric;
    }
    if (mapped)
        return kMapped;
    if (part.voronoi_n <= 0 && d.outer_kind == WOS_OUTER_SPHERE) {
        if (d.n_holes == 0)
            return kSphereOnly;
        bool concentric = d.n_holes == 1;
        for (int a = 0; a < d.dim; ++a)
            concentric = concentric && d.hole_center[0][a] == d.center[a];
        return concentric ? kAnnulus : kSphereHoles;
    }
    if (part.voronoi_n <= 0 && d.n_holes == 0 && d.outer_kind == WOS_OUTER_BOX) {
        bool cube = true;
        for (int a = 1; a < d.dim; ++a)
            cube = cube && d.half[a] == d.half[0];
        return cube ? kCubeOnly : kBoxOnly;
    }
    return kGeneric;
}

// Fills an instance record (points_r, tiles and counts pointers are left to
// the caller).
template <typename Real>
void fill_inst(const wos_domain &d, const wos_partition &part, const double *S,
               const double *points, int32_t M_D, uint32_t N, double eps,
               uint32_t stream_id, uint32_t k0, uint32_t k1, uint32_t step_cap,
               uint32_t *counts, uint32_t *unterm, WalkInst<Real> *I, bool mapped = false)
{
    std::memset(I, 0, sizeof(*I));
    fill_geom(d, part, I->g);
    for (int i = 0; i < 9; ++i)
        I->S[i] = i < d.dim * d.dim ? Real(S[i]) : Real(0);
    if (mapped && d.outer_kind == WOS_OUTER_SPHERE) {
        set_quadric(d, S, I->g);  // the paper's moves X + rho S U, larger rho
    } else if (mapped) {  // isotropic steps in y = S^{-1} x
        set_mapped(d, S, I->g);
        for (int i = 0; i < 9; ++i)
            I->S[i] = (i < d.dim * d.dim && i % (d.dim + 1) == 0) ? Real(1) : Real(0);
    }
    I->eps = Real(eps);
    I->stream_id = stream_id;
    I->N = N;
    I->k0 = k0;
    I->k1 = k1 ? k1 : N;
    I->step_cap = step_cap ? step_cap : 1000000u;
    I->M_D = M_D;
    I->points = points;
    I->points_r = nullptr;
    I->counts = counts;
    I->unterm = unterm;
}

// Block size, shared-memory histogram slots per warp (2 when they fit next
// to the exit queues in ~56 KiB per block, so that four blocks share an SM;
// else 1; else none), grid = SMs x resident blocks.
template <typename Real, int DIM, bool MULTI>
wos_status plan_grid(int kind, int32_t max_M_tot, const wos_opts &o, int sm_count,
                     int max_smem_optin, WalkPlan *P)
{
    P->kfn = pick_walk_kernel<Real, DIM, MULTI>(kind);
    P->block = o.block_size > 0 ? o.block_size : 256;
    const int warps = P->block / 32;
    const size_t qbytes = size_t(warps) * queue_bytes<Real, DIM>();
    const size_t slot_bytes = size_t(warps) * size_t((max_M_tot + 1) / 2) * 4;
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
    // the largest shared-memory carveout: an SM running walk blocks keeps
    // room for an SVD cluster CTA beside them (the walks barely use L1)
    cudaFuncSetAttribute(P->kfn, cudaFuncAttributePreferredSharedMemoryCarveout,
                         int(cudaSharedmemCarveoutMaxShared));
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, P->kfn, P->block, P->smem);
    if (e != cudaSuccess)
        return WOS_CUDA_ERROR;
    if (bps < 1)
        return WOS_INVALID_ARG;
    if (o.blocks_per_sm > 0)
        bps = std::min(bps, o.blocks_per_sm);
    P->grid = sm_count * bps;
    return WOS_OK;
}

// Tile size: about tiles_per_warp (default 16) tiles per warp over the whole
// launch, 64..16384 walks, a multiple of 32, at most the walks of one point.
inline uint32_t tile_size(const wos_opts &o, uint64_t total_walks, int grid, int block,
                          uint64_t per_point)
{
    const int warps = block / 32;
    const uint64_t tpw = o.tiles_per_warp > 0 ? uint64_t(o.tiles_per_warp) : 16ull;
    uint64_t tw = o.tile_walks > 0 ? uint64_t(o.tile_walks)
                                   : total_walks / (tpw * uint64_t(grid) * warps);
    tw = std::max<uint64_t>(tw, 64);
    tw = std::min<uint64_t>(tw, 16384);
    tw = (tw + 31) / 32 * 32;
    tw = std::min<uint64_t>(tw, per_point);
    return tw == 0 ? 1u : uint32_t(tw);
}

// Single-instance plan.
template <typename Real>
wos_status plan_walk_any(int dim, int kind, int32_t M_tot, const wos_opts &o, int sm_count,
                         int max_smem_optin, uint64_t per_point, int32_t M_D, WalkPlan *P)
{
    wos_status st = dim == 2
        ? plan_grid<Real, 2, false>(kind, M_tot, o, sm_count, max_smem_optin, P)
        : plan_grid<Real, 3, false>(kind, M_tot, o, sm_count, max_smem_optin, P);
    if (st != WOS_OK)
        return st;
    P->tile_w = tile_size(o, per_point * uint64_t(M_D), P->grid, P->block, per_point);
    P->tiles_per_point = uint32_t((per_point + P->tile_w - 1) / P->tile_w);
    P->n_tiles = uint64_t(P->tiles_per_point) * uint64_t(M_D);
    return WOS_OK;
}

// Fills p.one and the plan fields of a single-instance launch.
template <typename Real>
void apply_plan(const WalkPlan &P, WalkParams<Real> *p)
{
    p->one.tile_w = P.tile_w;
    p->one.tiles_per_point = P.tiles_per_point;
    p->one.tile_begin = 0;
    p->insts = nullptr;
    p->n_inst = 1;
    p->n_tiles = P.n_tiles;
    p->nslot = P.nslot;
    p->hist_words = (p->one.g.M_tot + 1) / 2;
}

inline int32_t refill_min_of(const wos_opts &o)
{
    return o.refill_min > 1 ? std::min(o.refill_min, 32) : 1;
}

// Default group: about 16 steps (3 Philox blocks of 5 steps for FP32 2-D
// walks, 8 of 2 for FP32 3-D and FP64 2-D, 16 of 1 for FP64 3-D); measured
// on the square, annulus, ball and cube operator builds, 12-20 steps per
// group beat 4 by 20-30 % and longer groups lose again.
constexpr int32_t kDefaultGroupSteps = 16;

template <typename Real>
inline int32_t group_blocks_of(const wos_opts &o, int dim)
{
    if (o.group_blocks > 0)
        return std::min(o.group_blocks, 16);
    const int G = dim == 2 ? Steps<Real, 2>::G : Steps<Real, 3>::G;
    return std::max(1, (kDefaultGroupSteps + G / 2) / G);
}

}  // namespace wos
