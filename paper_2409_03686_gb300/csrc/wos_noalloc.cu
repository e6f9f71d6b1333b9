// wos_noalloc.cu -- wos_build_operator_noalloc: the operator build for callers
// that must not allocate device memory.
//
// Some callers cannot call cudaMalloc (or cudaMallocAsync) at all: a process
// that runs under a device-memory budget reserved up front and admits work
// only by its footprint, or code hosted inside a framework that owns every
// device allocation (its own pool, its own accounting) and forbids others'.
// For them this entry point does the same build as wos_build_operator but
// takes its scratch -- the work-queue counter, the statistics counters and,
// for extrinsic Voronoi partitions, the site table -- from one fixed array in
// device memory that the library defines at file scope.  The caller still
// passes (and owns) every input and output array.
//
// The array is kNoAllocScratchBytes = 64 KiB: 256 bytes of counters, then at
// most kNoAllocMaxSites = 2048 Voronoi sites.  Every GPU that loads the library
// holds those 64 KiB until the process exits.  All calls on a device share the
// array and it keeps the last call's contents; each call clears the counters
// that must start at zero before its kernel runs.  Calls whose device work
// overlaps on the GPU (different streams, or no ordering between them) race
// on the array: order them on one stream or with events.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "walk_launch.cuh"
#include "wos.h"
#include "wos_internal.h"

using namespace wos;

namespace {

constexpr size_t kNoAllocScratchBytes = 64 * 1024;
constexpr size_t kCounterBytes = 256;
constexpr int32_t kNoAllocMaxSites = 2048;
constexpr int kMaxDevices = 64;
static_assert(kCounterBytes + size_t(kNoAllocMaxSites) * 3 * sizeof(double) <=
                  kNoAllocScratchBytes,
              "the site table must fit the scratch array");

// The scratch array.  In host code this name is only a stand-in for the
// symbol: its device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_addr_mu;
void *g_addr[kMaxDevices];
bool g_addr_ready[kMaxDevices];

// Device address of g_noalloc_scratch on `device` (which must be current).
// The first call on a device looks it up; later calls reuse it.
wos_status scratch_address(int device, unsigned char **out)
{
    if (device < 0 || device >= kMaxDevices)
        return WOS_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr_ready[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return e == cudaSuccess ? WOS_CUDA_ERROR : cuda_status(e);
        g_addr[device] = p;
        g_addr_ready[device] = true;
    }
    *out = static_cast<unsigned char *>(g_addr[device]);
    return WOS_OK;
}

template <typename Real>
wos_status build_noalloc(wos_context *ctx, unsigned char *scratch, const wos_domain &d,
                         const wos_partition &part, const double *S, const double *points,
                         int32_t M_D, uint32_t N, double eps, uint64_t seed,
                         const wos_opts &o_in, uint32_t *counts, uint32_t *unterm,
                         wos_stats *stats, cudaStream_t stream)
{
    WalkParams<Real> p;  // host stack, passed by value to the kernel
    std::memset(&p, 0, sizeof(p));
    const int dim = d.dim;
    wos_opts o = o_in;
    apply_tuning(ctx, sizeof(Real) == sizeof(double) ? WOS_FP64 : WOS_FP32, dim,
                 walk_kind(d, part, o.mapped != 0), &o);
    fill_inst<Real>(d, part, S, points, M_D, N, eps, o.stream_id, o.k0, o.k1, o.step_cap,
                    counts, unterm, &p.one, o.mapped != 0);  // points_r null: per walk
    philox_round_keys(seed, p.rk);
    p.trace_elem = o.trace_elem;
    p.trace_steps = o.trace_steps;
    p.trace_x = o.trace_x;
    const int32_t M = p.one.g.M_tot;

    WalkPlan plan;
    wos_status pst = plan_walk_any<Real>(dim, walk_kind(d, part, o.mapped != 0), M, o,
                                         ctx_sm_count(ctx),
                                         ctx_max_smem(ctx), uint64_t(p.one.k1 - p.one.k0),
                                         M_D, &plan);
    if (pst != WOS_OK)
        return pst;
    apply_plan(plan, &p);
    p.refill_min = refill_min_of(o);
    p.group_blocks = group_blocks_of<Real>(o, dim);
    const void *kfn = plan.kfn;
    const int grid = plan.grid, block = plan.block, nslot = plan.nslot;
    const size_t smem = plan.smem;
    const uint64_t tw = plan.tile_w;
    cudaError_t e = cudaSuccess;

    // scratch: counters at offset 0 (cleared every call), sites after them
    p.work = reinterpret_cast<unsigned long long *>(scratch);
    if (part.voronoi_n > 0) {
        Real staging[size_t(kNoAllocMaxSites) * 3];  // host stack, no allocation
        const size_t n = size_t(part.voronoi_n) * dim;
        for (size_t q = 0; q < n; ++q)
            staging[q] = Real(part.voronoi_sites[q]);
        Real *dsites = reinterpret_cast<Real *>(scratch + kCounterBytes);
        // pageable source: returns once the staging buffer has been read
        e = cudaMemcpyAsync(dsites, staging, n * sizeof(Real), cudaMemcpyHostToDevice,
                            stream);
        if (e != cudaSuccess)
            return cuda_status(e);
        p.one.g.vsites = dsites;
    }
    e = cudaMemsetAsync(scratch, 0, kCounterBytes, stream);
    if (e != cudaSuccess)
        return cuda_status(e);
    // observation points outside D: no walk runs (work[0] past every tile)
    e = launch_point_check(d, part, points, M_D, p.work, stream);
    count_launches(ctx, 1);
    if (e != cudaSuccess)
        return cuda_status(e);
    if (!o.accumulate) {
        e = cudaMemsetAsync(counts, 0, size_t(M_D) * M * 4, stream);
        if (e == cudaSuccess && unterm)
            e = cudaMemsetAsync(unterm, 0, size_t(M_D) * 4, stream);
        if (e != cudaSuccess)
            return cuda_status(e);
    }
    if (o.kernel_events[0])
        cudaEventRecord(static_cast<cudaEvent_t>(o.kernel_events[0]), stream);
    void *args[] = {&p};
    e = cudaLaunchKernel(kfn, dim3(grid), dim3(block), args, smem, stream);
    count_launches(ctx, 1);
    if (o.kernel_events[1])
        cudaEventRecord(static_cast<cudaEvent_t>(o.kernel_events[1]), stream);
    wos_status st = cuda_status(e);
    if (st == WOS_OK && stats) {
        unsigned long long w[6] = {0, 0, 0, 0, 0, 0};
        cudaMemcpyAsync(w, scratch, sizeof(w), cudaMemcpyDeviceToHost, stream);
        st = cuda_status(cudaStreamSynchronize(stream));
        std::memset(stats, 0, sizeof(*stats));
        stats->steps = w[1];
        stats->walks = w[2];
        stats->unterminated = w[3];
        stats->max_steps = uint32_t(w[4]);
        stats->grid = grid;
        stats->block = block;
        stats->tile_walks = int32_t(tw);
        stats->hist_slots = nslot;
        if (st == WOS_OK && w[5] > 0)
            st = WOS_POINT_OUTSIDE;
        else if (st == WOS_OK && w[3] > 0)
            st = WOS_STEP_CAP_HIT;
    }
    return st;
}

}  // namespace

extern "C" wos_status wos_build_operator_noalloc(
    wos_context *ctx, const wos_domain *domain, const double *K, const double *points,
    int32_t M_D, const wos_partition *partition, uint32_t N, double eps, uint64_t seed,
    const wos_opts *opts, uint32_t *counts, uint32_t *unterminated, wos_stats *stats,
    void *stream)
{
    // the checks of wos_build_operator, then the limit of the fixed scratch
    wos_opts o;
    double S[9];
    wos_status st = validate_build(ctx, domain, K, points, M_D, partition, N, eps, opts,
                                   counts, &o, S);
    if (st != WOS_OK)
        return st;
    if (partition->voronoi_n > kNoAllocMaxSites)
        return WOS_NOALLOC_LIMIT;
    const int dev = ctx_device(ctx);
    if (cudaSetDevice(dev) != cudaSuccess)
        return WOS_CUDA_ERROR;
    unsigned char *scratch = nullptr;
    st = scratch_address(dev, &scratch);
    if (st != WOS_OK)
        return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (o.precision == WOS_FP64)
        return build_noalloc<double>(ctx, scratch, *domain, *partition, S, points, M_D, N,
                                     eps, seed, o, counts, unterminated, stats, s);
    return build_noalloc<float>(ctx, scratch, *domain, *partition, S, points, M_D, N, eps,
                                seed, o, counts, unterminated, stats, s);
}
