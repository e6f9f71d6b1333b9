// wos_batch.cu -- many operator builds in one persistent launch per
// class of dimension and kernel kind (spec batching pattern; the paper
// builds one operator at a time with Algorithm MC-REM).
//
// All problems of one call share the Philox key and the walk precision; a
// problem's stream_id is its fourth counter word, so every walk (and every
// count) is bit-identical to the same problem built alone.  The problems of
// one class go into one launch of walk_kernel<..., MULTI = true>: a
// global tile counter spans the tiles of all of them (instance records in
// per-call device scratch), so instances of very different sizes and walk
// lengths keep every warp busy until the last tile.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "voronoi_grid.h"
#include "walk_launch.cuh"
#include "wos.h"
#include "wos_internal.h"

using namespace wos;

namespace {

struct ConvJob {
    const double *src;
    size_t dst_off;  // in elements of the destination array
    int32_t n;       // elements (M_D x dim)
};

template <typename Real>
__global__ void convert_points_batch_kernel(const ConvJob *jobs, Real *dst)
{
    const ConvJob j = jobs[blockIdx.x];
    for (int32_t q = threadIdx.x; q < j.n; q += blockDim.x)
        dst[j.dst_off + q] = Real(j.src[q]);
}

template <typename Real, int DIM>
wos_status launch_class(wos_context *ctx, const std::vector<int> &idx,
                        const wos_problem *probs, const std::vector<std::vector<double>> &S,
                        uint64_t seed, const wos_opts &o_in, cudaStream_t stream,
                        unsigned long long *work_out)
{
    const int n = int(idx.size());
    // kernel kind shared by the whole class, else the generic kernel
    const bool mapped = o_in.mapped != 0;
    int kind = walk_kind(*probs[idx[0]].domain, *probs[idx[0]].partition, mapped);
    int32_t max_M = 0;
    uint64_t total = 0;
    for (int q = 0; q < n; ++q) {
        const wos_problem &pb = probs[idx[q]];
        if (walk_kind(*pb.domain, *pb.partition, mapped) != kind)
            kind = kGeneric;
        max_M = std::max(max_M, num_elements(*pb.domain, *pb.partition));
        const uint32_t k1 = pb.k1 ? pb.k1 : pb.N;
        total += uint64_t(pb.M_D) * (k1 - pb.k0);
    }
    wos_opts o = o_in;
    apply_tuning(ctx, sizeof(Real) == sizeof(double) ? WOS_FP64 : WOS_FP32, DIM, kind, &o);
    WalkPlan plan;
    wos_status st = plan_grid<Real, DIM, true>(kind, max_M, o, ctx_sm_count(ctx),
                                               ctx_max_smem(ctx), &plan);
    if (st != WOS_OK)
        return st;

    // host-side instance records and scratch layout:
    // [work 64 B][instances][conversion jobs][sites][Voronoi grids][points in Real]
    std::vector<WalkInst<Real>> recs(n);
    std::vector<ConvJob> jobs;
    std::vector<VoronoiGrid> grids(n);
    std::vector<char> has_grid(n, 0);
    std::vector<int32_t> host_grid;  // every grid's offsets then candidates
    std::vector<size_t> grid_at(n, 0);
    size_t sites_elems = 0, pts_elems = 0;
    for (int q = 0; q < n; ++q) {
        const wos_problem &pb = probs[idx[q]];
        if (pb.partition->voronoi_n > 0) {
            sites_elems += size_t(pb.partition->voronoi_n) * DIM;
            if (build_voronoi_grid(*pb.domain, *pb.partition, &grids[q])) {
                has_grid[q] = 1;
                grid_at[q] = host_grid.size();
                host_grid.insert(host_grid.end(), grids[q].start.begin(), grids[q].start.end());
                host_grid.insert(host_grid.end(), grids[q].cand.begin(), grids[q].cand.end());
            }
        }
        pts_elems += size_t(pb.M_D) * DIM;
    }
    const bool convert = sizeof(Real) != sizeof(double);
    auto align = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t off_inst = 256;
    const size_t off_jobs = off_inst + align(sizeof(WalkInst<Real>) * n);
    const size_t off_sites = off_jobs + align(sizeof(ConvJob) * n);
    const size_t off_grid = off_sites + align(sites_elems * sizeof(Real));
    const size_t off_pts = off_grid + align(host_grid.size() * sizeof(int32_t));
    const size_t bytes = off_pts + (convert ? pts_elems * sizeof(Real) : 0);
    char *scratch = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&scratch), bytes, stream);
    if (e != cudaSuccess)
        return cuda_status(e);
    Real *dsites = reinterpret_cast<Real *>(scratch + off_sites);
    Real *dpts = reinterpret_cast<Real *>(scratch + off_pts);
    std::vector<Real> host_sites(sites_elems);
    size_t s_at = 0, p_at = 0;
    uint64_t tile_at = 0;
    for (int q = 0; q < n; ++q) {
        const wos_problem &pb = probs[idx[q]];
        WalkInst<Real> &I = recs[q];
        fill_inst<Real>(*pb.domain, *pb.partition, S[idx[q]].data(), pb.points, pb.M_D, pb.N,
                        pb.eps, pb.stream_id, pb.k0, pb.k1, pb.step_cap, pb.counts,
                        pb.unterminated, &I, mapped);
        if (pb.partition->voronoi_n > 0) {
            const size_t ns = size_t(pb.partition->voronoi_n) * DIM;
            for (size_t k = 0; k < ns; ++k)
                host_sites[s_at + k] = Real(pb.partition->voronoi_sites[k]);
            I.g.vsites = dsites + s_at;
            s_at += ns;
            if (has_grid[q]) {
                const int32_t *dg = reinterpret_cast<const int32_t *>(scratch + off_grid) +
                                    grid_at[q];
                set_voronoi_grid(grids[q], dg, dg + grids[q].start.size(), I.g);
            }
        }
        if (convert) {
            jobs.push_back(ConvJob{pb.points, p_at, pb.M_D * DIM});
            I.points_r = dpts + p_at;
            p_at += size_t(pb.M_D) * DIM;
        }
        const uint32_t per_point = I.k1 - I.k0;
        I.tile_w = tile_size(o, total, plan.grid, plan.block, uint64_t(per_point));
        I.tiles_per_point = (per_point + I.tile_w - 1) / I.tile_w;
        I.tile_begin = tile_at;
        tile_at += uint64_t(I.tiles_per_point) * uint64_t(pb.M_D);
        if (!o.accumulate) {
            cudaMemsetAsync(pb.counts, 0,
                            size_t(pb.M_D) * size_t(I.g.M_tot) * sizeof(uint32_t), stream);
            if (pb.unterminated)
                cudaMemsetAsync(pb.unterminated, 0, size_t(pb.M_D) * sizeof(uint32_t), stream);
        }
    }
    cudaMemsetAsync(scratch, 0, 64, stream);
    cudaMemcpyAsync(scratch + off_inst, recs.data(), sizeof(WalkInst<Real>) * n,
                    cudaMemcpyHostToDevice, stream);
    if (sites_elems)
        cudaMemcpyAsync(dsites, host_sites.data(), sites_elems * sizeof(Real),
                        cudaMemcpyHostToDevice, stream);
    if (!host_grid.empty())
        cudaMemcpyAsync(scratch + off_grid, host_grid.data(), host_grid.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice, stream);
    if (convert) {
        cudaMemcpyAsync(scratch + off_jobs, jobs.data(), sizeof(ConvJob) * jobs.size(),
                        cudaMemcpyHostToDevice, stream);
        convert_points_batch_kernel<Real><<<int(jobs.size()), 256, 0, stream>>>(
            reinterpret_cast<const ConvJob *>(scratch + off_jobs), dpts);
        count_launches(ctx, 1);
    }
    WalkParams<Real> *pp = new (std::nothrow) WalkParams<Real>();
    if (!pp) {
        cudaFreeAsync(scratch, stream);
        return WOS_OOM;
    }
    std::memset(pp, 0, sizeof(*pp));
    pp->insts = reinterpret_cast<const WalkInst<Real> *>(scratch + off_inst);
    pp->n_inst = n;
    philox_round_keys(seed, pp->rk);
    pp->n_tiles = tile_at;
    pp->work = reinterpret_cast<unsigned long long *>(scratch);
    pp->nslot = plan.nslot;
    pp->hist_words = (max_M + 1) / 2;
    pp->refill_min = refill_min_of(o);
    pp->group_blocks = group_blocks_of<Real>(o, DIM);
    if (o.kernel_events[0])
        cudaEventRecord(static_cast<cudaEvent_t>(o.kernel_events[0]), stream);
    void *args[] = {pp};
    e = cudaLaunchKernel(plan.kfn, dim3(plan.grid), dim3(plan.block), args, plan.smem, stream);
    count_launches(ctx, 1);
    if (o.kernel_events[1])
        cudaEventRecord(static_cast<cudaEvent_t>(o.kernel_events[1]), stream);
    delete pp;
    if (e == cudaSuccess && work_out)
        cudaMemcpyAsync(work_out, scratch, 5 * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, stream);
    cudaFreeAsync(scratch, stream);
    return cuda_status(e);
}

}  // namespace

extern "C" wos_status wos_build_operators_batched(wos_context *ctx, int32_t n,
                                                  const wos_problem *problems,
                                                  uint64_t seed, const wos_opts *opts,
                                                  wos_stats *stats, void *stream)
{
    if (!ctx || n < 1 || !problems)
        return WOS_INVALID_ARG;
    wos_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts)
        o = *opts;
    if (o.precision != WOS_FP32 && o.precision != WOS_FP64)
        return WOS_INVALID_ARG;
    if (o.block_size && (o.block_size % 32 != 0 || o.block_size > 256))
        return WOS_INVALID_ARG;
    if (o.hist_slots < -1 || o.hist_slots > 2 || o.k0 || o.k1 || o.trace_elem ||
        o.trace_steps || o.trace_x)
        return WOS_INVALID_ARG;  // whole walk ranges only, no traces, in a batch
    std::vector<std::vector<double>> S(n, std::vector<double>(9, 0.0));
    // classes: dimension x kernel kind, one launch each
    std::vector<int> by_class[2][kNumKinds];
    for (int q = 0; q < n; ++q) {
        const wos_problem &pb = problems[q];
        wos_status st = validate(pb.domain, pb.partition);
        if (st != WOS_OK)
            return st;
        const uint32_t k1 = pb.k1 ? pb.k1 : pb.N;
        if (pb.M_D < 1 || pb.N < 1 || !pb.points || !pb.counts || !(pb.eps > 0.0) ||
            pb.k0 >= k1 || k1 > pb.N)
            return WOS_INVALID_ARG;
        if (num_elements(*pb.domain, *pb.partition) < 1)
            return WOS_INVALID_ARG;
        st = setup_S(pb.domain->dim, pb.K, S[q].data());
        if (st != WOS_OK)
            return st;
        if (o.mapped != 0 && (o.mapped != 1 || !mapped_supported(*pb.domain)))
            return WOS_INVALID_ARG;
        const bool in_y = o.mapped && pb.domain->outer_kind != WOS_OUTER_SPHERE;
        if (o.precision == WOS_FP32 &&
            pb.eps < (in_y ? fp32_floor_mapped(*pb.domain, S[q].data())
                           : fp32_floor(*pb.domain)))
            return WOS_EPS_BELOW_FP32_FLOOR;
        by_class[pb.domain->dim - 2][walk_kind(*pb.domain, *pb.partition, o.mapped != 0)]
            .push_back(q);
    }
    cudaSetDevice(ctx_device(ctx));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long w[2 * kNumKinds][5] = {};
    // Within a class the instances go longest walks first (smallest eps:
    // E[N_eps] grows with log 1/eps, then the most walks), so that the tiles
    // drawn last are short and the launch drains quickly.  The order of the
    // tiles changes no walk: each walk's random numbers are fixed by its
    // counter.
    auto work_of = [&](int q) {
        const wos_problem &pb = problems[q];
        const uint32_t k1 = pb.k1 ? pb.k1 : pb.N;
        return double(pb.M_D) * double(k1 - pb.k0) * std::log(1.0 / pb.eps);
    };
    std::vector<int> order;  // classes, the most work first
    std::vector<double> cwork(2 * kNumKinds, 0.0);
    for (int c = 0; c < 2 * kNumKinds; ++c) {
        std::vector<int> &cls = by_class[c / kNumKinds][c % kNumKinds];
        if (cls.empty())
            continue;
        std::stable_sort(cls.begin(), cls.end(), [&](int a, int b) {
            if (problems[a].eps != problems[b].eps)
                return problems[a].eps < problems[b].eps;
            return work_of(a) > work_of(b);
        });
        for (int q : cls)
            cwork[c] += work_of(q);
        order.push_back(c);
    }
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return cwork[a] > cwork[b]; });
    // The classes run concurrently, each on a stream of the context forked
    // from `stream` and joined back to it: the persistent launches queue in
    // order of their work, and each one's blocks take the SMs the previous
    // one frees as it drains (one stream when the caller times the kernel).
    const bool concurrent = order.size() > 1 && !o.kernel_events[0] && !o.kernel_events[1];
    cudaEvent_t fork = nullptr;
    if (concurrent && (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
                       cudaEventRecord(fork, s) != cudaSuccess))
        return WOS_CUDA_ERROR;
    wos_status st = WOS_OK;
    for (int c : order) {
        const int dd = c / kNumKinds, kk = c % kNumKinds;
        const std::vector<int> &cls = by_class[dd][kk];
        cudaStream_t cs = s;
        if (concurrent) {
            cs = ctx_class_stream(ctx, c);
            if (!cs || cudaStreamWaitEvent(cs, fork, 0) != cudaSuccess) {
                st = WOS_CUDA_ERROR;
                break;
            }
        }
        unsigned long long *wo = stats ? w[c] : nullptr;
        if (o.precision == WOS_FP64)
            st = dd == 0 ? launch_class<double, 2>(ctx, cls, problems, S, seed, o, cs, wo)
                         : launch_class<double, 3>(ctx, cls, problems, S, seed, o, cs, wo);
        else
            st = dd == 0 ? launch_class<float, 2>(ctx, cls, problems, S, seed, o, cs, wo)
                         : launch_class<float, 3>(ctx, cls, problems, S, seed, o, cs, wo);
        if (concurrent) {
            cudaEvent_t join = nullptr;
            if (cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventRecord(join, cs) != cudaSuccess ||
                cudaStreamWaitEvent(s, join, 0) != cudaSuccess)
                st = st == WOS_OK ? WOS_CUDA_ERROR : st;
            if (join)
                cudaEventDestroy(join);
        }
        if (st != WOS_OK)
            break;
    }
    if (fork)
        cudaEventDestroy(fork);
    if (st != WOS_OK)
        return st;
    if (!stats)
        return WOS_OK;
    st = cuda_status(cudaStreamSynchronize(s));
    std::memset(stats, 0, sizeof(*stats));
    for (int c = 0; c < 2 * kNumKinds; ++c) {
        stats->steps += w[c][1];
        stats->walks += w[c][2];
        stats->unterminated += w[c][3];
        stats->max_steps = std::max<uint32_t>(stats->max_steps, uint32_t(w[c][4]));
    }
    if (st == WOS_OK && stats->unterminated > 0)
        st = WOS_STEP_CAP_HIT;
    return st;
}
