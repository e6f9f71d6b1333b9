// wos_serve.cu -- request queue with continuous batching (see include/wos.h).
//
// One worker thread per queue.  Each iteration it
//  1. admits queued requests in arrival order while the slot count and the
//     device-memory budget allow (inputs copied to the device, counts zeroed);
//  2. launches one batched walk slice over every admitted request that still
//     has walks to run: request q advances its walk range [k_q, k_q + slice)
//     with accumulate, so its counts stay resident and new arrivals join the
//     next slice; at most two slices are in flight;
//  3. for a request whose walks are complete: FP64 Jacobi SVD on a side stream
//     (after the slice's event), its singular values copied to the host; then
//     the truncation rank on the host and the TSVD reconstruction, results
//     copied back; then the request completes and its memory is released.
// The walks of request q use Philox key = queue seed and counter word =
// q's stream_id: every result equals the same request run alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "wos.h"
#include "wos_internal.h"

namespace {

enum ReqState { kQueued, kWalking, kSvd, kTsvd, kDone, kFailed };

struct Req {
    uint64_t ticket = 0;
    wos_domain dom;
    wos_partition part;
    std::vector<double> sites, points, nu, uD, u0, sigma;
    std::vector<uint8_t> gamma1;
    double K[9];
    int32_t M_D = 0, M_tot = 0, M_1 = 0, M_0 = 0, k = 0, r = 0;
    uint32_t N = 0, stream_id = 0, k_done = 0;
    double eps = 0.0, alpha = 0.0;
    double *out_u1 = nullptr, *out_S = nullptr;
    uint32_t *out_counts = nullptr;
    int32_t *out_r = nullptr;
    size_t footprint = 0;
    // device buffers (one allocation) and pinned host staging
    char *dbuf = nullptr;
    double *d_points = nullptr, *d_nu = nullptr, *d_uD = nullptr, *d_u0 = nullptr;
    double *d_sigma = nullptr, *d_U = nullptr, *d_S = nullptr, *d_V = nullptr, *d_u1 = nullptr;
    uint32_t *d_counts = nullptr;
    char *hbuf = nullptr;
    size_t hbytes = 0;
    double *h_S = nullptr, *h_u1 = nullptr;
    uint32_t *h_counts = nullptr;
    int side = 0;
    cudaEvent_t ev = nullptr;
    std::atomic<int> state{kQueued};  // ReqState; read by waiters
    wos_status status = WOS_NOT_READY;
    int32_t r_used = 0;
    // NULL selects the library's default weights 1/sqrt(M_D)
    const double *nu_ptr() const { return nu.empty() ? nullptr : d_nu; }
};

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Truncation at the first gap S[r-1]/S[r] >= 1.5 after S[r-1]/S[0] < 1e-3,
// else the last gap, else k.
int32_t auto_rank(const double *S, int32_t k)
{
    int32_t last_gap = 0;
    for (int32_t r = 1; r < k; ++r) {
        if (!(S[r] > 0.0))
            break;
        if (S[r - 1] / S[r] >= 1.5) {
            last_gap = r;
            if (S[r - 1] / S[0] < 1e-3)
                return r;
        }
    }
    return last_gap > 0 ? last_gap : k;
}

}  // namespace

struct wos_queue {
    wos_context *ctx = nullptr;
    wos_queue_opts o;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Req>> pending;
    std::vector<std::shared_ptr<Req>> inflight;
    std::map<uint64_t, std::shared_ptr<Req>> tickets;
    uint64_t next_ticket = 1;
    uint64_t budget_used = 0;
    bool stop = false;
    std::thread worker;
    cudaStream_t walk_stream = nullptr;
    std::vector<cudaStream_t> side;
    std::deque<cudaEvent_t> slices;
    // pinned host staging, reused across requests (cudaFreeHost would
    // synchronise the device under running slices)
    std::multimap<size_t, char *> pinned_free;
    std::vector<char *> pinned_all;
    wos_queue_stats stats;
};

namespace {

void finish(wos_queue *q, const std::shared_ptr<Req> &R, wos_status st)
{
    {
        std::lock_guard<std::mutex> lock(q->mu);
        R->status = st;
        R->state = st == WOS_OK ? kDone : kFailed;
        q->budget_used -= R->footprint;
        q->inflight.erase(std::remove(q->inflight.begin(), q->inflight.end(), R),
                          q->inflight.end());
        if (st == WOS_OK) ++q->stats.completed;
        else ++q->stats.failed;
        // release the inputs; the ticket keeps only the status
        R->points.clear(); R->points.shrink_to_fit();
        R->uD.clear(); R->u0.clear(); R->sigma.clear(); R->sites.clear();
        R->gamma1.clear();
    }
    q->cv_done.notify_all();
}

// Device and pinned buffers, inputs to the device (on the walk stream).
wos_status admit(wos_queue *q, Req &R)
{
    const int d = R.dom.dim;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
    const size_t o_pts = take(size_t(R.M_D) * d * 8), o_nu = take(size_t(R.M_D) * 8);
    const size_t o_uD = take(size_t(R.M_D) * 8), o_u0 = take(size_t(std::max(R.M_0, 1)) * 8);
    const size_t o_sig = take(size_t(R.M_tot) * 8);
    const size_t o_cnt = take(size_t(R.M_D) * R.M_tot * 4);
    const size_t o_U = take(size_t(R.M_D) * R.k * 8), o_S = take(size_t(R.k) * 8);
    const size_t o_V = take(size_t(R.M_1) * R.k * 8), o_u1 = take(size_t(R.M_1) * 8);
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&R.dbuf), off, q->walk_stream);
    if (e != cudaSuccess)
        return wos::cuda_status(e);
    R.d_points = reinterpret_cast<double *>(R.dbuf + o_pts);
    R.d_nu = reinterpret_cast<double *>(R.dbuf + o_nu);
    R.d_uD = reinterpret_cast<double *>(R.dbuf + o_uD);
    R.d_u0 = reinterpret_cast<double *>(R.dbuf + o_u0);
    R.d_sigma = reinterpret_cast<double *>(R.dbuf + o_sig);
    R.d_counts = reinterpret_cast<uint32_t *>(R.dbuf + o_cnt);
    R.d_U = reinterpret_cast<double *>(R.dbuf + o_U);
    R.d_S = reinterpret_cast<double *>(R.dbuf + o_S);
    R.d_V = reinterpret_cast<double *>(R.dbuf + o_V);
    R.d_u1 = reinterpret_cast<double *>(R.dbuf + o_u1);
    const size_t hbytes = align256(size_t(R.k) * 8) + align256(size_t(R.M_1) * 8) +
                          (R.out_counts ? size_t(R.M_D) * R.M_tot * 4 : 0);
    auto it = q->pinned_free.lower_bound(hbytes);
    if (it != q->pinned_free.end() && it->first <= 4 * hbytes + 4096) {
        R.hbuf = it->second;
        R.hbytes = it->first;
        q->pinned_free.erase(it);
    } else {
        e = cudaMallocHost(reinterpret_cast<void **>(&R.hbuf), hbytes);
        if (e != cudaSuccess) {
            R.hbuf = nullptr;
            return wos::cuda_status(e);
        }
        R.hbytes = hbytes;
        q->pinned_all.push_back(R.hbuf);
    }
    R.h_S = reinterpret_cast<double *>(R.hbuf);
    R.h_u1 = reinterpret_cast<double *>(R.hbuf + align256(size_t(R.k) * 8));
    R.h_counts = R.out_counts ? reinterpret_cast<uint32_t *>(
                                    R.hbuf + align256(size_t(R.k) * 8) +
                                    align256(size_t(R.M_1) * 8))
                              : nullptr;
    cudaStream_t s = q->walk_stream;
    cudaMemcpyAsync(R.d_points, R.points.data(), R.points.size() * 8, cudaMemcpyHostToDevice, s);
    if (!R.nu.empty())
        cudaMemcpyAsync(R.d_nu, R.nu.data(), R.nu.size() * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(R.d_uD, R.uD.data(), R.uD.size() * 8, cudaMemcpyHostToDevice, s);
    if (!R.u0.empty())
        cudaMemcpyAsync(R.d_u0, R.u0.data(), R.u0.size() * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(R.d_sigma, R.sigma.data(), R.sigma.size() * 8, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(R.d_counts, 0, size_t(R.M_D) * R.M_tot * 4, s);
    if (cudaEventCreateWithFlags(&R.ev, cudaEventDisableTiming) != cudaSuccess)
        return WOS_CUDA_ERROR;
    e = cudaGetLastError();
    return wos::cuda_status(e);
}

// Frees a request's device memory in stream order (on the walk stream while
// its walks may still be queued there, else on its side stream) and returns
// its pinned staging to the pool once nothing can still write it.
void release(wos_queue *q, Req &R)
{
    const bool walking = R.state == kQueued || R.state == kWalking;
    cudaStream_t s = walking ? q->walk_stream : q->side[R.side];
    if (R.dbuf)
        cudaFreeAsync(R.dbuf, s);
    R.dbuf = nullptr;
    if (R.hbuf) {
        if (R.state != kTsvd || (R.ev && cudaEventQuery(R.ev) != cudaSuccess))
            cudaStreamSynchronize(s);  // failure paths only
        q->pinned_free.emplace(R.hbytes, R.hbuf);
    }
    R.hbuf = nullptr;
    if (R.ev)
        cudaEventDestroy(R.ev);
    R.ev = nullptr;
}

void worker_main(wos_queue *q)
{
    cudaSetDevice(q->device);
    int next_side = 0;
    const int32_t max_inflight = q->o.max_inflight > 0 ? q->o.max_inflight : 64;
    const uint64_t budget = q->o.device_budget ? q->o.device_budget : (8ull << 30);
    const uint32_t slice = q->o.slice_walks ? q->o.slice_walks : 4096u;
    for (;;) {
        bool did = false;
        std::vector<std::shared_ptr<Req>> admitted;
        {
            std::unique_lock<std::mutex> lock(q->mu);
            if (q->stop && q->pending.empty() && q->inflight.empty())
                break;
            while (!q->pending.empty() && int32_t(q->inflight.size()) < max_inflight) {
                auto R = q->pending.front();
                if (q->budget_used + R->footprint > budget && !q->inflight.empty())
                    break;
                q->pending.pop_front();
                q->budget_used += R->footprint;
                q->inflight.push_back(R);
                ++q->stats.admitted;
                admitted.push_back(R);
            }
        }
        for (auto &R : admitted) {
            wos_status st = admit(q, *R);
            R->state = kWalking;
            if (st != WOS_OK) {
                release(q, *R);
                finish(q, R, st);
            }
            did = true;
        }
        // ---- one batched slice of walks over every walking request ---------
        std::vector<std::shared_ptr<Req>> walking;
        {
            std::lock_guard<std::mutex> lock(q->mu);
            for (auto &R : q->inflight)
                if (R->state == kWalking)
                    walking.push_back(R);
        }
        if (!walking.empty()) {
            while (q->slices.size() >= 2) {
                cudaEventSynchronize(q->slices.front());
                cudaEventDestroy(q->slices.front());
                q->slices.pop_front();
            }
            std::vector<wos_problem> probs(walking.size());
            uint64_t walks = 0;
            for (size_t i = 0; i < walking.size(); ++i) {
                Req &R = *walking[i];
                wos_problem &pb = probs[i];
                std::memset(&pb, 0, sizeof(pb));
                pb.domain = &R.dom;
                pb.partition = &R.part;
                pb.K = R.K;
                pb.points = R.d_points;
                pb.M_D = R.M_D;
                pb.N = R.N;
                pb.eps = R.eps;
                pb.stream_id = R.stream_id;
                pb.counts = R.d_counts;
                pb.k0 = R.k_done;
                pb.k1 = std::min(R.N, R.k_done + slice);
                walks += uint64_t(R.M_D) * (pb.k1 - pb.k0);
            }
            wos_opts o;
            std::memset(&o, 0, sizeof(o));
            o.precision = q->o.precision;
            o.accumulate = 1;
            wos_status st = wos_build_operators_batched(q->ctx, int32_t(probs.size()),
                                                        probs.data(), q->o.seed, &o, nullptr,
                                                        q->walk_stream);
            cudaEvent_t ev = nullptr;
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            cudaEventRecord(ev, q->walk_stream);
            q->slices.push_back(ev);
            {
                std::lock_guard<std::mutex> lock(q->mu);
                ++q->stats.slices;
                q->stats.walks += walks;
            }
            std::vector<std::shared_ptr<Req>> fin;
            for (size_t i = 0; i < walking.size(); ++i) {
                auto &R = walking[i];
                if (st != WOS_OK) {
                    release(q, *R);
                    finish(q, R, st);
                    continue;
                }
                R->k_done = probs[i].k1;
                if (R->k_done >= R->N)
                    fin.push_back(R);
            }
            if (!fin.empty()) {
                // walks done: their SVDs in one batched pass on a side
                // stream after this slice
                const int side = next_side++ % int(q->side.size());
                cudaStream_t s = q->side[side];
                cudaStreamWaitEvent(s, ev, 0);
                std::vector<wos_svd_problem> sp(fin.size());
                for (size_t i = 0; i < fin.size(); ++i) {
                    Req &R = *fin[i];
                    sp[i] = wos_svd_problem{R.d_counts, R.M_D, R.M_tot, R.N, R.gamma1.data(),
                                            R.nu_ptr(), R.d_sigma, R.d_U, R.d_S, R.d_V};
                }
                wos_status s2 = wos_op_svd_batched(q->ctx, int32_t(sp.size()), sp.data(),
                                                   nullptr, s, nullptr);
                for (auto &R : fin) {
                    R->side = side;
                    cudaMemcpyAsync(R->h_S, R->d_S, size_t(R->k) * 8, cudaMemcpyDeviceToHost, s);
                    cudaEventRecord(R->ev, s);
                    R->state = kSvd;
                    if (s2 != WOS_OK) {
                        release(q, *R);
                        finish(q, R, s2);
                    }
                }
            }
            did = true;
        }
        // ---- SVD done -> truncation rank, reconstruction --------------------
        std::vector<std::shared_ptr<Req>> phase;
        {
            std::lock_guard<std::mutex> lock(q->mu);
            phase = q->inflight;
        }
        for (auto &R : phase) {
            if (R->state != kSvd && R->state != kTsvd)
                continue;
            cudaError_t qe = cudaEventQuery(R->ev);
            if (qe == cudaErrorNotReady)
                continue;
            did = true;
            if (qe != cudaSuccess) {
                release(q, *R);
                finish(q, R, WOS_CUDA_ERROR);
                continue;
            }
            cudaStream_t s = q->side[R->side];
            if (R->state == kSvd) {
                R->r_used = R->r > 0 ? std::min(R->r, R->k) : auto_rank(R->h_S, R->k);
                wos_status st = wos_reconstruct(q->ctx, R->d_U, R->d_S, R->d_V, R->M_D, R->k,
                                                R->d_counts, R->M_tot, R->N, R->gamma1.data(),
                                                R->nu_ptr(), R->d_sigma, R->d_uD,
                                                R->M_0 > 0 && !R->u0.empty() ? R->d_u0 : nullptr,
                                                R->r_used, R->alpha, R->d_u1, nullptr, s);
                cudaMemcpyAsync(R->h_u1, R->d_u1, size_t(R->M_1) * 8, cudaMemcpyDeviceToHost, s);
                if (R->h_counts)
                    cudaMemcpyAsync(R->h_counts, R->d_counts, size_t(R->M_D) * R->M_tot * 4,
                                    cudaMemcpyDeviceToHost, s);
                cudaEventRecord(R->ev, s);
                R->state = kTsvd;
                if (st != WOS_OK) {
                    release(q, *R);
                    finish(q, R, st);
                }
            } else {
                std::memcpy(R->out_u1, R->h_u1, size_t(R->M_1) * 8);
                if (R->out_S)
                    std::memcpy(R->out_S, R->h_S, size_t(R->k) * 8);
                if (R->out_counts)
                    std::memcpy(R->out_counts, R->h_counts, size_t(R->M_D) * R->M_tot * 4);
                if (R->out_r)
                    *R->out_r = R->r_used;
                release(q, *R);
                finish(q, R, WOS_OK);
            }
        }
        if (!did) {  // nothing to launch: sleep until a submit or 50 us
            std::unique_lock<std::mutex> lock(q->mu);
            if (!q->stop)
                q->cv_work.wait_for(lock, std::chrono::microseconds(50));
        }
    }
    while (!q->slices.empty()) {
        cudaEventSynchronize(q->slices.front());
        cudaEventDestroy(q->slices.front());
        q->slices.pop_front();
    }
}

}  // namespace

extern "C" wos_status wos_queue_create(wos_context *ctx, const wos_queue_opts *opts,
                                       wos_queue **out)
{
    if (!ctx || !out)
        return WOS_INVALID_ARG;
    *out = nullptr;
    wos_queue_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts)
        o = *opts;
    if (o.precision != WOS_FP32 && o.precision != WOS_FP64)
        return WOS_INVALID_ARG;
    wos_queue *q = new (std::nothrow) wos_queue();
    if (!q)
        return WOS_OOM;
    q->ctx = ctx;
    q->o = o;
    q->device = wos::ctx_device(ctx);
    std::memset(&q->stats, 0, sizeof(q->stats));
    cudaSetDevice(q->device);
    if (cudaStreamCreateWithFlags(&q->walk_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete q;
        return WOS_CUDA_ERROR;
    }
    const int ns = o.side_streams > 0 ? o.side_streams : 8;
    for (int i = 0; i < ns; ++i) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
            break;
        q->side.push_back(s);
    }
    if (q->side.empty()) {
        cudaStreamDestroy(q->walk_stream);
        delete q;
        return WOS_CUDA_ERROR;
    }
    q->worker = std::thread(worker_main, q);
    *out = q;
    return WOS_OK;
}

extern "C" wos_status wos_queue_destroy(wos_queue *q)
{
    if (!q)
        return WOS_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lock(q->mu);
        q->stop = true;
    }
    q->cv_work.notify_all();
    if (q->worker.joinable())
        q->worker.join();
    cudaSetDevice(q->device);
    cudaStreamSynchronize(q->walk_stream);
    cudaStreamDestroy(q->walk_stream);
    for (cudaStream_t s : q->side) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    for (char *p : q->pinned_all)
        cudaFreeHost(p);
    delete q;
    return WOS_OK;
}

extern "C" wos_status wos_submit(wos_queue *q, const wos_request *rq, uint64_t *ticket)
{
    if (!q || !rq || !ticket || !rq->domain || !rq->partition || !rq->gamma1 || !rq->K ||
        !rq->points || !rq->uD || !rq->u_gamma1 || rq->M_D < 1 || rq->N < 1 ||
        !(rq->eps > 0.0) || rq->r < 0 || rq->tikhonov_alpha < 0.0)
        return WOS_INVALID_ARG;
    wos_status st = wos::validate(rq->domain, rq->partition);
    if (st != WOS_OK)
        return st;
    auto R = std::make_shared<Req>();
    R->dom = *rq->domain;
    R->part = *rq->partition;
    const int d = rq->domain->dim;
    R->M_tot = wos::num_elements(*rq->domain, *rq->partition);
    if (R->M_tot < 1)
        return WOS_INVALID_ARG;
    if (rq->partition->voronoi_n > 0) {
        R->sites.assign(rq->partition->voronoi_sites,
                        rq->partition->voronoi_sites + size_t(rq->partition->voronoi_n) * d);
        R->part.voronoi_sites = R->sites.data();
    }
    double Sroot[9];
    st = wos::setup_S(d, rq->K, Sroot);
    if (st != WOS_OK)
        return st;
    if (q->o.precision == WOS_FP32 && rq->eps < wos::fp32_floor(*rq->domain))
        return WOS_EPS_BELOW_FP32_FLOOR;
    std::memcpy(R->K, rq->K, sizeof(double) * d * d);
    R->gamma1.assign(rq->gamma1, rq->gamma1 + R->M_tot);
    for (uint8_t g : R->gamma1)
        (g ? R->M_1 : R->M_0) += 1;
    if (R->M_1 < 1)
        return WOS_INVALID_ARG;
    R->M_D = rq->M_D;
    R->k = std::min(R->M_D, R->M_1);
    R->N = rq->N;
    R->eps = rq->eps;
    R->stream_id = rq->stream_id;
    R->r = rq->r;
    R->alpha = rq->tikhonov_alpha;
    R->points.assign(rq->points, rq->points + size_t(R->M_D) * d);
    if (rq->nu)
        R->nu.assign(rq->nu, rq->nu + R->M_D);
    R->uD.assign(rq->uD, rq->uD + R->M_D);
    if (rq->u0 && R->M_0 > 0)
        R->u0.assign(rq->u0, rq->u0 + R->M_0);
    R->sigma.resize(R->M_tot);
    st = wos_element_measures(rq->domain, rq->partition, R->sigma.data());
    if (st != WOS_OK)
        return st;
    R->out_u1 = rq->u_gamma1;
    R->out_S = rq->S;
    R->out_counts = rq->counts;
    R->out_r = rq->r_used;
    // device footprint: inputs, counts, U S V, u1, and the SVD workspace
    const size_t m = size_t(std::max(R->M_D, R->M_1)), n = size_t(R->k);
    R->footprint = size_t(R->M_D) * (d + 4) * 8 + size_t(R->M_tot) * 8 +
                   size_t(R->M_D) * R->M_tot * 4 + (size_t(R->M_D) + R->M_1 + 1) * n * 8 +
                   (m * n + n * n + 2 * n) * 8 + 64 * 1024;
    const uint64_t budget = q->o.device_budget ? q->o.device_budget : (8ull << 30);
    if (R->footprint > budget)
        return WOS_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lock(q->mu);
        R->ticket = q->next_ticket++;
        q->tickets[R->ticket] = R;
        q->pending.push_back(R);
        ++q->stats.submitted;
        *ticket = R->ticket;
    }
    q->cv_work.notify_all();
    return WOS_OK;
}

extern "C" wos_status wos_poll(wos_queue *q, uint64_t ticket)
{
    if (!q)
        return WOS_INVALID_ARG;
    std::lock_guard<std::mutex> lock(q->mu);
    auto it = q->tickets.find(ticket);
    if (it == q->tickets.end())
        return WOS_INVALID_ARG;
    return it->second->state == kDone || it->second->state == kFailed ? it->second->status
                                                                      : WOS_NOT_READY;
}

extern "C" wos_status wos_wait(wos_queue *q, uint64_t ticket, int32_t timeout_ms)
{
    if (!q)
        return WOS_INVALID_ARG;
    std::unique_lock<std::mutex> lock(q->mu);
    auto it = q->tickets.find(ticket);
    if (it == q->tickets.end())
        return WOS_INVALID_ARG;
    auto R = it->second;
    auto done = [&] { return R->state == kDone || R->state == kFailed; };
    if (timeout_ms < 0)
        q->cv_done.wait(lock, done);
    else if (!q->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), done))
        return WOS_NOT_READY;
    return R->status;
}

extern "C" wos_status wos_queue_get_stats(wos_queue *q, wos_queue_stats *stats)
{
    if (!q || !stats)
        return WOS_INVALID_ARG;
    std::lock_guard<std::mutex> lock(q->mu);
    *stats = q->stats;
    stats->inflight = int32_t(q->inflight.size());
    stats->queued = int32_t(q->pending.size());
    return WOS_OK;
}
