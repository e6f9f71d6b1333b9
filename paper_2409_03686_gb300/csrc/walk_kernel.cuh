// walk_kernel.cuh -- the persistent walk-on-ellipsoids kernel (MC-REM body).
//
// Paper: Cimpean, Grecu & Marin, arXiv:2409.03686, Sec. 5.1, Algorithm
// MC-REM; Sec. 4.2, Eq. (wos chain) and (N epsilon x); Sec. 4.3,
// Eq. (WoE_matrix_MC).
//
// Design (one GB300, no tensor cores: the chain is scalar ALU/SFU work):
//  * Persistent grid: blocks_per_SM x SMs; every warp loops until the tile
//    queue is empty and its lanes are idle.
//  * Work = walks (instance, point i, walk k).  A tile is a run of walks of
//    one point; warps take tiles from a global counter (one atomic per tile).
//    One launch serves one instance (its record in the constant bank) or a
//    batch of instances of one precision and dimension (records in global
//    memory, each lane reading its own walk's record through L1).
//  * Every lane owns one walk at a time.  Walks advance in groups of
//    group_blocks x G steps, G steps per Philox4x32-10 block (G = 5 for FP32
//    2-D walks, which take 23-bit windows of the 128 bits, else 4 words /
//    words per step), so all lanes call Philox together; a lane whose walk
//    stops mid-group idles to the group's end.  At a group boundary the
//    finished lanes are refilled from the warp's tile (warp-level refill:
//    ballot + popc ranks), so warps stay full despite geometric walk
//    lengths.  Longer groups spread the refill and queue bookkeeping over
//    more steps at the price of more idle lane-steps after a walk stops.
//  * The Philox counter of step n of walk w is (n / G, w lo, w hi, stream):
//    results do not depend on scheduling or on the batch a walk runs in.
//  * Kinds whose distance depends on x - c only (disc / ball, box, cube,
//    annulus / shell) walk in coordinates relative to the centre c: the
//    start point is shifted once per tile and the exit point back once per
//    walk, which takes a subtraction per coordinate off every step (the same
//    bits when c = 0; otherwise a rounding of the sum in another place).
//  * A finished lane only pushes its stopped point into a per-warp queue in
//    shared memory; once 32 are queued the whole warp classifies them (pi of
//    App. A) and tallies them at full lane efficiency.
//  * Tally: each warp owns up to two shared-memory histograms (one per tile in
//    flight), two uint16 counts per 32-bit word (a tile has < 65536 walks).
//    A slot is flushed to HBM with coalesced integer atomics when its tile is
//    retired; a walk that outlives its slot (generation mismatch) adds to HBM
//    directly.  No inter-warp synchronisation anywhere.
#pragma once

#include <cuda_runtime.h>

#include "wos_device.cuh"

namespace wos {

// Kernel kinds: any domain; a disc / ball; a box; a disc / ball with holes;
// a disc / ball with one concentric hole (annulus, spherical shell: both
// boundary distances come from one radius); mapped walks (walk-on-spheres in
// y = S^{-1} x, the domain a convex polytope given by its faces); a box with
// equal half-extents (square, cube: h - max |x_a|); mapped walks on a disc /
// ball minus holes (steps of the largest ellipsoid X + rho S B inside D, rho
// a quadric lower bound of the distance in y), the general form and the one
// with a single concentric hole.
enum KernelKind : int {
    kGeneric = 0, kSphereOnly = 1, kBoxOnly = 2, kSphereHoles = 3, kAnnulus = 4,
    kMapped = 5, kCubeOnly = 6, kQuadric = 7, kQuadricConc = 8
};
constexpr int kNumKinds = 9;

// One instance of the operator build.
template <typename Real> struct WalkInst {
    Geom<Real> g;
    Real S[9];            // (K / lambda_max)^{1/2}, row-major DIM x DIM
    Real eps;
    uint32_t stream_id;   // fourth Philox counter word
    uint32_t N;           // walks per point: walk id = i * N + k
    uint32_t k0, k1;      // walk range of every point
    uint32_t step_cap;
    int32_t M_D;
    const double *points; // device, M_D x DIM
    const Real *points_r; // the same in walk precision, or null (convert here)
    uint32_t *counts;     // device, M_D x M_tot
    uint32_t *unterm;     // device, M_D (may be null)
    uint32_t tile_w;      // walks per tile
    uint32_t tiles_per_point;
    uint64_t tile_begin;  // first global tile of this instance (batches)
};

template <typename Real> struct WalkParams {
    WalkInst<Real> one;          // the instance of a single-instance launch
    const WalkInst<Real> *insts; // batch: instance records (device)
    int32_t n_inst;
    uint32_t rk[20];             // Philox key schedule (shared by a batch)
    int32_t *trace_elem;         // optional traces (single instance; tests)
    uint32_t *trace_steps;
    double *trace_x;
    uint64_t n_tiles;
    unsigned long long *work;    // [0] tile counter, [1] steps, [2] walks,
                                 // [3] unterminated, [4] max steps
    int32_t nslot;               // 0 (global tally), 1 or 2
    int32_t hist_words;          // ceil(M_tot / 2), max over a batch
    int32_t refill_min;          // refill when >= this many lanes need a walk
    int32_t group_blocks;        // Philox blocks per group of steps (>= 1)
};

template <typename Real, int DIM> struct Steps {
    // steps served by one Philox block: five 23-bit windows for FP32 2-D
    // walks, else whole words (one or two per uniform)
    static constexpr bool kPacked = DIM == 2 && sizeof(Real) == 4;
    static constexpr int kWordsPerStep = (DIM == 2 ? 1 : 2) * Uniform<Real>::kWords;
    static constexpr int G = kPacked ? kPacked2dSteps : 4 / kWordsPerStep;
};

// Direction of step s of a Philox block.
template <typename Real, int DIM>
__device__ __forceinline__ void step_direction(const uint32_t *w, int s, Real *U)
{
    if constexpr (Steps<Real, DIM>::kPacked) {
        const uint32_t win = window23(w, s);
        direction<Real, DIM>(&win, U);
    } else {
        direction<Real, DIM>(w + s * Steps<Real, DIM>::kWordsPerStep, U);
    }
}

template <typename Real, int DIM, int KIND>
__device__ __forceinline__ Real walk_dist(const Geom<Real> &g, const Real *x)
{
    if (KIND == kSphereOnly) {  // x relative to the centre
        Real s = x[0] * x[0];
#pragma unroll
        for (int a = 1; a < DIM; ++a)
            s = fma(x[a], x[a], s);
        return g.R - w_sqrt(s);
    }
    if (KIND == kBoxOnly) {  // x relative to the centre
        Real best = g.h[0] - w_fabs(x[0]);
#pragma unroll
        for (int a = 1; a < DIM; ++a)
            best = w_min(best, g.h[a] - w_fabs(x[a]));
        return best;
    }
    if (KIND == kCubeOnly) {  // x relative to the centre; every h[a] = h[0]
        // h - max_a |x_a| = min_a (h - |x_a|) bit for bit (the rounding of
        // h - t is monotone in t), one subtraction fewer
        Real m = w_fabs(x[0]);
#pragma unroll
        for (int a = 1; a < DIM; ++a)
            m = w_max(m, w_fabs(x[a]));
        return g.h[0] - m;
    }
    if (KIND == kSphereHoles) {
        Real r = sphere_dist<Real, DIM>(g, x);
        for (int h = 0; h < g.n_holes; ++h)
            r = w_min(r, hole_dist<Real, DIM>(g, h, x));
        return r;
    }
    if (KIND == kMapped) {  // exact distance to the polytope S^{-1} D
        Real r = g.pd[0];
#pragma unroll
        for (int a = 0; a < DIM; ++a)
            r = fma(-g.pn[0][a], x[a], r);
#pragma unroll
        for (int f = 1; f < kMaxPlanes; ++f) {
            if (f < g.np) {
                Real s = g.pd[f];
#pragma unroll
                for (int a = 0; a < DIM; ++a)
                    s = fma(-g.pn[f][a], x[a], s);
                r = w_min(r, s);
            }
        }
        return r;
    }
    if (KIND == kQuadric || KIND == kQuadricConc) {
        // Mapped chain on a disc / ball minus holes.  The largest rho with
        // X + rho S B(0, 1) inside D is the distance in y = S^{-1} x to the
        // mapped boundary (ellipses / ellipsoids); per component a lower
        // bound from a quadratic majorant of |S y - c|^2 - R^2 along a ray
        // (v = x - c, w = S v, lambda_max(S) = 1):
        //   outer:  (R^2 - |v|^2) / (|w| + sqrt(|w|^2 + R^2 - |v|^2)),
        //   hole:   max(F / (|w| + sqrt(|w|^2 - mu^2 F)), |v| - r),
        //           F = |v|^2 - r^2, mu = lambda_min(S);
        // both first-order exact at the boundary and >= the Euclidean
        // distance, <= 0 outside D (the walk then stops).  R^2 - |v|^2 is
        // formed as (R - |v|)(R + |v|), which keeps its digits near dD.
        Real v[DIM], rho2 = Real(0), w2 = Real(0);
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            v[a] = x[a] - g.c[a];
            rho2 = fma(v[a], v[a], rho2);
        }
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            Real wa = g.mS[a * DIM] * v[0];
#pragma unroll
            for (int b = 1; b < DIM; ++b)
                wa = fma(g.mS[a * DIM + b], v[b], wa);
            w2 = fma(wa, wa, w2);
        }
        const Real rho = w_sqrt(rho2), wn = w_sqrt(w2);
        const Real F0 = (g.R - rho) * (g.R + rho);
        Real r = w_div(F0, wn + w_sqrt(w_max(Real(0), w2 + F0)));
        if (KIND == kQuadricConc) {  // one hole of the same centre: v, w shared
            const Real r1 = g.hr[0];
            const Real F = (rho - r1) * (rho + r1);
            const Real sh = w_div(F, wn + w_sqrt(w_max(Real(0), fma(-g.qmu2, F, w2))));
            r = w_min(r, w_max(sh, rho - r1));
        } else {
            for (int h = 0; h < g.n_holes; ++h) {
                Real p2 = Real(0), q2 = Real(0), u[DIM];
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    u[a] = x[a] - g.hc[h][a];
                    p2 = fma(u[a], u[a], p2);
                }
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    Real wa = g.mS[a * DIM] * u[0];
#pragma unroll
                    for (int b = 1; b < DIM; ++b)
                        wa = fma(g.mS[a * DIM + b], u[b], wa);
                    q2 = fma(wa, wa, q2);
                }
                const Real p = w_sqrt(p2), r1 = g.hr[h];
                const Real F = (p - r1) * (p + r1);
                const Real sh = w_div(F, w_sqrt(q2) + w_sqrt(w_max(Real(0), fma(-g.qmu2, F, q2))));
                r = w_min(r, w_max(sh, p - r1));
            }
        }
        return r;
    }
    if (KIND == kAnnulus) {  // |x - c| once; both boundary distances from it
        Real s = Real(0);
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            s += x[a] * x[a];  // x relative to the centre
        }
        const Real rho = w_sqrt(s);
        return g.ahalf - w_fabs(rho - g.amid);  // = min(R - rho, rho - r_1)
    }
    return domain_dist<Real, DIM>(g, x);
}

// The element of a stopped point, with only the code the kernel kind needs.
template <typename Real, int DIM, int KIND>
__device__ __forceinline__ int32_t walk_classify(const Geom<Real> &g, const Real *x)
{
    if (KIND == kSphereOnly)
        return outer_sphere_cell<Real, DIM>(g, x);
    if (KIND == kBoxOnly || KIND == kCubeOnly)
        return outer_box_cell<Real, DIM>(g, x);
    if (KIND == kSphereHoles || KIND == kAnnulus)
        return sphere_holes_cell<Real, DIM>(g, x);
    if ((KIND == kQuadric || KIND == kQuadricConc) && g.vn == 0)
        return sphere_holes_cell<Real, DIM>(g, x);
    if (KIND == kMapped && g.vn == 0 && g.n_holes == 0 && g.outer_kind == kBox)
        return outer_box_cell<Real, DIM>(g, x);
    return classify<Real, DIM>(g, x);
}

// X += re S U (re = 0 leaves X as it is: a stopped walk keeps its point).
template <typename Real, int DIM>
__device__ __forceinline__ void step_move(const Real *S, const Real *U, Real re, Real *X)
{
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        Real su = S[a * DIM] * U[0];
#pragma unroll
        for (int b = 1; b < DIM; ++b)
            su = fma(S[a * DIM + b], U[b], su);
        X[a] = fma(re, su, X[a]);
    }
}

constexpr int kQueue = 64;  // per-warp exit queue (entries)

// Shared-memory bytes of one warp's exit queue: DIM coordinates and five
// words (point, instance, walk k, slot generation, N_eps) per entry.
template <typename Real, int DIM>
__host__ __device__ constexpr size_t queue_bytes()
{
    return size_t(kQueue) * (DIM * sizeof(Real) + 5 * sizeof(uint32_t));
}

// Flush one warp-private slot into a counts row.
__device__ __forceinline__ void flush_slot(uint32_t *slot, int32_t words,
                                           uint32_t *counts_row, int lane)
{
    for (int32_t w = lane; w < words; w += 32) {
        uint32_t v = slot[w];
        if (v) {
            slot[w] = 0u;
            uint32_t lo = v & 0xFFFFu, hi = v >> 16;
            if (lo) atomicAdd(counts_row + 2 * w, lo);
            if (hi) atomicAdd(counts_row + 2 * w + 1, hi);
        }
    }
    __syncwarp();
}

// Registers: at most 64 a thread (four 256-thread blocks fill an SM's 64 K);
// single-instance 2-D FP32 walks fit in 56 without spills, which leaves 8 K
// registers of an SM for a 128-thread SVD cluster CTA (64 registers) beside
// four walk blocks when the SVD of one operator overlaps the walks of the
// next.  (Batched launches, which read their instance records from memory,
// would spill at 56.)
template <typename Real, int DIM, int KIND, bool MULTI>
__global__ void __maxnreg__((sizeof(Real) == 4 && DIM == 2 && !MULTI) ? 56 : 64)
walk_kernel(const __grid_constant__ WalkParams<Real> p)
{
    constexpr int G = Steps<Real, DIM>::G;
    constexpr unsigned FULL = 0xFFFFFFFFu;
    extern __shared__ uint32_t smem[];
    const WalkInst<Real> *__restrict__ insts = p.insts;
    auto inst = [&](int32_t q) -> const WalkInst<Real> & {
        return MULTI ? insts[q] : p.one;
    };

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    // warp-uniform tile / slot state
    int32_t tile_inst = 0, tile_i = 0;
    uint32_t tile_k = 0, tile_kend = 0;
    bool no_more = false;
    int32_t slot_cur = 0;
    uint32_t gen0 = 0, gen1 = 0;
    int32_t pt0 = -1, pt1 = -1, in0 = 0, in1 = 0;
    // shared memory: [exit queues of all warps][histogram slots of all warps]
    unsigned char *qbase = reinterpret_cast<unsigned char *>(smem) +
                           size_t(warp) * queue_bytes<Real, DIM>();
    Real *qx = reinterpret_cast<Real *>(qbase);                      // [DIM][kQueue]
    uint32_t *qi = reinterpret_cast<uint32_t *>(qx + DIM * kQueue);  // point
    uint32_t *qinst = qi + kQueue;                                   // instance
    uint32_t *qk = qinst + kQueue;                                   // walk k
    uint32_t *qsg = qk + kQueue;                                     // gen << 1 | slot
    uint32_t *qn_steps = qsg + kQueue;                               // N_eps
    uint32_t *hist = reinterpret_cast<uint32_t *>(
                         reinterpret_cast<unsigned char *>(smem) +
                         size_t(blockDim.x >> 5) * queue_bytes<Real, DIM>()) +
                     warp * (p.nslot > 0 ? p.nslot : 1) * p.hist_words;
    for (int32_t w = lane; w < p.nslot * p.hist_words; w += 32)
        hist[w] = 0u;
    int32_t qn = 0;  // queued exits (warp-uniform)
    __syncwarp();

    // classify and tally queue entries [q0, q0 + cnt) (cnt <= 32), one per lane
    auto drain = [&](int32_t q0, int32_t cnt) {
        if (lane < cnt) {
            int32_t e = q0 + lane;
            Real Xe[DIM];
#pragma unroll
            for (int a = 0; a < DIM; ++a)
                Xe[a] = qx[a * kQueue + e];
            const int32_t ei = int32_t(qi[e]);
            const WalkInst<Real> &I = inst(MULTI ? int32_t(qinst[e]) : 0);
            const uint32_t sg = qsg[e];
            const int32_t j = walk_classify<Real, DIM, KIND>(I.g, Xe);
            if (!MULTI && p.trace_elem) {
                size_t q = size_t(ei) * (I.k1 - I.k0) + (qk[e] - I.k0);
                p.trace_elem[q] = j;
                if (p.trace_steps) p.trace_steps[q] = qn_steps[e];
                if (p.trace_x) {
#pragma unroll
                    for (int a = 0; a < DIM; ++a)
                        p.trace_x[q * DIM + a] = double(Xe[a]);
                }
            }
            const uint32_t es = sg & 1u, eg = sg >> 1;
            const uint32_t g_now = es ? gen1 : gen0;
            if (p.nslot > 0 && eg == g_now)
                atomicAdd(hist + es * p.hist_words + (j >> 1), 1u << ((j & 1) * 16));
            else
                atomicAdd(I.counts + size_t(ei) * I.g.M_tot + j, 1u);
        }
        __syncwarp();
    };

    // lane state
    Real X[DIM];
    int32_t li = 0, linst = 0;
    uint32_t lk = 0, wlo = 0, whi = 0, nstep = 0;
    int32_t lslot = 0;
    uint32_t lgen = 0;
    bool active = false;
    unsigned long long my_steps = 0;
    uint32_t my_walks = 0, my_max = 0, my_unterm = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a)
        X[a] = Real(0);
    // warp-uniform state of the current tile: start point and walk-id base
    Real tile_x[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
        tile_x[a] = Real(0);
    uint64_t tile_wbase = 0;

    for (;;) {
        // ---- refill: lanes without a walk take the next walks of the warp's
        // tile; every lane runs the same select sequence (no divergence).
        unsigned need_mask = __ballot_sync(FULL, !active);
        if (need_mask != 0u &&
            (int32_t(__popc(need_mask)) >= p.refill_min || need_mask == FULL)) {
            while (need_mask != 0u && !no_more) {
                if (tile_k == tile_kend) {
                    unsigned long long t = 0;
                    if (lane == 0)
                        t = atomicAdd(p.work, 1ull);
                    t = __shfl_sync(FULL, t, 0);
                    if (t >= p.n_tiles) {
                        no_more = true;
                        break;
                    }
                    int32_t q = 0;
                    if (MULTI) {  // last instance whose first tile is <= t
                        int32_t lo = 0, hi = p.n_inst - 1;
                        while (lo < hi) {
                            int32_t mid = (lo + hi + 1) >> 1;
                            if (insts[mid].tile_begin <= t) lo = mid;
                            else hi = mid - 1;
                        }
                        q = lo;
                    }
                    const WalkInst<Real> &T = inst(q);
                    const uint64_t tl = t - T.tile_begin;
                    const uint32_t ti = uint32_t(tl / T.tiles_per_point);
                    const uint32_t tr = uint32_t(tl - uint64_t(ti) * T.tiles_per_point);
                    tile_inst = q;
                    tile_i = int32_t(ti);
                    tile_k = T.k0 + tr * T.tile_w;
                    tile_kend = min(tile_k + T.tile_w, T.k1);
                    tile_wbase = uint64_t(ti) * T.N;
#pragma unroll
                    for (int a = 0; a < DIM; ++a)
                        tile_x[a] = T.points_r ? T.points_r[size_t(ti) * DIM + a]
                                               : Real(T.points[size_t(ti) * DIM + a]);
                    if (KIND == kSphereOnly || KIND == kBoxOnly || KIND == kCubeOnly ||
                        KIND == kAnnulus) {
#pragma unroll
                        for (int a = 0; a < DIM; ++a)
                            tile_x[a] -= T.g.c[a];  // walk relative to the centre
                    }
                    if (KIND == kMapped) {  // the walk runs in y = S^{-1} x
                        Real y[DIM];
#pragma unroll
                        for (int a = 0; a < DIM; ++a) {
                            y[a] = Real(0);
#pragma unroll
                            for (int b = 0; b < DIM; ++b)
                                y[a] = fma(T.g.mSinv[a * DIM + b], tile_x[b], y[a]);
                        }
#pragma unroll
                        for (int a = 0; a < DIM; ++a)
                            tile_x[a] = y[a];
                    }
                    if (p.nslot > 0) {
                        int32_t s = (p.nslot == 2) ? (slot_cur ^ 1) : 0;
                        int32_t old_pt = s ? pt1 : pt0;
                        if (old_pt >= 0) {
                            const WalkInst<Real> &O = inst(s ? in1 : in0);
                            flush_slot(hist + s * p.hist_words, p.hist_words,
                                       O.counts + size_t(old_pt) * O.g.M_tot, lane);
                        }
                        if (s) { ++gen1; pt1 = tile_i; in1 = tile_inst; }
                        else { ++gen0; pt0 = tile_i; in0 = tile_inst; }
                        slot_cur = s;
                    }
                    continue;
                }
                const uint32_t avail = tile_kend - tile_k;
                const uint32_t rank = __popc(need_mask & lt_mask);
                const uint32_t n = __popc(need_mask);
                const uint32_t take = n < avail ? n : avail;
                const bool got = ((need_mask >> lane) & 1u) && rank < take;
                const uint32_t k = tile_k + rank;
                const uint64_t wid = tile_wbase + k;
#pragma unroll
                for (int a = 0; a < DIM; ++a)
                    X[a] = got ? tile_x[a] : X[a];
                wlo = got ? uint32_t(wid) : wlo;
                whi = got ? uint32_t(wid >> 32) : whi;
                lk = got ? k : lk;
                li = got ? tile_i : li;
                if (MULTI)
                    linst = got ? tile_inst : linst;
                nstep = got ? 0u : nstep;
                lslot = got ? slot_cur : lslot;
                lgen = got ? (slot_cur ? gen1 : gen0) : lgen;
                active = active || got;
                tile_k += take;
                need_mask &= ~__ballot_sync(FULL, got);
            }
        }
        if (!__any_sync(FULL, active))
            break;

        // ---- one group of G steps of the chain (Eq. (wos chain)) -----------
        // Branch-free: every lane evaluates every step (a lane without a walk
        // computes values nobody reads) and a stopped walk keeps X.  The cap
        // test runs per group: per step only within G steps of the cap.
        bool stop = false, capped = false;
        {
            const WalkInst<Real> &I = inst(linst);
            const uint32_t nb = uint32_t(p.group_blocks);
            const uint32_t blk0 = nstep / G;  // a group starts on a block boundary
            uint32_t w[4];
            if (!active || nstep + uint32_t(G) * nb <= I.step_cap) {
                // No stop flag: a walk that reached the eps-shell moves by
                // 0 * S U, keeps X bit for bit (up to the sign of a zero),
                // so every later distance repeats the same r <= eps and the
                // walk stays put; the last step's test says whether it stopped.
                bool go = true;
#pragma unroll 1
                for (uint32_t b = 0; b < nb; ++b) {
                    philox4x32_10(blk0 + b, wlo, whi, I.stream_id, p.rk, w);
#pragma unroll
                    for (int s = 0; s < G; ++s) {
                        const Real r = walk_dist<Real, DIM, KIND>(I.g, X);
                        go = !(r <= I.eps);
                        Real U[DIM];
                        step_direction<Real, DIM>(w, s, U);
                        step_move<Real, DIM>(I.S, U, go ? r : Real(0), X);
                        nstep += go ? 1u : 0u;
                    }
                }
                stop = !go;
            } else {
#pragma unroll 1
                for (uint32_t b = 0; b < nb; ++b) {
                    philox4x32_10(blk0 + b, wlo, whi, I.stream_id, p.rk, w);
#pragma unroll
                    for (int s = 0; s < G; ++s) {
                        const Real r = walk_dist<Real, DIM, KIND>(I.g, X);
                        const bool at_eps = r <= I.eps;
                        const bool at_cap = nstep >= I.step_cap;
                        const bool go = !stop && !at_eps && !at_cap;
                        capped = capped || (!stop && !at_eps && at_cap);
                        stop = stop || !go;
                        Real U[DIM];
                        step_direction<Real, DIM>(w, s, U);
                        step_move<Real, DIM>(I.S, U, go ? r : Real(0), X);
                        nstep += go ? 1u : 0u;
                    }
                }
            }
        }
        const bool fin = active && stop;
        const unsigned fin_mask = __ballot_sync(FULL, fin);
        if (fin_mask == 0u)
            continue;
        if ((KIND == kSphereOnly || KIND == kBoxOnly || KIND == kCubeOnly ||
             KIND == kAnnulus) && fin) {
            const WalkInst<Real> &I = inst(linst);
#pragma unroll
            for (int a = 0; a < DIM; ++a)
                X[a] += I.g.c[a];  // exit point back in x
        }
        if (KIND == kMapped && fin) {  // exit point back in x = S y
            const WalkInst<Real> &I = inst(linst);
            Real xo[DIM];
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                xo[a] = Real(0);
#pragma unroll
                for (int b = 0; b < DIM; ++b)
                    xo[a] = fma(I.g.mS[a * DIM + b], X[b], xo[a]);
            }
#pragma unroll
            for (int a = 0; a < DIM; ++a)
                X[a] = xo[a];
        }

        // ---- queue the finished walks; tally 32 at a time (Eq. (WoE_matrix_MC))
        const unsigned cap_mask = __ballot_sync(FULL, fin && capped);
        if (cap_mask != 0u && fin && capped) {  // walk left unterminated at the cap
            const WalkInst<Real> &I = inst(linst);
            ++my_unterm;
            if (I.unterm)
                atomicAdd(I.unterm + li, 1u);
            if (!MULTI && p.trace_elem) {
                size_t q = size_t(li) * (I.k1 - I.k0) + (lk - I.k0);
                p.trace_elem[q] = -1;
                if (p.trace_steps) p.trace_steps[q] = nstep;
                if (p.trace_x) {
#pragma unroll
                    for (int a = 0; a < DIM; ++a)
                        p.trace_x[q * DIM + a] = double(X[a]);
                }
            }
        }
        const unsigned push_mask = fin_mask & ~cap_mask;
        if ((push_mask >> lane) & 1u) {
            const int32_t e = qn + int32_t(__popc(push_mask & lt_mask));
#pragma unroll
            for (int a = 0; a < DIM; ++a)
                qx[a * kQueue + e] = X[a];
            qi[e] = uint32_t(li);
            if (MULTI)
                qinst[e] = uint32_t(linst);
            qsg[e] = (lgen << 1) | uint32_t(lslot);
            if (!MULTI && p.trace_elem) {
                qk[e] = lk;
                qn_steps[e] = nstep;
            }
        }
        qn += int32_t(__popc(push_mask));
        my_steps += fin ? nstep : 0u;
        my_walks += fin ? 1u : 0u;
        my_max = (fin && nstep > my_max) ? nstep : my_max;
        active = active && !fin;
        __syncwarp();
        if (qn >= 32) {
            drain(qn - 32, 32);
            qn -= 32;
        }
    }

    // ---- retire: drain the queue, flush the slots, add the statistics -------
    if (qn > 0)
        drain(0, qn);
    if (p.nslot > 0) {
        if (pt0 >= 0) {
            const WalkInst<Real> &O = inst(in0);
            flush_slot(hist, p.hist_words, O.counts + size_t(pt0) * O.g.M_tot, lane);
        }
        if (p.nslot == 2 && pt1 >= 0) {
            const WalkInst<Real> &O = inst(in1);
            flush_slot(hist + p.hist_words, p.hist_words,
                       O.counts + size_t(pt1) * O.g.M_tot, lane);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        my_steps += __shfl_xor_sync(FULL, my_steps, off);
        my_walks += __shfl_xor_sync(FULL, my_walks, off);
        my_unterm += __shfl_xor_sync(FULL, my_unterm, off);
        uint32_t o = __shfl_xor_sync(FULL, my_max, off);
        my_max = o > my_max ? o : my_max;
    }
    if (lane == 0) {
        atomicAdd(p.work + 1, my_steps);
        atomicAdd(p.work + 2, (unsigned long long)my_walks);
        if (my_unterm) atomicAdd(p.work + 3, (unsigned long long)my_unterm);
        atomicMax(p.work + 4, (unsigned long long)my_max);
    }
}

}  // namespace wos
