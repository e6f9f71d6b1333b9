// wos_svd.cu -- FP64 one-sided Jacobi SVD of the scaled operator and the
// r-TSVD reconstruction (paper Sec. 2, Eq. (SVD), (u1r); Sec. 4.3,
// Eq. (A_r_MC), (u_omega_M1_r_MC A); Sec. 5.1, Eq. (tsvd solution
// simulations)).
//
// B = diag(nu) (C[:, Gamma_1] / N) diag(sigma_{Gamma_1})^{-1/2} is formed in
// FP64, oriented so that the worked matrix W has m >= n columns-of-length-m,
// and its columns are orthogonalised by one-sided (Hestenes) Jacobi rotations
// in the parallel round-robin order: each round pairs the n columns into n/2
// disjoint pairs, one CTA per pair; n - 1 rounds make a sweep that touches
// every pair once.  Rounds are ordered by per-column version flags, sweeps by
// a grid barrier of a cooperative launch (every wait is bounded and reports
// WOS_DEVICE_TIMEOUT).  A pair is
// rotated when |w_p . w_q| > tol sqrt(|w_p|^2 |w_q|^2), tol = 1e-15, the
// relative test of Demmel & Veselic (1992); the build stops after a sweep
// without rotations.  FP64 is used for everything here: the operator is
// severely ill-conditioned (its singular values decay exponentially).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "wos.h"
#include "wos_internal.h"

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr double kTol = 1e-15;
// A sweep whose pairs all had |cos| = |w_p . w_q| / (|w_p| |w_q|) <= kLast
// rotated by angles that small; the cyclic sweep's quadratic convergence
// leaves every cosine at O(kLast^2) ~ 1e-15 after it, at kTol, so no
// verifying sweep follows it (what it would still rotate changes the
// singular values by O(cos^2), far below FP64 rounding).
constexpr double kLast = 3e-8;
constexpr int kMaxSweeps = 80;
constexpr int kPairThreads = 128;
static_assert(kPairThreads == 128, "the partial sums below assume four warps");

struct SvdWork {
    double *W;        // m x n, column-major (column j contiguous)
    double *Vw;       // n x n, column-major
    int m, n;         // worked orientation, m >= n
    int n_pad;        // n rounded up to even (a dummy column when odd)
    unsigned *bar;    // [0] arrive count, [1] generation, [2..4] rotation
                      // counters of sweeps mod 3, [5] status, [6] sweeps,
                      // [8..13] per sweep mod 3 (uint64): 1 if a rotated pair
                      // had cos^2 > kLast^2
    unsigned *ver;    // n_pad column versions (rounds finished per column)
    double *nrm;      // n squared column norms (kernels without V only)
    double *dsc, *dinv; // n column scales d_j and 1 / d_j (kernels without V:
                        // the column is d_j times the stored one)
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(FULL, v, o);
    return __shfl_sync(FULL, v, 0);  // one value for every lane
}

// Grid barrier for a cooperative launch; bounded wait (about 2 s) that
// records WOS_DEVICE_TIMEOUT in bar[5] instead of hanging.
__device__ bool grid_barrier(unsigned *bar, unsigned nblocks)
{
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *gen = bar + 1;
        unsigned g = *gen;
        __threadfence();
        unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long t0 = clock64();
            while (*gen == g) {
                __nanosleep(32);
                if (clock64() - t0 > 4000000000LL) {
                    atomicExch(bar + 5, unsigned(WOS_DEVICE_TIMEOUT));
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        if (*(volatile unsigned *)(bar + 5) != 0u)
            ok = 0;
    }
    __syncthreads();
    return ok != 0;
}

// Column index of round-robin position `pos` in round `r` (circle method:
// position 0 fixed, the other n_pad - 1 positions rotate).
__device__ __forceinline__ int rr_player(int pos, int r, int n_pad)
{
    if (pos == 0)
        return 0;
    return 1 + (pos - 1 + r) % (n_pad - 1);
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *a)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(unsigned *a, unsigned v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

// Wait (bounded, about 2 s) until column version ver[c] >= want.
__device__ bool wait_version(const unsigned *ver, int c, unsigned want, unsigned *status)
{
    if (ld_acquire(ver + c) >= want)
        return true;
    long long t0 = clock64();
    for (unsigned it = 1;; ++it) {
        if (ld_acquire(ver + c) >= want)
            return true;
        if ((it & 63u) == 0u) {
            if (clock64() - t0 > 4000000000LL) {
                atomicExch(status, unsigned(WOS_DEVICE_TIMEOUT));
                return false;
            }
            if (*(volatile unsigned *)status != 0u)
                return false;
        }
    }
}

// Sums of (a, b, g) over the 32 lanes of a warp with six additions per lane
// (instead of fifteen for three butterflies): the first two exchange steps
// split the values between lane halves and quarters, the last three are a
// butterfly on one value.  On return lanes 0-7 hold sum(a), lanes 8-15
// sum(b), lanes 16-23 sum(g).
__device__ __forceinline__ double warp_sum3(double a, double b, double g, int lane)
{
    const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
    double k0 = hi16 ? g : a, k1 = hi16 ? 0.0 : b;
    k0 += __shfl_xor_sync(FULL, hi16 ? a : g, 16);
    k1 += __shfl_xor_sync(FULL, hi16 ? b : 0.0, 16);
    double k = hi8 ? k1 : k0;
    k += __shfl_xor_sync(FULL, hi8 ? k0 : k1, 8);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1)
        k += __shfl_xor_sync(FULL, k, o);
    return k;
}

// Rotation (c, s) that makes the pair orthogonal, from the Gram entries
// al = |x|^2, be = |y|^2, ga = x.y (Hestenes; Rutishauser's smaller angle):
// with h = (be - al) / 2 and r = sqrt(h^2 + ga^2), cos(2 theta) = |h| / r, so
// c^2 = (1 + |h| / r) / 2 and s = sign(h) ga / (2 r c).  Two reciprocal
// square roots and no division: the dependent FP64 chain is the critical
// path of a round.
__device__ __forceinline__ void jacobi_rotation(double al, double be, double ga, double &c,
                                                double &s)
{
    const double h = 0.5 * (be - al);
    const double y = rsqrt(fma(h, h, ga * ga));  // 1 / r
    const double c2 = fma(fabs(h) * y, 0.5, 0.5);
    const double gy = copysign(0.5, h) * ga * y;
    const double z = rsqrt(c2);                  // 1 / c
    c = c2 * z;
    s = gy * z;
}


// Jacobi without the accumulated V, for the large problems (worked matrices
// of more than 256 columns, where the FP64 work of the sweeps bounds the
// factorisation): the right singular vectors of W come from X's final
// columns and the left ones from W itself afterwards (L = W P X_final), so a
// pair reads and rotates only its two columns of X.  Its Gram entries take
// one dot product instead of three: the squared norms are kept per column in
// nrm[] and carried through each rotation by the identities of a rotation
// that makes the pair orthogonal, |x_p'|^2 = |x_p|^2 - t g and |x_q'|^2 =
// |x_q|^2 + t g (g = x_p . x_q, t = s / c); a norm whose identity cancelled
// more than 63/64 of its terms is recomputed from the rotated column in the
// same pass (the final singular values are recomputed exactly anyway).
//
// A CTA of four warps takes four pairs of a round, a warp per pair with the
// pair's two columns in its registers (RPL rows a lane, the rest streamed),
// and one warp forms the four rotations at once (lane k for pair k): an FP64
// warp instruction holds its sub-partition's FP64 unit for 64 cycles
// whatever its active lanes, so the scalar chain of a rotation is shared by
// four pairs, and a pair's reduction is one warp's.  Rounds, flags, stopping
// rule and the order of the pairs are those of jacobi_body.
//
// Both kernels without V (this one and jacobi_lean_body) add a pair's dot
// product, and a recomputed norm, in one canonical order, so that a problem
// gets the same bits from either (alone or in a batch): lane l of the
// pair's warp(s) owns rows l + 32 k, k < RPL; four chains c = k mod 4 (the
// rows past 32 RPL on chain 0), the lane's value (g0 + g1) + (g2 + g3), then
// the butterfly of warp_sum over the 32 lanes.
constexpr double kRecompute = 1.0 / 64.0;
constexpr int kGroupPairs = 4;             // pairs (warps) per CTA

// Scaled rotations (the square-root-free form of plane rotations, after
// Gentleman, and Anda & Park's dynamic scaling): column j is stored as xt_j
// with x_j = d_j xt_j.  The rotation (c, s) of the pair, t = s / c, becomes
//     xt_p' = xt_p - tau_p xt_q,  tau_p = t d_q / d_p,   d_p' = c d_p,
//     xt_q' = xt_q + tau_q xt_p,  tau_q = t d_p / d_q,   d_q' = c d_q,
// one FMA per row and column instead of a product and an FMA; the scales
// only shrink (c <= 1), so a column whose scale falls below 2^-80 has it
// folded into the stored values in the same pass (d = 1 again).  Its Gram
// entries: x_p . x_q = d_p d_q (xt_p . xt_q); the squared norms of x are
// carried as before.  Every kernel without V calls this on one lane per
// pair and applies the result in the same arithmetic, so they form the same
// bits.  f: 1 rotate, 2 / 4 recompute the norm of p / q, 8 / 16 fold the
// scale of p / q (multiply the new values by mp / mq).
struct ScaledRot {
    double tp, tq;   // tau_p, tau_q
    double mp, mq;   // fold multipliers (the new scales)
    double sp, sq;   // factor of a recomputed stored norm: d'^2, or 1 after a fold
    int f;
};

constexpr double kFoldBelow = 8.271806125530277e-25;  // 2^-80

// A pair's carried quantities: squared norms, scales and inverse scales of
// columns p and q (read at the start of a round, off the rotation's path).
struct PairState {
    double al, be, dp, dq, ep, eq;
};

__device__ __forceinline__ PairState load_pair_state(const SvdWork &w, int p, int q)
{
    PairState s;
    s.al = __ldcg(w.nrm + p);
    s.be = __ldcg(w.nrm + q);
    s.dp = __ldcg(w.dsc + p);
    s.dq = __ldcg(w.dsc + q);
    s.ep = __ldcg(w.dinv + p);
    s.eq = __ldcg(w.dinv + q);
    return s;
}

__device__ __forceinline__ ScaledRot scaled_rotation(const SvdWork &w, int p, int q,
                                                     const PairState &ps, double gh, bool *big)
{
    ScaledRot r = {0.0, 0.0, 1.0, 1.0, 1.0, 1.0, 0};
    const double al = ps.al, be = ps.be, dp = ps.dp, dq = ps.dq, ep = ps.ep, eq = ps.eq;
    const double g = gh * dp * dq;
    const double ab = al * be, g2 = g * g;
    if (!(al != 0.0 && be != 0.0 && g2 > (kTol * kTol) * ab))
        return r;
    // the rotation of jacobi_rotation, with z = 1 / c and t = s / c
    const double h = 0.5 * (be - al);
    const double y = rsqrt(fma(h, h, g * g));
    const double c2 = fma(fabs(h) * y, 0.5, 0.5);
    const double gy = copysign(0.5, h) * g * y;
    const double z = rsqrt(c2);
    const double c = c2 * z, t = gy * z * z;
    *big = *big || g2 > (kLast * kLast) * ab;
    r.f = 1;
    r.tp = t * dq * ep;
    r.tq = t * dp * eq;
    double ndp = c * dp, ndq = c * dq, nep = z * ep, neq = z * eq;
    if (ndp < kFoldBelow) {
        r.f |= 8;
        r.mp = ndp;
        ndp = 1.0;
        nep = 1.0;
    }
    if (ndq < kFoldBelow) {
        r.f |= 16;
        r.mq = ndq;
        ndq = 1.0;
        neq = 1.0;
    }
    w.dsc[p] = ndp;
    w.dinv[p] = nep;
    w.dsc[q] = ndq;
    w.dinv[q] = neq;
    r.sp = ndp * ndp;
    r.sq = ndq * ndq;
    const double tg = t * g;
    const double an = al - tg, bn = be + tg;
    const double scale = al + be + fabs(tg);
    if (!(an > kRecompute * scale))
        r.f |= 2;
    else
        w.nrm[p] = an;
    if (!(bn > kRecompute * scale))
        r.f |= 4;
    else
        w.nrm[q] = bn;
    return r;
}

// The rotated stored values of a row (x, y) under r.
__device__ __forceinline__ void scaled_update(const ScaledRot &r, double x, double y, double &xn,
                                              double &yn)
{
    xn = fma(-r.tp, y, x);
    yn = fma(r.tq, x, y);
    if (r.f & 8)
        xn *= r.mp;
    if (r.f & 16)
        yn *= r.mq;
}
constexpr int kGroupThreads = 32 * kGroupPairs;

template <int RPL>
__device__ void jacobi_group_body(const SvdWork &w, const int bid, const int nblk)
{
    __shared__ double gk[kGroupPairs];       // xt_p . xt_q of each pair
    __shared__ ScaledRot prm[kGroupPairs];   // each pair's scaled rotation
    __shared__ int s_rot, s_big;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int half = w.n_pad / 2;
    const int groups = (half + kGroupPairs - 1) / kGroupPairs;
    const int m = w.m, n = w.n;
    unsigned *status = w.bar + 5;
    unsigned long long *maxcos = reinterpret_cast<unsigned long long *>(w.bar + 8);
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        unsigned *rot = w.bar + 2 + (sweep % 3);
        if (bid == 0 && tid == 0) {
            w.bar[2 + ((sweep + 1) % 3)] = 0u;
            maxcos[(sweep + 1) % 3] = 0ull;
        }
        if (tid == 0) {
            s_rot = 0;
            s_big = 0;
        }
        bool my_big = false;
        int my_rot = 0;
        for (int r = 0; r < w.n_pad - 1; ++r) {
            const unsigned R = unsigned(sweep) * unsigned(w.n_pad - 1) + unsigned(r);
            for (int gi = bid; gi < groups; gi += nblk) {
                const int pr = gi * kGroupPairs + wid;  // this warp's pair
                int p = n, q = n;                       // none past the last pair
                if (pr < half) {
                    const int a = rr_player(pr, r, w.n_pad);
                    const int b = rr_player(w.n_pad - 1 - pr, r, w.n_pad);
                    p = min(a, b);
                    q = max(a, b);
                }
                const bool live = pr < half && q < n;   // a real pair (not the dummy)
                bool ok = true;
                if (pr < half && lane == 0)
                    ok = wait_version(w.ver, p, R, status);
                else if (live && lane == 1)
                    ok = wait_version(w.ver, q, R, status);
                if (!__syncthreads_and(ok))
                    return;
                // lane k of warp 0 reads pair k's carried state now (its
                // rotation needs it after the dot products)
                PairState ps = {0.0, 0.0, 1.0, 1.0, 1.0, 1.0};
                int pk = n, qk = n;
                if (wid == 0 && lane < kGroupPairs) {
                    const int prk = gi * kGroupPairs + lane;
                    if (prk < half) {
                        const int a = rr_player(prk, r, w.n_pad);
                        const int b = rr_player(w.n_pad - 1 - prk, r, w.n_pad);
                        pk = min(a, b);
                        qk = max(a, b);
                        if (qk < n)
                            ps = load_pair_state(w, pk, qk);
                    }
                }
                double xr[RPL], yr[RPL];
                double *wp = w.W + size_t(live ? p : 0) * m, *wq = w.W + size_t(live ? q : 0) * m;
                double g0 = 0.0, g1 = 0.0, g2 = 0.0, g3 = 0.0;
                if (live) {
#pragma unroll
                    for (int k = 0; k < RPL; ++k) {
                        const int i = lane + 32 * k;
                        xr[k] = i < m ? __ldcg(wp + i) : 0.0;
                        yr[k] = i < m ? __ldcg(wq + i) : 0.0;
                    }
#pragma unroll
                    for (int k = 0; k < RPL; k += 4) {  // four chains: DFMA latency
                        g0 = fma(xr[k], yr[k], g0);
                        g1 = fma(xr[k + 1], yr[k + 1], g1);
                        g2 = fma(xr[k + 2], yr[k + 2], g2);
                        g3 = fma(xr[k + 3], yr[k + 3], g3);
                    }
                    for (int i = lane + 32 * RPL; i < m; i += 32)
                        g0 = fma(__ldcg(wp + i), __ldcg(wq + i), g0);
                    const double g = warp_sum((g0 + g1) + (g2 + g3));
                    if (lane == 0)
                        gk[wid] = g;
                }
                __syncthreads();
                // warp 0 forms the rotations of the CTA's pairs, lane k for pair k
                if (wid == 0 && lane < kGroupPairs) {
                    ScaledRot sr = {0.0, 0.0, 1.0, 1.0, 1.0, 1.0, 0};
                    if (qk < n) {
                        sr = scaled_rotation(w, pk, qk, ps, gk[lane], &my_big);
                        my_rot += sr.f & 1;
                    }
                    prm[lane] = sr;
                }
                __syncthreads();
                const ScaledRot sr = prm[wid];
                const int f = sr.f;
                if (live && f == 1) {
                    // the common case: two FMAs a row, no predicated FP64
                    // work (a warp FP64 instruction holds the unit for 64
                    // cycles even with its lanes predicated off)
#pragma unroll
                    for (int k = 0; k < RPL; ++k) {
                        const int i = lane + 32 * k;
                        const double x = fma(-sr.tp, yr[k], xr[k]);
                        const double y = fma(sr.tq, xr[k], yr[k]);
                        if (i < m) {
                            __stcg(wp + i, x);
                            __stcg(wq + i, y);
                        }
                    }
                    for (int i = lane + 32 * RPL; i < m; i += 32) {
                        const double x0 = __ldcg(wp + i), y0 = __ldcg(wq + i);
                        __stcg(wp + i, fma(-sr.tp, y0, x0));
                        __stcg(wq + i, fma(sr.tq, x0, y0));
                    }
                } else if (live && (f & 1)) {
                    double np2[4] = {0.0, 0.0, 0.0, 0.0}, nq2[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
                    for (int k = 0; k < RPL; ++k) {
                        const int i = lane + 32 * k;
                        double x, y;
                        scaled_update(sr, xr[k], yr[k], x, y);
                        if (i < m) {
                            __stcg(wp + i, x);
                            __stcg(wq + i, y);
                            if (f & 2)
                                np2[k & 3] = fma(x, x, np2[k & 3]);
                            if (f & 4)
                                nq2[k & 3] = fma(y, y, nq2[k & 3]);
                        }
                    }
                    for (int i = lane + 32 * RPL; i < m; i += 32) {
                        double x, y;
                        scaled_update(sr, __ldcg(wp + i), __ldcg(wq + i), x, y);
                        __stcg(wp + i, x);
                        __stcg(wq + i, y);
                        if (f & 2)
                            np2[0] = fma(x, x, np2[0]);
                        if (f & 4)
                            nq2[0] = fma(y, y, nq2[0]);
                    }
                    if (f & 2) {  // warp-uniform
                        const double t = warp_sum((np2[0] + np2[1]) + (np2[2] + np2[3]));
                        if (lane == 0)
                            w.nrm[p] = t * sr.sp;
                    }
                    if (f & 4) {
                        const double t = warp_sum((nq2[0] + nq2[1]) + (nq2[2] + nq2[3]));
                        if (lane == 0)
                            w.nrm[q] = t * sr.sq;
                    }
                }
                __syncthreads();
                if (tid == 0) {
                    // the CTA's stores are ordered before the flags by the
                    // barrier above and this fence (a release pattern)
                    __threadfence();
                    for (int k = 0; k < kGroupPairs; ++k) {
                        const int prk = gi * kGroupPairs + k;
                        if (prk >= half)
                            break;
                        const int a = rr_player(prk, r, w.n_pad);
                        const int b = rr_player(w.n_pad - 1 - prk, r, w.n_pad);
                        st_relaxed(w.ver + min(a, b), R + 1u);
                        if (max(a, b) < n)
                            st_relaxed(w.ver + max(a, b), R + 1u);
                    }
                }
            }
        }
        if (wid == 0 && lane < kGroupPairs) {
            if (my_rot)
                atomicAdd(&s_rot, my_rot);
            if (my_big)
                atomicOr(&s_big, 1);
        }
        __syncthreads();
        if (tid == 0) {
            if (s_rot)
                atomicAdd(rot, unsigned(s_rot));
            if (s_big)
                atomicMax(maxcos + (sweep % 3), 1ull);
        }
        if (!grid_barrier(w.bar, unsigned(nblk)))
            return;
        const unsigned long long big = *(volatile unsigned long long *)(maxcos + (sweep % 3));
        bool done = *(volatile unsigned *)rot == 0u || big == 0ull;
        if (bid == 0 && tid == 0)
            w.bar[6] = unsigned(sweep + 1);
        if (done)
            return;
    }
    if (bid == 0 && tid == 0)
        atomicExch(w.bar + 5, unsigned(WOS_NO_CONVERGENCE));
}

// The same sweeps with a CTA of kPairThreads threads per pair: the shorter
// critical path of a round when the batch has too few pairs to fill the GPU
// (a lone problem), where the grouped kernel's one-warp pairs would leave
// FP64 units idle.  Warp w, lane l holds the rows l + 32 k with k = w mod 4
// of the canonical order (chain w of the grouped kernel's lane l; warp 0 also
// the rows past 32 RPL), and warp 0 combines the four chains of each lane
// as that kernel does, so the two give the same bits.
template <int RPL>
__device__ void jacobi_lean_body(const SvdWork &w, const int bid, const int nblk)
{
    constexpr int J = RPL / 4;  // rows a thread
    static_assert(kPairThreads == 128, "four warps: the four chains of the canonical order");
    __shared__ double part[4][32];
    __shared__ ScaledRot prm;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int half = w.n_pad / 2;
    const int m = w.m, n = w.n;
    unsigned *status = w.bar + 5;
    unsigned long long *maxcos = reinterpret_cast<unsigned long long *>(w.bar + 8);
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        unsigned *rot = w.bar + 2 + (sweep % 3);
        if (bid == 0 && tid == 0) {
            w.bar[2 + ((sweep + 1) % 3)] = 0u;
            maxcos[(sweep + 1) % 3] = 0ull;
        }
        bool my_big = false;
        for (int r = 0; r < w.n_pad - 1; ++r) {
            const unsigned R = unsigned(sweep) * unsigned(w.n_pad - 1) + unsigned(r);
            for (int pr = bid; pr < half; pr += nblk) {
                int a = rr_player(pr, r, w.n_pad);
                int b = rr_player(w.n_pad - 1 - pr, r, w.n_pad);
                int p = min(a, b), q = max(a, b);
                bool ok = true;
                if (tid == 0)
                    ok = wait_version(w.ver, p, R, status);
                else if (tid == 32 && q < n)
                    ok = wait_version(w.ver, q, R, status);
                if (!__syncthreads_and(ok))
                    return;
                bool rotated = false;
                if (q < n) {
                    double *wp = w.W + size_t(p) * m, *wq = w.W + size_t(q) * m;
                    PairState ps = {0.0, 0.0, 1.0, 1.0, 1.0, 1.0};
                    if (tid == 0)
                        ps = load_pair_state(w, p, q);
                    double xr[J], yr[J];
                    double g = 0.0;
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        const int i = lane + 32 * (4 * j + wid);
                        xr[j] = i < m ? __ldcg(wp + i) : 0.0;
                        yr[j] = i < m ? __ldcg(wq + i) : 0.0;
                    }
#pragma unroll
                    for (int j = 0; j < J; ++j)
                        g = fma(xr[j], yr[j], g);
                    if (wid == 0)
                        for (int i = lane + 32 * RPL; i < m; i += 32)
                            g = fma(__ldcg(wp + i), __ldcg(wq + i), g);
                    part[wid][lane] = g;
                    __syncthreads();
                    if (wid == 0) {
                        g = warp_sum((part[0][lane] + part[1][lane]) +
                                     (part[2][lane] + part[3][lane]));
                        if (lane == 0)
                            prm = scaled_rotation(w, p, q, ps, g, &my_big);
                    }
                    __syncthreads();
                    const ScaledRot sr = prm;
                    const int f = sr.f;
                    if (f == 1) {  // the common case, as in the grouped kernel
                        rotated = true;
#pragma unroll
                        for (int j = 0; j < J; ++j) {
                            const int i = lane + 32 * (4 * j + wid);
                            const double x = fma(-sr.tp, yr[j], xr[j]);
                            const double y = fma(sr.tq, xr[j], yr[j]);
                            if (i < m) {
                                __stcg(wp + i, x);
                                __stcg(wq + i, y);
                            }
                        }
                        if (wid == 0)
                            for (int i = lane + 32 * RPL; i < m; i += 32) {
                                const double x0 = __ldcg(wp + i), y0 = __ldcg(wq + i);
                                __stcg(wp + i, fma(-sr.tp, y0, x0));
                                __stcg(wq + i, fma(sr.tq, x0, y0));
                            }
                    } else if (f & 1) {
                        rotated = true;
                        double np2 = 0.0, nq2 = 0.0;
#pragma unroll
                        for (int j = 0; j < J; ++j) {
                            const int i = lane + 32 * (4 * j + wid);
                            double x, y;
                            scaled_update(sr, xr[j], yr[j], x, y);
                            if (i < m) {
                                __stcg(wp + i, x);
                                __stcg(wq + i, y);
                                if (f & 2)
                                    np2 = fma(x, x, np2);
                                if (f & 4)
                                    nq2 = fma(y, y, nq2);
                            }
                        }
                        if (wid == 0)
                            for (int i = lane + 32 * RPL; i < m; i += 32) {
                                double x, y;
                                scaled_update(sr, __ldcg(wp + i), __ldcg(wq + i), x, y);
                                __stcg(wp + i, x);
                                __stcg(wq + i, y);
                                if (f & 2)
                                    np2 = fma(x, x, np2);
                                if (f & 4)
                                    nq2 = fma(y, y, nq2);
                            }
                        if (f & 6) {  // CTA-uniform: the flag is in shared memory
                            __shared__ double rp[2][4][32];
                            rp[0][wid][lane] = np2;
                            rp[1][wid][lane] = nq2;
                            __syncthreads();
                            if (wid == 0) {
                                if (f & 2) {
                                    const double t = warp_sum((rp[0][0][lane] + rp[0][1][lane]) +
                                                              (rp[0][2][lane] + rp[0][3][lane]));
                                    if (lane == 0)
                                        w.nrm[p] = t * sr.sp;
                                }
                                if (f & 4) {
                                    const double t = warp_sum((rp[1][0][lane] + rp[1][1][lane]) +
                                                              (rp[1][2][lane] + rp[1][3][lane]));
                                    if (lane == 0)
                                        w.nrm[q] = t * sr.sq;
                                }
                            }
                        }
                    }
                }
                __syncthreads();
                if (tid == 0) {
                    // the CTA's stores are ordered before the flags by the
                    // barrier above and this fence (a release pattern)
                    __threadfence();
                    st_relaxed(w.ver + p, R + 1u);
                    if (q < n)
                        st_relaxed(w.ver + q, R + 1u);
                    if (rotated)
                        atomicAdd(rot, 1u);
                }
            }
        }
        if (tid == 0 && my_big)
            atomicMax(maxcos + (sweep % 3), 1ull);
        if (!grid_barrier(w.bar, unsigned(nblk)))
            return;
        const unsigned long long big = *(volatile unsigned long long *)(maxcos + (sweep % 3));
        bool done = *(volatile unsigned *)rot == 0u || big == 0ull;
        if (bid == 0 && tid == 0)
            w.bar[6] = unsigned(sweep + 1);
        if (done)
            return;
    }
    if (bid == 0 && tid == 0)
        atomicExch(w.bar + 5, unsigned(WOS_NO_CONVERGENCE));
}

// One pair per CTA of kPairThreads threads; the m rows are split over the
// CTA (RPT rows per thread kept in registers, the rest streamed) so a pair
// uses a whole SM's FP64 pipe.  Rounds are ordered by column versions: ver[c]
// counts the rounds that have finished with column c, so the pair (p, q) of
// global round R starts once ver[p] >= R and ver[q] >= R (the previous
// round's writers of p and q are done; warps 0 and 1 wait for one each).
// Only one grid barrier per sweep remains, for the convergence test.  Columns
// are read and written through L2 (ld.cg / st.cg): other SMs update them
// between rounds; one fence orders a pair's stores before its two flags.
template <int RPT>
__device__ void jacobi_body(const SvdWork &w, const int bid, const int nblk)
{
    __shared__ double part[3][kPairThreads / 32];
    __shared__ double cs[2];
    __shared__ int flag;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int half = w.n_pad / 2;
    const int m = w.m, n = w.n;
    unsigned *status = w.bar + 5;
    unsigned long long *maxcos = reinterpret_cast<unsigned long long *>(w.bar + 8);
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        unsigned *rot = w.bar + 2 + (sweep % 3);
        if (bid == 0 && tid == 0) {
            w.bar[2 + ((sweep + 1) % 3)] = 0u;
            maxcos[(sweep + 1) % 3] = 0ull;
        }
        bool my_big = false;  // a rotated pair had cos^2 > kLast^2 (thread 0)
        for (int r = 0; r < w.n_pad - 1; ++r) {
            const unsigned R = unsigned(sweep) * unsigned(w.n_pad - 1) + unsigned(r);
            for (int pr = bid; pr < half; pr += nblk) {
                int a = rr_player(pr, r, w.n_pad);
                int b = rr_player(w.n_pad - 1 - pr, r, w.n_pad);
                int p = min(a, b), q = max(a, b);
                bool ok = true;
                if (tid == 0)
                    ok = wait_version(w.ver, p, R, status);
                else if (tid == 32 && q < n)
                    ok = wait_version(w.ver, q, R, status);
                if (!__syncthreads_and(ok))
                    return;
                bool rotated = false;
                if (q < n) {
                    double *wp = w.W + size_t(p) * m, *wq = w.W + size_t(q) * m;
                    double *vp = w.Vw + size_t(p) * n, *vq = w.Vw + size_t(q) * n;
                    double xr[RPT], yr[RPT], vx[RPT], vy[RPT];
                    double al = 0.0, be = 0.0, ga = 0.0;
#pragma unroll
                    for (int k = 0; k < RPT; ++k) {
                        int i = tid + k * kPairThreads;
                        xr[k] = i < m ? __ldcg(wp + i) : 0.0;
                        yr[k] = i < m ? __ldcg(wq + i) : 0.0;
                        vx[k] = i < n ? __ldcg(vp + i) : 0.0;
                        vy[k] = i < n ? __ldcg(vq + i) : 0.0;
                    }
#pragma unroll
                    for (int k = 0; k < RPT; ++k) {
                        if (tid + k * kPairThreads < m) {
                            al = fma(xr[k], xr[k], al);
                            be = fma(yr[k], yr[k], be);
                            ga = fma(xr[k], yr[k], ga);
                        }
                    }
                    for (int i = tid + RPT * kPairThreads; i < m; i += kPairThreads) {
                        double x = __ldcg(wp + i), y = __ldcg(wq + i);
                        al = fma(x, x, al);
                        be = fma(y, y, be);
                        ga = fma(x, y, ga);
                    }
                    const double red = warp_sum3(al, be, ga, lane);
                    if ((lane & 7) == 0 && lane < 24)
                        part[lane >> 3][wid] = red;
                    __syncthreads();
                    // one thread combines the partial sums and computes the
                    // rotation (FP64 is scarce on this part: 2 FMA/clk/SM)
                    if (tid == 0) {
                        al = (part[0][0] + part[0][1]) + (part[0][2] + part[0][3]);
                        be = (part[1][0] + part[1][1]) + (part[1][2] + part[1][3]);
                        ga = (part[2][0] + part[2][1]) + (part[2][2] + part[2][3]);
                        double c = 1.0, sn = 0.0;
                        int rot_flag = 0;
                        // rotate when |ga| > tol sqrt(al be), tested squared
                        const double ab = al * be, g2 = ga * ga;
                        if (al != 0.0 && be != 0.0 && g2 > (kTol * kTol) * ab) {
                            jacobi_rotation(al, be, ga, c, sn);
                            rot_flag = 1;
                            my_big = my_big || g2 > (kLast * kLast) * ab;  // no division
                        }
                        cs[0] = c;
                        cs[1] = sn;
                        flag = rot_flag;
                    }
                    __syncthreads();
                    if (flag) {
                        rotated = true;
                        const double c = cs[0], s = cs[1];
#pragma unroll
                        for (int k = 0; k < RPT; ++k) {
                            int i = tid + k * kPairThreads;
                            if (i < m) {
                                __stcg(wp + i, c * xr[k] - s * yr[k]);
                                __stcg(wq + i, s * xr[k] + c * yr[k]);
                            }
                            if (i < n) {
                                __stcg(vp + i, c * vx[k] - s * vy[k]);
                                __stcg(vq + i, s * vx[k] + c * vy[k]);
                            }
                        }
                        for (int i = tid + RPT * kPairThreads; i < m; i += kPairThreads) {
                            double x = __ldcg(wp + i), y = __ldcg(wq + i);
                            __stcg(wp + i, c * x - s * y);
                            __stcg(wq + i, s * x + c * y);
                        }
                        for (int i = tid + RPT * kPairThreads; i < n; i += kPairThreads) {
                            double x = __ldcg(vp + i), y = __ldcg(vq + i);
                            __stcg(vp + i, c * x - s * y);
                            __stcg(vq + i, s * x + c * y);
                        }
                    }
                }
                __syncthreads();
                if (tid == 0) {
                    // the CTA's stores are ordered before the flags by the
                    // barrier above and this fence (a fence followed by
                    // relaxed stores is a release pattern)
                    __threadfence();
                    st_relaxed(w.ver + p, R + 1u);
                    if (q < n)
                        st_relaxed(w.ver + q, R + 1u);
                    if (rotated)
                        atomicAdd(rot, 1u);
                }
            }
        }
        if (tid == 0 && my_big)
            atomicMax(maxcos + (sweep % 3), 1ull);
        if (!grid_barrier(w.bar, unsigned(nblk)))
            return;
        const unsigned long long big = *(volatile unsigned long long *)(maxcos + (sweep % 3));
        bool done = *(volatile unsigned *)rot == 0u || big == 0ull;
        if (bid == 0 && tid == 0)
            w.bar[6] = unsigned(sweep + 1);
        if (done)
            return;
    }
    if (bid == 0 && tid == 0)
        atomicExch(w.bar + 5, unsigned(WOS_NO_CONVERGENCE));
}

// ---------------------------------------------------------------------------
// FP32 preconditioning of the sweeps without V.  FP64 is scarce on this part
// (an FP64 warp instruction holds its sub-partition's unit for 64 cycles, 2
// FMA/clk/SM against 128 in FP32), and the FP64 sweeps on X = R^T are the
// bulk of a large factorisation.  So sweeps first run on an FP32 copy of X,
// which only steers the angles; the product J of their rotations, made
// orthogonal to FP64 rounding by two Newton-Schulz steps (Q = J (3 I -
// J^T J) / 2, whose error is quadratic in that of J; Higham, "Functions of
// Matrices", Sec. 8.3), gives the FP64 sweeps' start X Q: the same singular
// values and left vectors as X (Q is orthogonal), with columns already
// orthogonal to about FP32 precision, so quadratic convergence sets in at
// once and a few FP64 sweeps remain (the mixed-precision preconditioned
// one-sided Jacobi SVD of Higham, Tisseur, Webb & Zhang, with the
// low-precision factor taken from Jacobi itself).  The results keep the FP64
// sweeps' accuracy.
//
// The FP32 sweeps run on C CTAs per problem (C about n / 24, at most 32),
// X in their shared memory: block-cyclic one-sided Jacobi (the columns in
// 2C blocks of b, two per CTA; the blocks meet in the round-robin order,
// every pair of columns once a sweep: the pairs inside each block in the
// sweep's first block round, then those across the two blocks), a warp per
// pair, the sub-rounds of a block round separated by CTA barriers only and
// the block rounds by a grid barrier of the problem's CTAs (the blocks move
// through L2).  Across the blocks, warp w keeps column w of its CTA's first
// block in registers and meets the second block's columns in turn, which
// pass from warp to warp through shared memory.  Each CTA also forms the
// 2b x 2b product G of a block round's rotations of its 2b columns; J is
// rebuilt from those afterwards by pc32_replay_kernel (J <- J G for each
// block round in order, rows of J independent), so the sweeps carry no V.
constexpr float kTol32 = 1e-6f;   // rotate when |cos| > kTol32 (FP32 dots)
constexpr float kLast32 = 1e-3f;  // stop after a sweep with every |cos| <= this
constexpr int kMaxSweeps32 = 16;  // then stop anyway (preconditioning only)
constexpr int kPc32MaxCtas = 32;  // CTAs per problem, at most
constexpr int kPc32MaxB = 16;     // widest block (warps of a CTA)
constexpr int kPc32Chunks = 6;    // float4 rows a lane holds: columns of <= 768 rows

struct Pc32Job {
    float *X;         // m x n, column-major (FP32 copy of X), rotated in place
    float *G;         // per sweep, block round and CTA: the 2b x 2b product of
                      // its rotations (column-major)
    unsigned *bar;    // [6] sweeps, [8..10] per sweep mod 3: a |cos| > kLast32
    double *J;        // n x n: the product of the rotations (replay)
    int m, n, b;      // b a multiple of 4, n <= 2 C b
    int C;            // CTAs (2C blocks)
    int ms;           // m rounded up to 128: the shared-memory column stride
};

// Error-free product (Dekker): a b = p + e.
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = a * b;
    e = fmaf(a, b, -p);
}

// cos and sin of the rotation with tangent t (|t| <= 1), each within about
// half an FP32 ulp: c = (1 + t^2)^{-1/2} from the FP32 reciprocal square
// root and one Newton step y (1 + (1 - u y^2) / 2), u = 1 + t^2 and the
// residual 1 - u y^2 formed in float-float, then rounded; s = t c.
__device__ __forceinline__ void accurate_cos_sin(float t, float &c, float &s)
{
    float p, pe;
    two_prod(t, t, p, pe);
    const float uh = 1.0f + p;             // |p| <= 1: fast two-sum
    const float ul = ((1.0f - uh) + p) + pe;
    const float y = rsqrtf(uh);
    float q, qe, w, we;
    two_prod(y, y, q, qe);
    two_prod(uh, q, w, we);
    const float res = (1.0f - w) - (we + fmaf(uh, qe, ul * q));  // 1 - u y^2
    c = fmaf(0.5f * y, res, y);
    s = t * c;
}

// Sums over the warp by xor butterflies: every lane gets the same sums.
__device__ __forceinline__ void warp_sum3f(float &a, float &b, float &g)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(FULL, a, o);
        b += __shfl_xor_sync(FULL, b, o);
        g += __shfl_xor_sync(FULL, g, o);
    }
}

// The rotation of a pair from al = |x|^2, be = |y|^2, ga = x.y: false when
// it is not rotated (|cos| <= kTol32, or a zero or non-finite norm); *big
// when |cos| > kLast32.  Rutishauser's smaller angle, t = sign(h) g /
// (|h| + sqrt(h^2 + g^2)), h = (be - al) / 2, scale-free.
__device__ __forceinline__ bool pc32_rotation(float al, float be, float ga, float &c, float &sn,
                                              bool &big)
{
    c = 1.0f;
    sn = 0.0f;
    big = false;
    if (!(al > 0.0f && be > 0.0f && al <= 3.0e38f && be <= 3.0e38f))
        return false;
    // the angle needs no correct rounding (cos and sin are formed accurately
    // from whatever tangent this gives): approximate reciprocal, square root
    // and quotient of the special-function unit
    const float sc = __fdividef(1.0f, fmaxf(al, be));  // al, be <= 1, |ga| <= 1 after it
    const float a1 = al * sc, b1 = be * sc, g1 = ga * sc;
    const float ab = a1 * b1, g2 = g1 * g1;
    if (!(g2 > (kTol32 * kTol32) * ab))
        return false;
    const float h = 0.5f * (b1 - a1);
    const float q = fmaf(h, h, g2);  // > 0
    const float t = copysignf(1.0f, h) * __fdividef(g1, fabsf(h) + q * rsqrtf(q));
    accurate_cos_sin(t, c, sn);
    big = g2 > (kLast32 * kLast32) * ab;
    return true;
}

// Columns la, lb of G (b2 x b2, shared memory) rotated like the pair.
__device__ __forceinline__ void pc32_rotate_g(float *G, int b2, int la, int lb, float c,
                                              float sn, int lane)
{
    for (int k = lane; k < b2; k += 32) {
        const float ga = G[la * b2 + k], gb = G[lb * b2 + k];
        G[la * b2 + k] = fmaf(c, ga, -sn * gb);
        G[lb * b2 + k] = fmaf(sn, ga, c * gb);
    }
}

// One warp orthogonalises the FP32 columns x, y (ms rows, shared memory)
// and rotates G's columns la, lb with them; returns whether |cos| > kLast32.
__device__ __forceinline__ bool pc32_pair_smem(float *x, float *y, int ms, float *G, int b2,
                                               int la, int lb, int lane)
{
    float al = 0.0f, be = 0.0f, ga = 0.0f;
    for (int i = lane; i < ms; i += 32) {
        const float xv = x[i], yv = y[i];
        al = fmaf(xv, xv, al);
        be = fmaf(yv, yv, be);
        ga = fmaf(xv, yv, ga);
    }
    warp_sum3f(al, be, ga);
    float c, sn;
    bool big;
    if (pc32_rotation(al, be, ga, c, sn, big)) {
        for (int i = lane; i < ms; i += 32) {
            const float xv = x[i], yv = y[i];
            x[i] = fmaf(c, xv, -sn * yv);
            y[i] = fmaf(sn, xv, c * yv);
        }
        pc32_rotate_g(G, b2, la, lb, c, sn, lane);
    }
    return big;
}

// Columns [blk b, blk b + b) of X between global memory (ld m, through L2)
// and shared memory (ld ms; zeros past row m and past column n).
__device__ void pc32_load(const Pc32Job &J, int blk, float *dst)
{
    const int m = J.m, ms = J.ms, b = J.b, c0 = blk * b;
    const int nc = min(b, max(0, J.n - c0));
    if ((m & 3) == 0) {
        const int m4 = m / 4, ms4 = ms / 4;
        for (int e = threadIdx.x; e < b * ms4; e += blockDim.x) {
            const int c = e / ms4, i4 = e - c * ms4;
            float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (c < nc && i4 < m4)
                v = __ldcg(reinterpret_cast<const float4 *>(J.X + size_t(c0 + c) * m) + i4);
            reinterpret_cast<float4 *>(dst + size_t(c) * ms)[i4] = v;
        }
    } else {
        for (int e = threadIdx.x; e < b * ms; e += blockDim.x) {
            const int c = e / ms, i = e - c * ms;
            dst[e] = (c < nc && i < m) ? __ldcg(J.X + size_t(c0 + c) * m + i) : 0.0f;
        }
    }
}
__device__ void pc32_store(const Pc32Job &J, int blk, const float *src)
{
    const int m = J.m, ms = J.ms, b = J.b, c0 = blk * b;
    const int nc = min(b, max(0, J.n - c0));
    if ((m & 3) == 0) {
        const int m4 = m / 4, ms4 = ms / 4;
        for (int e = threadIdx.x; e < nc * m4; e += blockDim.x) {
            const int c = e / m4, i4 = e - c * m4;
            __stcg(reinterpret_cast<float4 *>(J.X + size_t(c0 + c) * m) + i4,
                   reinterpret_cast<const float4 *>(src + size_t(c) * ms)[i4]);
        }
    } else {
        for (int e = threadIdx.x; e < nc * m; e += blockDim.x) {
            const int c = e / m, i = e - c * m;
            __stcg(J.X + size_t(c0 + c) * m + i, src[size_t(c) * ms + i]);
        }
    }
}

// The CTAs of a launch are split among np problems: problem p owns CTAs
// [begin[p], begin[p + 1]) and synchronises only among them (its own
// flags and barrier words).
__device__ __forceinline__ int problem_of(const int *begin, int np)
{
    int lo = 0, hi = np - 1;
    while (lo < hi) {  // last p with begin[p] <= blockIdx.x
        const int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= int(blockIdx.x)) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int RPT>
__global__ void __launch_bounds__(kPairThreads)
jacobi_kernel(const SvdWork *works, const int *begin, int np)
{
    const int p = problem_of(begin, np);
    const SvdWork w = works[p];
    jacobi_body<RPT>(w, int(blockIdx.x) - begin[p], begin[p + 1] - begin[p]);
}

// At most 48 registers a thread (ten 128-thread CTAs per SM), or 40 (twelve:
// a CTA per pair for the four 1024 x 768 problems of a batch, which ten an
// SM cannot hold -- a CTA with two pairs a round would set every round's
// pace; the same arithmetic, some registers spilled).
template <int RPL, int MINB = 10>
__global__ void __launch_bounds__(kPairThreads, MINB)
jacobi_lean_kernel(const SvdWork *works, const int *begin, int np)
{
    const int p = problem_of(begin, np);
    const SvdWork w = works[p];
    jacobi_lean_body<RPL>(w, int(blockIdx.x) - begin[p], begin[p + 1] - begin[p]);
}

template <int RPL>
__global__ void __launch_bounds__(kGroupThreads, 3)
jacobi_group_kernel(const SvdWork *works, const int *begin, int np)
{
    const int p = problem_of(begin, np);
    const SvdWork w = works[p];
    jacobi_group_body<RPL>(w, int(blockIdx.x) - begin[p], begin[p + 1] - begin[p]);
}

// The FP32 sweeps: a cooperative launch, problem p on CTAs [begin[p],
// begin[p + 1]) (J.C of them), b warps a CTA; dynamic shared memory: the
// two blocks (b ms floats each) and G.  Lane l of a warp holds rows 128 k +
// 4 l .. + 3 of a column.  Every CTA of a problem takes the same branches
// (its grid barriers; bounded: WOS_DEVICE_TIMEOUT in bar[5] and an exit).
__global__ void __launch_bounds__(32 * kPc32MaxB)
pc32_sweeps_kernel(const Pc32Job *jobs, const int *begin, int np)
{
    extern __shared__ float4 pc32_sm[];
    const int pb = problem_of(begin, np);
    const Pc32Job J = jobs[pb];
    const int cta = int(blockIdx.x) - begin[pb], C = J.C, NB = 2 * C;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int b = J.b, ms = J.ms, b2 = 2 * b, nk = ms / 128;
    float *R0 = reinterpret_cast<float *>(pc32_sm), *R1 = R0 + size_t(b) * ms;
    float *G = R1 + size_t(b) * ms;
    __shared__ int s_big;
    unsigned *flags = J.bar + 8;
    const float4 zero4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int sweep = 0; sweep < kMaxSweeps32; ++sweep) {
        if (cta == 0 && threadIdx.x == 0)
            flags[(sweep + 1) % 3] = 0u;
        if (threadIdx.x == 0)
            s_big = 0;
        bool big = false;
        for (int r = 0; r < NB - 1; ++r) {
            const int bA = rr_player(cta, r, NB);
            const int bB = rr_player(NB - 1 - cta, r, NB);
            pc32_load(J, bA, R0);
            pc32_load(J, bB, R1);
            for (int e = threadIdx.x; e < b2 * b2; e += blockDim.x)
                G[e] = (e / b2 == e % b2) ? 1.0f : 0.0f;
            __syncthreads();
            if (r == 0) {
                // pairs inside each block: round-robin on its b columns,
                // warps [0, b/2) on block A and [b/2, b) on block B
                const int hb = b / 2, w2 = wid < hb ? wid : wid - hb;
                float *blk = wid < hb ? R0 : R1;
                const int l0 = wid < hb ? 0 : b;
                for (int u = 0; u < b - 1; ++u) {
                    const int i = rr_player(w2, u, b), j = rr_player(b - 1 - w2, u, b);
                    const int lo = min(i, j), hi = max(i, j);
                    big |= pc32_pair_smem(blk + size_t(lo) * ms, blk + size_t(hi) * ms, ms, G, b2,
                                          l0 + lo, l0 + hi, lane);
                    __syncthreads();
                }
            }
            // pairs across the blocks: A[w] (registers) with B[(w + u) mod b];
            // slot k of the current buffer holds B[(k + u) mod b]
            float4 xr[kPc32Chunks], yr[kPc32Chunks];
#pragma unroll
            for (int k = 0; k < kPc32Chunks; ++k)
                xr[k] = k < nk ? reinterpret_cast<const float4 *>(R0 + size_t(wid) * ms)[32 * k + lane]
                               : zero4;
            __syncthreads();  // R0 is free: the next buffer
            float *cur = R1, *nxt = R0;
            for (int u = 0; u < b; ++u) {
                const float4 *y4 = reinterpret_cast<const float4 *>(cur + size_t(wid) * ms);
                float al = 0.0f, be = 0.0f, ga = 0.0f;
#pragma unroll
                for (int k = 0; k < kPc32Chunks; ++k) {
                    const float4 y = k < nk ? y4[32 * k + lane] : zero4;
                    yr[k] = y;
                    al = fmaf(xr[k].x, xr[k].x, fmaf(xr[k].y, xr[k].y, fmaf(xr[k].z, xr[k].z, fmaf(xr[k].w, xr[k].w, al))));
                    be = fmaf(y.x, y.x, fmaf(y.y, y.y, fmaf(y.z, y.z, fmaf(y.w, y.w, be))));
                    ga = fmaf(xr[k].x, y.x, fmaf(xr[k].y, y.y, fmaf(xr[k].z, y.z, fmaf(xr[k].w, y.w, ga))));
                }
                warp_sum3f(al, be, ga);
                float c, sn;
                bool bg;
                const bool rot = pc32_rotation(al, be, ga, c, sn, bg);
                big |= bg;
                // y rotated on its way to the next warp
                float4 *o4 = reinterpret_cast<float4 *>(nxt + size_t((wid + b - 1) % b) * ms);
#pragma unroll
                for (int k = 0; k < kPc32Chunks; ++k)
                    if (k < nk) {
                        const float4 x = xr[k], y = yr[k];
                        if (rot) {
                            xr[k] = make_float4(fmaf(c, x.x, -sn * y.x), fmaf(c, x.y, -sn * y.y),
                                                fmaf(c, x.z, -sn * y.z), fmaf(c, x.w, -sn * y.w));
                            o4[32 * k + lane] =
                                make_float4(fmaf(sn, x.x, c * y.x), fmaf(sn, x.y, c * y.y),
                                            fmaf(sn, x.z, c * y.z), fmaf(sn, x.w, c * y.w));
                        } else {
                            o4[32 * k + lane] = y;
                        }
                    }
                if (rot)
                    pc32_rotate_g(G, b2, wid, b + (wid + u) % b, c, sn, lane);
                __syncthreads();
                float *t = cur;
                cur = nxt;
                nxt = t;
            }
            // b is even: cur is R1 again, B in order; A back into R0
#pragma unroll
            for (int k = 0; k < kPc32Chunks; ++k)
                if (k < nk)
                    reinterpret_cast<float4 *>(R0 + size_t(wid) * ms)[32 * k + lane] = xr[k];
            __syncthreads();
            pc32_store(J, bA, R0);
            pc32_store(J, bB, R1);
            float *gl = J.G + ((size_t(sweep) * (NB - 1) + r) * C + cta) * size_t(b2) * b2;
            for (int e = threadIdx.x; e < b2 * b2; e += blockDim.x)
                __stcg(gl + e, G[e]);
            // the blocks' stores before any CTA loads them
            if (!grid_barrier(J.bar, unsigned(C)))
                return;
        }
        if (big && lane == 0)
            atomicOr(&s_big, 1);
        __syncthreads();
        if (threadIdx.x == 0 && s_big)
            atomicOr(flags + sweep % 3, 1u);
        if (!grid_barrier(J.bar, unsigned(C)))
            return;
        const bool done = *(volatile unsigned *)(flags + sweep % 3) == 0u;
        if (cta == 0 && threadIdx.x == 0)
            J.bar[6] = unsigned(sweep + 1);
        if (done)
            break;
    }
}

// J = the product of the block rounds' G in their order: J <- J G_c on the
// 2b columns of CTA c's two blocks, for every c of each block round.  Each
// CTA owns kRpRows rows of J (independent) in shared memory, double
// buffered; a thread forms output column j of one G for all kRpRows rows.
constexpr int kRpRows = 8;

// The CTAs of a launch serve np problems: problem p owns CTAs [begin[p],
// begin[p + 1]).
__global__ void __launch_bounds__(256)
pc32_replay_kernel(const Pc32Job *jobs, const int *begin, int np)
{
    extern __shared__ float4 rp_smem[];
    const int pb = problem_of(begin, np);
    const Pc32Job J = jobs[pb];
    const int n = J.n, b = J.b, b2 = 2 * b, C = J.C, NB = 2 * C, L = NB * b;
    float *cur = reinterpret_cast<float *>(rp_smem), *nxt = cur + size_t(kRpRows) * L;
    const int r0 = (int(blockIdx.x) - begin[pb]) * kRpRows;
    for (int e = threadIdx.x; e < kRpRows * L; e += blockDim.x) {
        const int rr = e / L, j = e - rr * L;
        cur[e] = (r0 + rr == j) ? 1.0f : 0.0f;
    }
    __syncthreads();
    const int nsw = int(*(volatile unsigned *)(J.bar + 6));
    const int tasks = C * b2;
    for (int z = 0; z < nsw; ++z)
        for (int r = 0; r < NB - 1; ++r) {
            const float *gr = J.G + (size_t(z) * (NB - 1) + r) * C * size_t(b2) * b2;
            for (int t = threadIdx.x; t < tasks; t += blockDim.x) {
                const int c = t / b2, j = t - c * b2;
                const int bA = rr_player(c, r, NB);
                const int bB = rr_player(NB - 1 - c, r, NB);
                const float4 *g4 = reinterpret_cast<const float4 *>(gr + (size_t(c) * b2 + j) * b2);
                float acc[kRpRows];
#pragma unroll
                for (int rr = 0; rr < kRpRows; ++rr)
                    acc[rr] = 0.0f;
                for (int k4 = 0; k4 < b2 / 4; ++k4) {
                    const float4 g = __ldcg(g4 + k4);
                    const int k = 4 * k4;
                    const int col = k < b ? bA * b + k : bB * b + (k - b);
#pragma unroll
                    for (int rr = 0; rr < kRpRows; ++rr) {
                        const float4 v = *reinterpret_cast<const float4 *>(cur + size_t(rr) * L + col);
                        acc[rr] = fmaf(v.x, g.x, fmaf(v.y, g.y, fmaf(v.z, g.z, fmaf(v.w, g.w, acc[rr]))));
                    }
                }
                const int oc = j < b ? bA * b + j : bB * b + (j - b);
#pragma unroll
                for (int rr = 0; rr < kRpRows; ++rr)
                    nxt[size_t(rr) * L + oc] = acc[rr];
            }
            __syncthreads();
            float *tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
    for (int e = threadIdx.x; e < kRpRows * n; e += blockDim.x) {
        const int rr = e / n, j = e - rr * n;
        if (r0 + rr < n)
            J.J[size_t(j) * n + r0 + rr] = double(cur[size_t(rr) * L + j]);  // J[i][j]
    }
}

// X32 = X rounded to FP32 (m x n, both ld m).
__global__ void to32_kernel(const double *X, size_t mn, float *X32)
{
    for (size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x; t < mn;
         t += size_t(gridDim.x) * blockDim.x)
        X32[t] = float(X[t]);
}

// Squared norms of the n columns (length m) of w.W into w.nrm, a warp per
// column.
__global__ void column_sq_norms_kernel(SvdWork w)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int j = gw; j < w.n; j += nw) {
        const double *c = w.W + size_t(j) * w.m;
        double s = 0.0;
        for (int i = lane; i < w.m; i += 32)
            s = fma(c[i], c[i], s);
        s = warp_sum(s);
        if (lane == 0) {
            w.nrm[j] = s;
            w.dsc[j] = 1.0;
            w.dinv[j] = 1.0;
        }
    }
}

// X[:, j] *= d_j: the stored columns of the sweeps without V back to X.
__global__ void fold_scales_kernel(SvdWork w)
{
    const size_t nn = size_t(w.n) * w.m;
    for (size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x; t < nn;
         t += size_t(gridDim.x) * blockDim.x)
        w.W[t] *= w.dsc[t / w.m];
}

// Z = P X: row perm[k] of Z is row k of X (n x n, column-major), so that the
// columns of Z are the right singular vectors of W scaled by sigma.
__global__ void permute_rows_kernel(const double *X, const int *perm, int n, double *Z)
{
    const size_t nn = size_t(n) * n;
    for (size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x; t < nn;
         t += size_t(gridDim.x) * blockDim.x) {
        const int j = int(t / n), k = int(t - size_t(j) * n);
        Z[size_t(j) * n + perm[k]] = X[t];
    }
}

// One product of a batched GEMM launch (blockIdx.z = the job): C = alpha
// op(A) B + beta D in FP64, column-major: op(A) = A (m x k, lda) or A^T (A
// k x m, lda); B k x n (ldb); C and D m x n (ldc); no D when it is null.
struct GemmJob {
    const double *A, *B, *D;
    double *C;
    int m, n, k, lda, ldb, ldc;
    double alpha, beta;
};

// 64 x 64 tiles of C per block of 256 threads, 4 x 4 per thread, k in steps
// of 16 through shared memory; the launch's x, y cover the largest job (the
// tiles outside a smaller one return).  SYM (C = A^T A, m = n): only the
// tiles on and above the diagonal, each written to both triangles (element
// (i, j) and (j, i) are the same products in the same order).
constexpr int kGemmTile = 64, kGemmK = 16;

template <bool TA, bool SYM = false>
__global__ void __launch_bounds__(256)
dgemm_kernel(const GemmJob *jobs)
{
    const GemmJob g = jobs[blockIdx.z];
    const int m = g.m, n = g.n, k = g.k;
    const int i0 = blockIdx.x * kGemmTile, j0 = blockIdx.y * kGemmTile;
    if ((SYM && blockIdx.x > blockIdx.y) || i0 >= m || j0 >= n)
        return;
    __shared__ double As[kGemmK][kGemmTile + 1];
    __shared__ double Bs[kGemmK][kGemmTile + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;  // 16 x 16 threads, 4 x 4 each
    const double *A = g.A, *B = g.B;
    const int lda = g.lda, ldb = g.ldb;
    double acc[4][4] = {};
    for (int l0 = 0; l0 < k; l0 += kGemmK) {
        // A tile: 64 rows x 16 columns of op(A); B tile: 16 rows x 64 columns
        for (int e = tid; e < kGemmTile * kGemmK; e += 256) {
            if (TA) {  // consecutive threads along k (A's columns are contiguous)
                const int ll = e % kGemmK, ii = e / kGemmK;
                const int gi = i0 + ii, gl = l0 + ll;
                As[ll][ii] = (gi < m && gl < k) ? A[size_t(gi) * lda + gl] : 0.0;
            } else {
                const int ii = e % kGemmTile, ll = e / kGemmTile;
                const int gi = i0 + ii, gl = l0 + ll;
                As[ll][ii] = (gi < m && gl < k) ? A[size_t(gl) * lda + gi] : 0.0;
            }
            const int lb = e % kGemmK, jj = e / kGemmK;
            const int gl2 = l0 + lb, gj = j0 + jj;
            Bs[lb][jj] = (gl2 < k && gj < n) ? B[size_t(gj) * ldb + gl2] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int ll = 0; ll < kGemmK; ++ll) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[ll][tx + 16 * u];
                b[u] = Bs[ll][ty + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int gi = i0 + tx + 16 * u, gj = j0 + ty + 16 * v;
            if (gi < m && gj < n) {
                const size_t o = size_t(gj) * g.ldc + gi;
                g.C[o] = g.D ? fma(g.alpha, acc[u][v], g.beta * g.D[o]) : g.alpha * acc[u][v];
                if (SYM)
                    g.C[size_t(gi) * g.ldc + gj] = g.C[o];
            }
        }
}

// C = D + alpha fl32(A) fl32(B - I) with FP32 products and sums (A, B, C, D
// FP64, n x n, column-major, ld n; C may not alias A or B; job fields m = n,
// D, alpha): the correction terms of the Newton-Schulz steps, Q (Q^T Q - I),
// whose size (1e-4 and below) makes FP32's relative rounding negligible next
// to FP64's.  The tiling of dgemm_kernel.
__global__ void __launch_bounds__(256)
ns_correction_kernel(const GemmJob *jobs)
{
    const GemmJob g = jobs[blockIdx.z];
    const int n = g.n;
    const int i0 = blockIdx.x * kGemmTile, j0 = blockIdx.y * kGemmTile;
    if (i0 >= n || j0 >= n)
        return;
    __shared__ float As[kGemmK][kGemmTile + 1];
    __shared__ float Bs[kGemmK][kGemmTile + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const double *A = g.A, *B = g.B;
    float acc[4][4] = {};
    for (int l0 = 0; l0 < n; l0 += kGemmK) {
        for (int e = tid; e < kGemmTile * kGemmK; e += 256) {
            const int ii = e % kGemmTile, ll = e / kGemmTile;
            const int gi = i0 + ii, gl = l0 + ll;
            As[ll][ii] = (gi < n && gl < n) ? float(A[size_t(gl) * n + gi]) : 0.0f;
            const int lb = e % kGemmK, jj = e / kGemmK;
            const int gl2 = l0 + lb, gj = j0 + jj;
            Bs[lb][jj] = (gl2 < n && gj < n)
                             ? float(B[size_t(gj) * n + gl2] - (gl2 == gj ? 1.0 : 0.0))
                             : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int ll = 0; ll < kGemmK; ++ll) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[ll][tx + 16 * u];
                b[u] = Bs[ll][ty + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int gi = i0 + tx + 16 * u, gj = j0 + ty + 16 * v;
            if (gi < n && gj < n) {
                const size_t o = size_t(gj) * n + gi;
                g.C[o] = fma(g.alpha, double(acc[u][v]), g.D[o]);
            }
        }
}

enum GemmKind { kGemmNN = 0, kGemmSyrk = 1, kGemmNsCorrection = 2 };

// One launch for every job (dev: room for jobs.size() records; stream order
// lets consecutive launches reuse it).
cudaError_t gemm_batch(cudaStream_t st, GemmKind kind, const std::vector<GemmJob> &jobs,
                       GemmJob *dev, int *launches)
{
    if (jobs.empty())
        return cudaSuccess;
    int mm = 1, nn = 1;
    for (const GemmJob &g : jobs) {
        mm = std::max(mm, g.m);
        nn = std::max(nn, g.n);
    }
    cudaMemcpyAsync(dev, jobs.data(), sizeof(GemmJob) * jobs.size(), cudaMemcpyHostToDevice, st);
    const dim3 gg(unsigned((mm + kGemmTile - 1) / kGemmTile),
                  unsigned((nn + kGemmTile - 1) / kGemmTile), unsigned(jobs.size()));
    if (kind == kGemmNN)
        dgemm_kernel<false><<<gg, 256, 0, st>>>(dev);
    else if (kind == kGemmSyrk)
        dgemm_kernel<true, true><<<gg, 256, 0, st>>>(dev);
    else
        ns_correction_kernel<<<gg, 256, 0, st>>>(dev);
    ++*launches;
    return cudaGetLastError();
}

GemmJob gemm_nn(int m, int n, int k, const double *A, const double *B, double *C)
{
    return GemmJob{A, B, nullptr, C, m, n, k, m, k, m, 1.0, 0.0};
}
GemmJob gemm_syrk(int n, int k, const double *A, double *M)  // M = A^T A
{
    return GemmJob{A, A, nullptr, M, n, n, k, k, k, n, 1.0, 0.0};
}
GemmJob gemm_ns(int n, const double *A, const double *M, const double *D, double *C)
{
    return GemmJob{A, M, D, C, n, n, n, n, n, n, -0.5, 0.0};  // C = D - A (M - I) / 2
}


// B (worked orientation): W[:, col] with col over Gamma_1 elements (or
// over points when transposed); V_w = I.
__global__ void form_B_kernel(SvdWork w, const uint32_t *counts, int M_D, int M_tot,
                              double invN, const int *g1_idx, int M_1,
                              const double *nu, const double *sigma, int transposed)
{
    size_t total = size_t(M_D) * M_1;
    double nu_def = 1.0 / sqrt(double(M_D));
    for (size_t q = blockIdx.x * size_t(blockDim.x) + threadIdx.x; q < total;
         q += size_t(gridDim.x) * blockDim.x) {
        int i = int(q / M_1), l = int(q % M_1);
        int j = g1_idx[l];
        double v = (nu ? nu[i] : nu_def) * double(counts[size_t(i) * M_tot + j]) * invN /
                   sqrt(sigma[j]);
        if (!transposed)
            w.W[size_t(l) * M_D + i] = v;  // column l, row i
        else
            w.W[size_t(i) * M_1 + l] = v;  // column i, row l
    }
    size_t nn = size_t(w.n) * w.n;
    for (size_t q = blockIdx.x * size_t(blockDim.x) + threadIdx.x; q < nn;
         q += size_t(gridDim.x) * blockDim.x)
        w.Vw[q] = (q / w.n == q % w.n) ? 1.0 : 0.0;
}

__global__ void column_norms_kernel(SvdWork w, double *sv)
{
    int lane = threadIdx.x & 31;
    int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int nw = (gridDim.x * blockDim.x) >> 5;
    for (int j = gw; j < w.n; j += nw) {
        const double *c = w.W + size_t(j) * w.m;
        double s = 0.0;
        for (int i = lane; i < w.m; i += 32)
            s = fma(c[i], c[i], s);
        s = warp_sum(s);
        if (lane == 0)
            sv[j] = sqrt(s);
    }
}

// ---------------------------------------------------------------------------
// Preconditioning (Drmac & Veselic, "New fast and accurate Jacobi SVD
// algorithm", SIAM J. Matrix Anal. Appl. 29 (2008)): W P = Q R by Householder
// QR with column pivoting (Businger & Golub), then one-sided Jacobi on
// X = R^T, which converges in fewer sweeps than on W itself (15-17 -> 10 on
// the operators of the benchmark geometries) and works on n-long columns.
// From X = U_X Sigma V_X^T: W = (Q V_X) Sigma (P U_X)^T.
// ---------------------------------------------------------------------------
constexpr int kQrThreads = 256;
constexpr double kTol3z = 1.4901161193847656e-08;  // sqrt(2^-52), xLAQP2's test

struct QrWork {
    double *A;        // m x n column-major, factored in place (R above, v below)
    int m, n;
    double *tau;      // n reflector scalars
    int *perm;        // n: physical column of pivot k
    double *cn;       // n: squared norm of rows k..m-1 of each column
    double *cn0;      // n: the same at its last exact computation
    int *done;        // n: column already a pivot
    double *pval;     // per CTA and pivot parity: largest remaining squared
    int *pidx;        // norm and its column (lowest index on ties); two sets,
                      // so a CTA may publish pivot k + 1 while another still
                      // reads pivot k (pivot k + 2 needs every CTA's k + 1 arrival)
    unsigned *bar;    // [0] arrivals (monotonic), [1] reflector k ready (k + 1),
                      // [5] status
};

__device__ __forceinline__ void red_add_release(unsigned *a, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

// Wait (bounded, about 2 s) until *a >= want; records WOS_DEVICE_TIMEOUT in
// *status and returns false on time-out or when another CTA already did.
__device__ bool wait_at_least(const unsigned *a, unsigned want, unsigned *status)
{
    if (ld_acquire(a) >= want)
        return true;
    const long long t0 = clock64();
    for (unsigned it = 1;; ++it) {
        if (ld_acquire(a) >= want)
            return true;
        if ((it & 63u) == 0u) {
            if (clock64() - t0 > 4000000000LL) {
                atomicExch(status, unsigned(WOS_DEVICE_TIMEOUT));
                return false;
            }
            if (*(volatile unsigned *)status != 0u)
                return false;
        }
    }
}

// Sum of one double per thread over the block, returned to every thread.
// One thread adds the warps' partial sums (a warp FP64 instruction holds its
// sub-partition's FP64 unit for 64 cycles whatever its active lanes, so the
// other warps must not repeat the additions) and publishes the total in
// red[32]; red holds at least 33 doubles.
__device__ double block_sum(double v, double *red)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0)
        red[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < int(blockDim.x >> 5); ++q)
            s += red[q];
        red[32] = s;
    }
    __syncthreads();
    return red[32];
}

// Index of the largest value over the block (lowest index on ties), returned
// to every thread.
__device__ int block_argmax(double v, int i, double *red, int *ired)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(FULL, v, o);
        const int oi = __shfl_xor_sync(FULL, i, o);
        if (ov > v || (ov == v && oi < i)) {
            v = ov;
            i = oi;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        red[wid] = v;
        ired[wid] = i;
    }
    __syncthreads();
    double bv = red[0];
    int bi = ired[0];
    for (int q = 1; q < int(blockDim.x >> 5); ++q)
        if (red[q] > bv || (red[q] == bv && ired[q] < bi)) {
            bv = red[q];
            bi = ired[q];
        }
    return bi;
}

// Cooperative: CTA b owns the physical columns c = b (mod gridDim.x).  Per
// pivot k: every CTA publishes its largest remaining column norm; after a grid
// barrier every CTA takes the same global argmax pc; pc's owner builds the
// reflector of rows k..m-1 (xLARFG: beta = -sign(alpha) ||x||, tau =
// (beta - alpha) / beta, v = x / (alpha - beta)); after a second barrier every
// CTA applies it to its remaining columns and downdates their norms,
// recomputing one exactly when cancellation has eaten half its digits
// (xLAQP2's test).  Barriers are bounded (WOS_DEVICE_TIMEOUT).
__device__ void qrcp_body(const QrWork &q, const int b, const int G)
{
    __shared__ double red[36];  // warp partials, [32] a block sum, [33..35] scalars
    __shared__ int ired[32];
    const int tid = threadIdx.x;
    const int m = q.m, n = q.n;
    for (int c = b; c < n; c += G) {
        const double *col = q.A + size_t(c) * m;
        double s = 0.0;
        for (int i = tid; i < m; i += blockDim.x)
            s = fma(col[i], col[i], s);
        s = block_sum(s, red);
        if (tid == 0) {
            q.cn[c] = s;
            q.cn0[c] = s;
        }
    }
    for (int k = 0; k < n; ++k) {
        if (tid == 0) {
            double bv = -1.0;
            int bi = -1;
            for (int c = b; c < n; c += G)
                if (!q.done[c] && q.cn[c] > bv) {
                    bv = q.cn[c];
                    bi = c;
                }
            q.pval[(k & 1) * G + b] = bv;
            q.pidx[(k & 1) * G + b] = bi;
        }
        // arrival counter: every CTA adds 1 per pivot (release) and waits
        // until all G have arrived for this pivot (acquire)
        __syncthreads();
        __shared__ int go;
        if (tid == 0) {
            red_add_release(q.bar, 1u);
            go = wait_at_least(q.bar, unsigned(G) * unsigned(k + 1), q.bar + 5);
        }
        __syncthreads();
        if (!go)
            return;
        // global argmax of the partials (largest norm, lowest column on ties):
        // the partials are read in parallel and reduced in the block
        double bv = -1.0;
        int pc = 0x7fffffff;
        for (int g = tid; g < G; g += blockDim.x) {
            const int i = __ldcg(q.pidx + (k & 1) * G + g);
            const double v = __ldcg(q.pval + (k & 1) * G + g);
            if (i >= 0 && (v > bv || (v == bv && i < pc))) {
                bv = v;
                pc = i;
            }
        }
        pc = block_argmax(bv, pc, red, ired);
        if (pc < 0 || pc >= n)
            pc = 0;  // unreachable: n - k columns remain
        if (pc % G == b) {
            double *col = q.A + size_t(pc) * m;
            double xn2 = 0.0;
            for (int i = k + 1 + tid; i < m; i += blockDim.x)
                xn2 = fma(col[i], col[i], xn2);
            xn2 = block_sum(xn2, red);
            const double alpha = col[k];
            // the scalars by two threads of two warps (tau, and the scale)
            if (xn2 > 0.0 && (tid == 0 || tid == 32)) {
                const double bt = -copysign(sqrt(fma(alpha, alpha, xn2)), alpha);
                if (tid == 0) {
                    red[33] = bt;
                    red[34] = (bt - alpha) / bt;
                } else {
                    red[35] = 1.0 / (alpha - bt);
                }
            }
            __syncthreads();
            double tau = 0.0, beta = alpha;
            if (xn2 > 0.0) {
                beta = red[33];
                tau = red[34];
                const double scal = red[35];
                for (int i = k + 1 + tid; i < m; i += blockDim.x)
                    col[i] *= scal;
            }
            __syncthreads();
            if (tid == 0) {
                col[k] = beta;
                q.tau[k] = tau;
                q.perm[k] = pc;
                q.done[pc] = 1;
                __threadfence();  // the block's column writes (ordered by the barrier above)
                st_relaxed(q.bar + 1, unsigned(k + 1));
            }
            __syncthreads();
        } else {
            if (tid == 0)
                go = wait_at_least(q.bar + 1, unsigned(k + 1), q.bar + 5);
            __syncthreads();
            if (!go)
                return;
        }
        const double tau = __ldcg(q.tau + k);
        const double *v = q.A + size_t(pc) * m;
        for (int c = b; c < n; c += G) {
            if (q.done[c])
                continue;
            double *col = q.A + size_t(c) * m;
            if (tau != 0.0) {
                double w = 0.0;
                for (int i = k + 1 + tid; i < m; i += blockDim.x)
                    w = fma(__ldcg(v + i), col[i], w);
                w = block_sum(w, red) + col[k];
                const double tw = tau * w;
                for (int i = k + 1 + tid; i < m; i += blockDim.x)
                    col[i] = fma(-tw, __ldcg(v + i), col[i]);
                __syncthreads();
                if (tid == 0)
                    col[k] -= tw;
            }
            __syncthreads();
            // |x|^2 - r^2, or an exact recomputation when cancellation has
            // eaten half the digits (xLAQP2's test multiplied out: no
            // division on the FP64 pipe)
            const double r = col[k], cn = q.cn[c];
            double t = 0.0;
            bool recompute = false;
            if (cn > 0.0) {
                t = fmax(fma(-r, r, cn), 0.0);
                recompute = t <= kTol3z * q.cn0[c];
            }
            if (recompute) {
                double s = 0.0;
                for (int i = k + 1 + tid; i < m; i += blockDim.x)
                    s = fma(col[i], col[i], s);
                s = block_sum(s, red);
                if (tid == 0) {
                    q.cn[c] = s;
                    q.cn0[c] = s;
                }
            } else if (tid == 0) {
                q.cn[c] = t;
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(kQrThreads)
qrcp_kernel(const QrWork *works, const int *begin, int np)
{
    const int p = problem_of(begin, np);
    const QrWork q = works[p];
    qrcp_body(q, int(blockIdx.x) - begin[p], begin[p + 1] - begin[p]);
}

// Householder QR without pivoting of the columns taken in a fixed order
// (perm: decreasing norm, sort_columns_kernel), for the problems whose
// sweeps start from FP32 ones: those sweeps, not the pivoting, precondition
// the FP64 sweeps, and the singular values' relative accuracy rests on the
// column-wise backward stability of Householder QR, pivoted or not.  With
// the order fixed there is no pivot search, so no grid-wide step per
// column: CTA b owns positions k = b (mod G); the owner of position k forms
// reflector k (xLARFG, as qrcp_body) once the k reflectors before it have
// reached its column, and publishes it with a flag (done[k]); every CTA
// applies the reflectors in order to its later columns, the owner of
// position k + 1 first to that column, so that the next reflector follows
// after one flag latency, one column update and one reflector (look-ahead).
// The waits are bounded (WOS_DEVICE_TIMEOUT).
__device__ void qrs_reflect(const QrWork &q, int k, double *red)
{
    const int tid = threadIdx.x, m = q.m;
    double *c = q.A + size_t(q.perm[k]) * m;
    double xn2 = 0.0;
    for (int i = k + 1 + tid; i < m; i += blockDim.x)
        xn2 = fma(c[i], c[i], xn2);
    xn2 = block_sum(xn2, red);
    const double alpha = c[k];
    if (xn2 > 0.0 && (tid == 0 || tid == 32)) {
        const double bt = -copysign(sqrt(fma(alpha, alpha, xn2)), alpha);
        if (tid == 0) {
            red[33] = bt;
            red[34] = (bt - alpha) / bt;
        } else {
            red[35] = 1.0 / (alpha - bt);
        }
    }
    __syncthreads();
    if (xn2 > 0.0) {
        const double scal = red[35];
        for (int i = k + 1 + tid; i < m; i += blockDim.x)
            c[i] *= scal;
    }
    __syncthreads();
    if (tid == 0) {
        c[k] = xn2 > 0.0 ? red[33] : alpha;
        q.tau[k] = xn2 > 0.0 ? red[34] : 0.0;
        __threadfence();  // the block's column writes (ordered by the barrier above)
        st_relaxed(reinterpret_cast<unsigned *>(q.done) + k, 1u);
    }
    __syncthreads();
}

// Column at position pos <- H_k (column): w = c_k + v . c (v_k = 1), c -= tau w v.
__device__ void qrs_apply(const QrWork &q, int k, int pos, double tau, double *red)
{
    const int tid = threadIdx.x, m = q.m;
    if (tau == 0.0)
        return;
    const double *v = q.A + size_t(q.perm[k]) * m;
    double *c = q.A + size_t(q.perm[pos]) * m;
    double w = 0.0;
    for (int i = k + 1 + tid; i < m; i += blockDim.x)
        w = fma(__ldcg(v + i), c[i], w);
    w = block_sum(w, red) + c[k];
    const double tw = tau * w;
    for (int i = k + 1 + tid; i < m; i += blockDim.x)
        c[i] = fma(-tw, __ldcg(v + i), c[i]);
    __syncthreads();
    if (tid == 0)
        c[k] -= tw;
    __syncthreads();
}

// Columns at positions pos[0..cnt) (cnt <= 4) <- H_k (column), their dot
// products with v reduced together: a transposed butterfly leaves column j's
// warp sum in lanes 8j..8j+7 after 6 additions a lane (instead of 5 a
// column), then one thread a column adds the warps' partials.
__device__ void qrs_apply4(const QrWork &q, int k, const int *pos, int cnt, double tau,
                           double *red)
{
    __shared__ double part[4][32];  // [column][warp]
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, m = q.m;
    if (tau == 0.0)
        return;
    const double *v = q.A + size_t(q.perm[k]) * m;
    double *c[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
        c[j] = q.A + size_t(q.perm[pos[j < cnt ? j : 0]]) * m;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = k + 1 + tid; i < m; i += blockDim.x) {
        const double vi = __ldcg(v + i);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j < cnt)
                a[j] = fma(vi, c[j][i], a[j]);
    }
    const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
    double k0 = hi16 ? a[2] : a[0], k1 = hi16 ? a[3] : a[1];
    k0 += __shfl_xor_sync(FULL, hi16 ? a[0] : a[2], 16);
    k1 += __shfl_xor_sync(FULL, hi16 ? a[1] : a[3], 16);
    double t = hi8 ? k1 : k0;
    t += __shfl_xor_sync(FULL, hi8 ? k0 : k1, 8);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1)
        t += __shfl_xor_sync(FULL, t, o);
    if ((lane & 7) == 0)
        part[lane >> 3][wid] = t;  // lanes 0, 8, 16, 24: columns 0, 1, 2, 3
    __syncthreads();
    if (tid < cnt) {
        double w = 0.0;
        for (int g = 0; g < int(blockDim.x >> 5); ++g)
            w += part[tid][g];
        red[tid] = tau * (w + q.A[size_t(q.perm[pos[tid]]) * m + k]);  // tau w
    }
    __syncthreads();
    double tw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
        tw[j] = j < cnt ? red[j] : 0.0;
    for (int i = k + 1 + tid; i < m; i += blockDim.x) {
        const double vi = __ldcg(v + i);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j < cnt)
                c[j][i] = fma(-tw[j], vi, c[j][i]);
    }
    __syncthreads();
    if (tid < cnt)
        q.A[size_t(q.perm[pos[tid]]) * m + k] -= red[tid];
    __syncthreads();
}

__device__ void qrs_body(const QrWork &q, const int b, const int G)
{
    __shared__ double red[36];
    __shared__ int go;
    const int n = q.n;
    const unsigned *flag = reinterpret_cast<const unsigned *>(q.done);
    if (b == 0)
        qrs_reflect(q, 0, red);
    for (int k = 0; k < n - 1; ++k) {
        if (k % G != b) {
            if (threadIdx.x == 0)
                go = wait_version(flag, k, 1u, q.bar + 5);
            __syncthreads();
            if (!go)
                return;
        }
        const double tau = __ldcg(q.tau + k);
        int pos = k + 1 + ((b - (k + 1)) % G + G) % G;  // this CTA's first position > k
        if (pos == k + 1) {  // look-ahead: the next reflector first
            qrs_apply(q, k, pos, tau, red);
            qrs_reflect(q, k + 1, red);
            pos += G;
        }
        while (pos < n) {  // the rest four columns at a time
            int ps[4], cnt = 0;
            for (; cnt < 4 && pos < n; pos += G)
                ps[cnt++] = pos;
            qrs_apply4(q, k, ps, cnt, tau, red);
        }
    }
}

constexpr int kQrsThreads = 256;

__global__ void __launch_bounds__(kQrsThreads)
qrs_kernel(const QrWork *works, const int *begin, int np)
{
    const int p = problem_of(begin, np);
    const QrWork q = works[p];
    qrs_body(q, int(blockIdx.x) - begin[p], begin[p + 1] - begin[p]);
}

// perm = the columns of A (m x n) in decreasing order of their squared norms
// cn (lowest index on ties): a thread per column counts the columns before it.
__global__ void sort_columns_kernel(const QrWork q)
{
    extern __shared__ double sort_cn[];  // the n norms (dynamic, n doubles)
    for (int i = threadIdx.x; i < q.n; i += blockDim.x)
        sort_cn[i] = q.cn[i];
    __syncthreads();
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < q.n; j += gridDim.x * blockDim.x) {
        const double v = sort_cn[j];
        int rank = 0;
        for (int i = 0; i < q.n; ++i) {
            const double u = sort_cn[i];
            rank += (u > v || (u == v && i < j)) ? 1 : 0;
        }
        q.perm[rank] = j;
    }
}

// Squared norms of A's n columns (length m) into cn, a warp per column.
__global__ void qr_col_norms_kernel(const QrWork q)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int j = gw; j < q.n; j += nw) {
        const double *c = q.A + size_t(j) * q.m;
        double s = 0.0;
        for (int i = lane; i < q.m; i += 32)
            s = fma(c[i], c[i], s);
        s = warp_sum(s);
        if (lane == 0)
            q.cn[j] = s;
    }
}

// X = R^T (n x n column-major): column i of X = row i of R, R[i][j] =
// A[i][perm[j]] for j >= i; V_X = I.
__global__ void build_x_kernel(const QrWork q, double *X, double *Vx)
{
    const size_t nn = size_t(q.n) * q.n;
    for (size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x; t < nn;
         t += size_t(gridDim.x) * blockDim.x) {
        const int i = int(t / q.n), j = int(t - size_t(i) * q.n);
        X[t] = j >= i ? q.A[size_t(q.perm[j]) * q.m + i] : 0.0;
        Vx[t] = i == j ? 1.0 : 0.0;
    }
}

// L = Q [V_X; 0] = H_0 H_1 ... H_{n-1} [V_X; 0]: one warp per column, the
// reflectors applied last to first (columns are independent: no barrier).
// The columns of every problem of a batch are numbered consecutively
// (problem p's start at jobs[p].col0).
struct LeftJob {
    QrWork q;
    const double *Vx;
    double *L;
    int col0;
};

__global__ void form_left_kernel(const LeftJob *jobs, int njobs, int ncols)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int g = gw; g < ncols; g += nw) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].col0 <= g) lo = mid;
            else hi = mid - 1;
        }
        const LeftJob &J = jobs[lo];
        const QrWork &q = J.q;
        const int m = q.m, n = q.n, c = g - J.col0;
        double *y = J.L + size_t(c) * m;
        for (int i = lane; i < m; i += 32)
            y[i] = i < n ? J.Vx[size_t(c) * n + i] : 0.0;
        __syncwarp();
        for (int k = n - 1; k >= 0; --k) {
            const double tau = q.tau[k];
            if (tau == 0.0)
                continue;
            const double *v = q.A + size_t(q.perm[k]) * m;
            double w = 0.0;
            for (int i = k + 1 + lane; i < m; i += 32)
                w = fma(v[i], y[i], w);
            w = warp_sum(w) + y[k];
            const double tw = tau * w;
            for (int i = k + 1 + lane; i < m; i += 32)
                y[i] = fma(-tw, v[i], y[i]);
            __syncwarp();
            if (lane == 0)
                y[k] -= tw;
            __syncwarp();
        }
    }
}

// Outputs of the preconditioned path: left vectors of W in L (m x n, unit
// columns), right vectors of W = P (X_final / sigma).  Rank, sign and layout
// as finalize_kernel.
__global__ void finalize_pre_kernel(const double *L, const double *X, const int *perm,
                                    const double *sv, int m, int n, int transposed,
                                    int lean, double *U, double *S, double *V)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int k = n;
    for (int j = gw; j < k; j += nw) {
        const double sj = sv[j];
        int rank = 0;
        for (int i = lane; i < k; i += 32) {
            const double si = sv[i];
            rank += (si > sj || (si == sj && i < j)) ? 1 : 0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            rank += __shfl_xor_sync(FULL, rank, o);
        const double inv = sj > 0.0 ? 1.0 / sj : 0.0;
        // L's columns: unit (Q V_X), or sigma^2 times unit without V (W P X)
        const double ls = lean ? inv * inv : 1.0;
        const double *lc = L + size_t(j) * m;
        const double *xc = X + size_t(j) * n;
        // sign: largest-magnitude entry of the B-side right vector (lowest
        // B row index on ties): L when transposed, else P X
        double big = -1.0;
        int arg = 0x7fffffff;
        double at = 0.0;
        const int rn = transposed ? m : n;
        for (int i = lane; i < rn; i += 32) {
            const double val = transposed ? lc[i] * ls : xc[i];
            const int row = transposed ? i : perm[i];
            const double a = fabs(val);
            if (a > big || (a == big && row < arg)) {
                big = a;
                arg = row;
                at = val;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(FULL, big, o);
            const int oa = __shfl_xor_sync(FULL, arg, o);
            const double ov = __shfl_xor_sync(FULL, at, o);
            if (ob > big || (ob == big && oa < arg)) {
                big = ob;
                arg = oa;
                at = ov;
            }
        }
        const double sign = at >= 0.0 ? 1.0 : -1.0;
        if (lane == 0)
            S[rank] = sj;
        if (!transposed) {
            for (int i = lane; i < m; i += 32)   // U: M_D = m rows
                U[size_t(i) * k + rank] = sign * (lc[i] * ls);
            for (int i = lane; i < n; i += 32)   // V: M_1 = n rows
                V[size_t(perm[i]) * k + rank] = sign * xc[i] * inv;
        } else {
            for (int i = lane; i < m; i += 32)   // V: M_1 = m rows
                V[size_t(i) * k + rank] = sign * (lc[i] * ls);
            for (int i = lane; i < n; i += 32)   // U: M_D = n rows
                U[size_t(perm[i]) * k + rank] = sign * xc[i] * inv;
        }
    }
}

constexpr int kPrecondMinN = 32;  // smaller problems run Jacobi on W directly

// Rank of every column by descending norm (ties by index), sign from the
// largest-magnitude entry of the B-side right vector, then the outputs
// U (M_D x k), S (k), V (M_1 x k), row-major.
__global__ void finalize_kernel(SvdWork w, const double *sv, int transposed,
                                double *U, double *S, double *V)
{
    int lane = threadIdx.x & 31;
    int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int nw = (gridDim.x * blockDim.x) >> 5;
    const int k = w.n;
    for (int j = gw; j < k; j += nw) {
        double sj = sv[j];
        int rank = 0;
        for (int i = lane; i < k; i += 32) {
            double si = sv[i];
            rank += (si > sj || (si == sj && i < j)) ? 1 : 0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            rank += __shfl_xor_sync(FULL, rank, o);
        // B-side right vector: V_w column (not transposed) or W column / s
        const double *rv = transposed ? (w.W + size_t(j) * w.m) : (w.Vw + size_t(j) * w.n);
        int rn = transposed ? w.m : w.n;
        double big = -1.0;
        int arg = 0;
        for (int i = lane; i < rn; i += 32) {
            double a = fabs(rv[i]);
            if (a > big) { big = a; arg = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double ob = __shfl_xor_sync(FULL, big, o);
            int oa = __shfl_xor_sync(FULL, arg, o);
            if (ob > big || (ob == big && oa < arg)) { big = ob; arg = oa; }
        }
        double sign = rv[arg] >= 0.0 ? 1.0 : -1.0;
        double inv = sj > 0.0 ? 1.0 / sj : 0.0;
        if (lane == 0)
            S[rank] = sj;
        const double *wc = w.W + size_t(j) * w.m;
        const double *vc = w.Vw + size_t(j) * w.n;
        if (!transposed) {
            for (int i = lane; i < w.m; i += 32)   // U: M_D = m rows
                U[size_t(i) * k + rank] = sign * wc[i] * inv;
            for (int i = lane; i < w.n; i += 32)   // V: M_1 = n rows
                V[size_t(i) * k + rank] = sign * vc[i];
        } else {
            for (int i = lane; i < w.m; i += 32)   // V: M_1 = m rows
                V[size_t(i) * k + rank] = sign * wc[i] * inv;
            for (int i = lane; i < w.n; i += 32)   // U: M_D = n rows
                U[size_t(i) * k + rank] = sign * vc[i];
        }
    }
}

#include "svd_cluster.cuh"

// ---------------------------------------------------------------------------
// TSVD pieces
// ---------------------------------------------------------------------------
// y_i = x_i + alpha * sum_j (C[i][j] / N) f_j  over all M_tot elements.
__global__ void counts_matvec_kernel(const uint32_t *counts, int M_D, int M_tot,
                                     double invN, const double *f, const double *x,
                                     double alpha, double *y)
{
    int lane = threadIdx.x & 31;
    int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = gw; i < M_D; i += nw) {
        const uint32_t *row = counts + size_t(i) * M_tot;
        double s = 0.0;
        for (int j = lane; j < M_tot; j += 32)
            s = fma(double(row[j]), f[j], s);
        s = warp_sum(s);
        if (lane == 0)
            y[i] = (x ? x[i] : 0.0) + alpha * s * invN;
    }
}

// f[j] = u0 on Gamma_0 (in Gamma_0 order), 0 on Gamma_1; or u1 on Gamma_1.
__global__ void scatter_kernel(const int *idx, int n, const double *vals, double *f)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
        f[idx[q]] = vals ? vals[q] : 0.0;
}

// t_c = filter(S_c) * sum_i U[i][c] nu_i b_i, c < r (one warp per c).
__global__ void tsvd_t_kernel(const double *U, const double *S, int M_D, int k, int r,
                              const double *nu, const double *b, double alpha, double *t)
{
    int lane = threadIdx.x & 31;
    int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int nw = (gridDim.x * blockDim.x) >> 5;
    double nu_def = 1.0 / sqrt(double(M_D));
    for (int c = gw; c < r; c += nw) {
        double s = 0.0;
        for (int i = lane; i < M_D; i += 32)
            s = fma(U[size_t(i) * k + c], (nu ? nu[i] : nu_def) * b[i], s);
        s = warp_sum(s);
        if (lane == 0) {
            double sc = S[c];
            double filt = alpha > 0.0 ? sc / (sc * sc + alpha) : (sc > 0.0 ? 1.0 / sc : 0.0);
            t[c] = filt * s;
        }
    }
}

// u1[l] = sigma_{g1[l]}^{-1/2} sum_{c<r} V[l][c] t_c
__global__ void tsvd_u_kernel(const double *V, int M_1, int k, int r, const double *t,
                              const int *g1_idx, const double *sigma, double *u1)
{
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < M_1; l += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < r; ++c)
            s = fma(V[size_t(l) * k + c], t[c], s);
        u1[l] = s / sqrt(sigma[g1_idx[l]]);
    }
}

struct Lists {
    std::vector<int> g1, g0;
};

Lists split(const uint8_t *gamma1, int M_tot)
{
    Lists L;
    for (int j = 0; j < M_tot; ++j)
        (gamma1[j] ? L.g1 : L.g0).push_back(j);
    return L;
}

// One SVD problem of a batch: inputs, orientation and its workspace.
struct SvdProb {
    const uint32_t *counts;
    int M_D, M_tot, M_1, transposed;
    uint32_t N;
    const double *nu, *sigma;
    double *U, *S, *V;
    Lists L;
    bool pre;
    bool lean;       // grid-wide Jacobi without V (more than 256 columns)
    bool mixed;      // lean, with the FP32 preconditioning sweeps first
    double *X0;      // mixed: X = R^T (the FP64 sweeps start from X Q)
    Pc32Job pc;      // mixed: the FP32 sweeps' work
    int cl;          // cluster size of the cluster kernel, 0 = grid-wide kernels
    SvdWork w, wj;   // W itself, and the matrix Jacobi works on (W or X = R^T)
    QrWork q;
    double *sv, *Lb;
    double *W0;      // lean: a copy of W (the QR overwrites W)
    int *g1;
    int qgrid;
};

// Columns above which the grid-wide Jacobi runs without V (jacobi_lean_body):
// the sizes the cluster kernel cannot take, where the sweeps' FP64 work
// bounds the factorisation.
constexpr int kLeanMinN = kClMaxN + 1;

int rpt_of(int m)
{
    // the fewest rows per thread that hold a column (a masked-off row still
    // costs its warp's FP64 instruction)
    const int need = (m + kPairThreads - 1) / kPairThreads;
    return need <= 6 ? (need < 1 ? 1 : need) : 8;
}

// Rows a lane keeps in registers in the lean sweeps (a column of m rows
// over a warp; longer columns stream the rest).
int rpl_of(int m)
{
    const int need = (m + 31) / 32;
    return need <= 8 ? 8 : need <= 16 ? 16 : need <= 24 ? 24 : 32;
}

const void *jacobi_group_kernel_rpl(int rpl)
{
    switch (rpl) {
    case 8: return reinterpret_cast<const void *>(&jacobi_group_kernel<8>);
    case 16: return reinterpret_cast<const void *>(&jacobi_group_kernel<16>);
    case 24: return reinterpret_cast<const void *>(&jacobi_group_kernel<24>);
    default: return reinterpret_cast<const void *>(&jacobi_group_kernel<32>);
    }
}

const void *jacobi_lean_kernel_rpl(int rpl, bool dense = false)
{
    if (dense)
        switch (rpl) {
        case 8: return reinterpret_cast<const void *>(&jacobi_lean_kernel<8, 12>);
        case 16: return reinterpret_cast<const void *>(&jacobi_lean_kernel<16, 12>);
        case 24: return reinterpret_cast<const void *>(&jacobi_lean_kernel<24, 12>);
        default: return reinterpret_cast<const void *>(&jacobi_lean_kernel<32, 12>);
        }
    switch (rpl) {
    case 8: return reinterpret_cast<const void *>(&jacobi_lean_kernel<8>);
    case 16: return reinterpret_cast<const void *>(&jacobi_lean_kernel<16>);
    case 24: return reinterpret_cast<const void *>(&jacobi_lean_kernel<24>);
    default: return reinterpret_cast<const void *>(&jacobi_lean_kernel<32>);
    }
}

// The FP32 sweeps' CTAs for n columns (blocks of about 12 columns), their
// block width (a multiple of 4, n <= 2 C b), the shared-memory column stride
// for m rows, and the shared memory of their two kernels.
int pc32_ctas(int n)
{
    return std::min(kPc32MaxCtas, std::max(2, (n + 23) / 24));
}
int pc32_b(int n)
{
    const int nb = 2 * pc32_ctas(n);
    return 4 * ((n + 4 * nb - 1) / (4 * nb));
}
int pc32_ms(int m)
{
    return (m + 127) / 128 * 128;
}
size_t pc32_smem(int n)
{
    const size_t b = size_t(pc32_b(n));
    return (2 * b * pc32_ms(n) + 4 * b * b) * sizeof(float);
}
size_t pc32_replay_smem(int n)
{
    return size_t(2) * kRpRows * 2 * pc32_ctas(n) * pc32_b(n) * sizeof(float);
}

// Opts kfn in to the most dynamic shared memory a CTA may have next to its
// static shared memory (always the same value, so that concurrent callers
// never see a smaller limit); false if that fails.
bool allow_max_smem(const void *kfn, const wos_context *ctx)
{
    cudaFuncAttributes fa = {};
    if (cudaFuncGetAttributes(&fa, kfn) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int dyn = wos::ctx_max_smem(ctx) - int(fa.sharedSizeBytes);
    if (dyn <= 0 ||
        cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) !=
            cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

// Whether the FP32 sweeps take an n-column problem (n x n X): its blocks
// fit the warps and the shared memory of a CTA, its columns a lane's
// registers, and its CTAs the GPU.
bool pc32_fits(const wos_context *ctx, int n)
{
    if (n < 32 || pc32_b(n) > kPc32MaxB || pc32_ms(n) > 128 * kPc32Chunks)
        return false;
    const void *sk = reinterpret_cast<const void *>(&pc32_sweeps_kernel);
    const void *rk = reinterpret_cast<const void *>(&pc32_replay_kernel);
    if (!allow_max_smem(sk, ctx) || !allow_max_smem(rk, ctx))
        return false;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, sk, 32 * pc32_b(n), pc32_smem(n)) !=
        cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaFuncAttributes fr = {};
    if (cudaFuncGetAttributes(&fr, rk) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return bps >= 1 && pc32_ctas(n) <= bps * wos::ctx_sm_count(ctx) &&
           pc32_replay_smem(n) + fr.sharedSizeBytes <= size_t(wos::ctx_max_smem(ctx));
}

const void *jacobi_kernel_rpt(int rpt)
{
    switch (rpt) {
    case 1: return reinterpret_cast<const void *>(&jacobi_kernel<1>);
    case 2: return reinterpret_cast<const void *>(&jacobi_kernel<2>);
    case 3: return reinterpret_cast<const void *>(&jacobi_kernel<3>);
    case 4: return reinterpret_cast<const void *>(&jacobi_kernel<4>);
    case 5: return reinterpret_cast<const void *>(&jacobi_kernel<5>);
    case 6: return reinterpret_cast<const void *>(&jacobi_kernel<6>);
    default: return reinterpret_cast<const void *>(&jacobi_kernel<8>);
    }
}

// Cooperative launches over groups of problems whose CTAs are co-resident:
// problem p's CTAs are [begin[p], begin[p] + grid_p).  The work records and
// the begin table go to the device (dev_recs: room for all problems).
template <typename Rec>
cudaError_t launch_groups(const void *kfn, int threads, int budget, const std::vector<int> &idx,
                          const std::vector<int> &grids, const std::vector<Rec> &recs,
                          Rec *dev_recs, int *dev_begin, cudaStream_t st, int *launches,
                          size_t smem = 0)
{
    size_t at = 0;
    while (at < idx.size()) {
        size_t end = at;
        int total = 0;
        while (end < idx.size() && (end == at || total + grids[idx[end]] <= budget))
            total += grids[idx[end++]];
        const int np = int(end - at);
        std::vector<Rec> r(np);
        std::vector<int> begin(np + 1, 0);
        for (int q = 0; q < np; ++q) {
            r[q] = recs[idx[at + q]];
            begin[q + 1] = begin[q] + grids[idx[at + q]];
        }
        Rec *dr = dev_recs + at;
        int *db = dev_begin + at;
        cudaMemcpyAsync(dr, r.data(), sizeof(Rec) * np, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(db, begin.data(), sizeof(int) * (np + 1), cudaMemcpyHostToDevice, st);
        const Rec *cdr = dr;
        const int *cdb = db;
        int cnp = np;
        void *args[] = {&cdr, &cdb, &cnp};
        cudaError_t e =
            cudaLaunchCooperativeKernel(kfn, dim3(total), dim3(threads), args, smem, st);
        ++*launches;
        if (e != cudaSuccess)
            return e;
        at = end;
    }
    return cudaSuccess;
}

// Whether a cluster of CL CTAs with smem bytes of dynamic shared memory each
// can be resident at all.
bool cluster_launchable(int CL, size_t smem)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(CL));
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = unsigned(CL);
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, svd_cluster_kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nc >= 1;
}

// Cluster size of the cluster kernel for an m x n worked matrix, or 0 when
// it does not fit (more than 256 columns, or more shared memory than a CTA
// may have).
int cluster_fit(const wos_context *ctx, int m, int n, int pre)
{
    if (n < 1 || n > kClMaxN)
        return 0;
    const int n_pad = std::max(2, n + (n & 1));
    const int CL = std::min(kClMaxCtas, n_pad / 2);
    const ClLayout L = cl_layout(m, n, pre, CL);
    if (L.PP > kClWarps || L.total > size_t(wos::ctx_max_smem(ctx)))
        return 0;
    // every launch may use up to the opt-in maximum (always the same value,
    // so that concurrent callers never see a smaller limit)
    cudaFuncSetAttribute(svd_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(svd_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         wos::ctx_max_smem(ctx));
    // the largest carveout, like the walk kernel, so either kernel finds
    // room on an SM the other one runs on
    cudaFuncSetAttribute(svd_cluster_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                         int(cudaSharedmemCarveoutMaxShared));
    return cluster_launchable(CL, L.total) ? CL : 0;
}

// The whole SVD pipeline for a batch of problems (one stream): per-problem
// small kernels, then the factorisations -- one cluster launch per cluster
// size for the problems that fit a cluster, batched cooperative QR and
// Jacobi launches for the others -- then the left vectors and the outputs.
wos_status svd_batch(wos_context *ctx, std::vector<SvdProb> &P, int32_t *sweeps,
                     cudaStream_t st, void *const *jacobi_events = nullptr)
{
    const int np = int(P.size());
    const int sms = wos::ctx_sm_count(ctx);
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    int qbps = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&qbps, qrcp_kernel, kQrThreads, 0);
    const int qbudget = std::max(1, qbps) * sms;
    // workspace layout
    std::vector<size_t> o_base(np);
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off += al(b); return o; };
    struct Off {
        size_t W, V, sv, bar, ver, g1, X, L, tau, perm, cn, cn0, done, pv, pi, qbar, W0, nrm;
        size_t J, J2, X32, G, bar32;
    };
    std::vector<Off> O(np);
    for (int p = 0; p < np; ++p) {
        SvdProb &b = P[p];
        SvdWork &w = b.w;
        w.m = b.transposed ? b.M_1 : b.M_D;
        w.n = b.transposed ? b.M_D : b.M_1;
        w.n_pad = std::max(2, w.n + (w.n & 1));
        b.pre = w.n >= kPrecondMinN;
        b.cl = wos::ctx_svd_path(ctx) == WOS_SVD_GRID ? 0 : cluster_fit(ctx, w.m, w.n, b.pre);
        b.lean = b.pre && !b.cl && w.n >= kLeanMinN;
        b.mixed = b.lean && wos::ctx_svd_path(ctx) != WOS_SVD_FP64_SWEEPS && pc32_fits(ctx, w.n);
        b.qgrid = b.pre ? std::max(1, std::min({w.n, 2 * sms, qbudget})) : 0;
        Off &o = O[p];
        o.W = take(size_t(w.m) * w.n * 8);
        o.V = take(size_t(w.n) * w.n * 8);
        o.sv = take(size_t(w.n) * 8);
        o.bar = take(64);
        o.ver = take(size_t(w.n_pad) * 4);
        o.g1 = take(size_t(b.M_1) * 4);
        if (b.pre) {
            o.X = take(size_t(w.n) * w.n * 8);
            o.L = take(size_t(w.m) * w.n * 8);
            o.tau = take(size_t(w.n) * 8);
            o.perm = take(size_t(w.n) * 4);
            o.cn = take(size_t(w.n) * 8);
            o.cn0 = take(size_t(w.n) * 8);
            o.done = take(size_t(w.n) * 4);
            o.pv = take(size_t(b.qgrid) * 2 * 8);
            o.pi = take(size_t(b.qgrid) * 2 * 4);
            o.qbar = take(64);
        }
        if (b.lean) {
            o.W0 = take(size_t(w.m) * w.n * 8);
            o.nrm = take(size_t(w.n) * 8 * 3);  // norms, scales, inverse scales
        }
        if (b.mixed) {
            const size_t nn = size_t(w.n) * w.n, b2 = 2 * size_t(pc32_b(w.n));
            o.J = take(nn * 8);
            o.J2 = take(nn * 8);
            o.X32 = take(nn * 4);
            const size_t C = size_t(pc32_ctas(w.n));
            o.G = take(size_t(kMaxSweeps32) * (2 * C - 1) * C * b2 * b2 * 4);
            o.bar32 = take(64);
        }
    }
    const size_t o_jrec = take(sizeof(SvdWork) * np), o_qrec = take(sizeof(QrWork) * np);
    const size_t o_pcrec = take(sizeof(Pc32Job) * np);
    const size_t o_gemm = take(sizeof(GemmJob) * np);
    const size_t o_rprec = take(sizeof(Pc32Job) * np + sizeof(int) * (np + 1));
    const size_t o_left = take(sizeof(LeftJob) * np);
    const size_t o_cjob = take(sizeof(ClusterJob) * np);
    const size_t o_begin = take(sizeof(int) * (3 * np + 4));
    char *base = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&base), off, st);
    if (e != cudaSuccess)
        return wos::cuda_status(e);
    int launches = 0;
    std::vector<SvdWork> jrecs(np);
    std::vector<QrWork> qrecs(np);
    std::vector<int> qidx, pidx, jgrids(np, 0), qgrids(np, 0);
    std::vector<ClusterJob> cjobs(np);
    for (int p = 0; p < np; ++p) {
        SvdProb &b = P[p];
        const Off &o = O[p];
        SvdWork &w = b.w;
        w.W = reinterpret_cast<double *>(base + o.W);
        w.Vw = reinterpret_cast<double *>(base + o.V);
        w.bar = reinterpret_cast<unsigned *>(base + o.bar);
        w.ver = reinterpret_cast<unsigned *>(base + o.ver);
        b.sv = reinterpret_cast<double *>(base + o.sv);
        b.g1 = reinterpret_cast<int *>(base + o.g1);
        cudaMemsetAsync(w.bar, 0, 64, st);
        cudaMemsetAsync(w.ver, 0, al(size_t(w.n_pad) * 4), st);
        cudaMemcpyAsync(b.g1, b.L.g1.data(), size_t(b.M_1) * 4, cudaMemcpyHostToDevice, st);
        form_B_kernel<<<sms * 4, 256, 0, st>>>(w, b.counts, b.M_D, b.M_tot, 1.0 / double(b.N),
                                              b.g1, b.M_1, b.nu, b.sigma, b.transposed);
        ++launches;
        b.W0 = nullptr;
        b.X0 = nullptr;
        if (b.lean) {
            b.W0 = reinterpret_cast<double *>(base + o.W0);
            cudaMemcpyAsync(b.W0, w.W, size_t(w.m) * w.n * 8, cudaMemcpyDeviceToDevice, st);
        }
        b.wj = w;
        b.wj.nrm = b.lean ? reinterpret_cast<double *>(base + o.nrm) : nullptr;
        b.wj.dsc = b.lean ? b.wj.nrm + w.n : nullptr;
        b.wj.dinv = b.lean ? b.wj.nrm + 2 * size_t(w.n) : nullptr;
        if (b.pre) {
            QrWork &q = b.q;
            q.A = w.W;
            q.m = w.m;
            q.n = w.n;
            q.tau = reinterpret_cast<double *>(base + o.tau);
            q.perm = reinterpret_cast<int *>(base + o.perm);
            q.cn = reinterpret_cast<double *>(base + o.cn);
            q.cn0 = reinterpret_cast<double *>(base + o.cn0);
            q.done = reinterpret_cast<int *>(base + o.done);
            q.pval = reinterpret_cast<double *>(base + o.pv);
            q.pidx = reinterpret_cast<int *>(base + o.pi);
            q.bar = reinterpret_cast<unsigned *>(base + o.qbar);
            cudaMemsetAsync(q.done, 0, size_t(w.n) * 4, st);
            cudaMemsetAsync(q.bar, 0, 64, st);
            b.wj.W = reinterpret_cast<double *>(base + o.X);
            b.wj.m = w.n;
            b.Lb = reinterpret_cast<double *>(base + o.L);
            if (b.mixed) {  // X = R^T to X0; the FP64 sweeps work on X Q in J2's place
                b.X0 = b.wj.W;
                b.wj.W = reinterpret_cast<double *>(base + o.J2);
                Pc32Job &v = b.pc;
                v.X = reinterpret_cast<float *>(base + o.X32);
                v.G = reinterpret_cast<float *>(base + o.G);
                v.bar = reinterpret_cast<unsigned *>(base + o.bar32);
                v.J = reinterpret_cast<double *>(base + o.J);
                v.m = w.n;
                v.n = w.n;
                v.b = pc32_b(w.n);
                v.C = pc32_ctas(w.n);
                v.ms = pc32_ms(w.n);
                cudaMemsetAsync(v.bar, 0, 64, st);
            }
            qrecs[p] = q;
            qgrids[p] = b.qgrid;
            pidx.push_back(p);
            if (!b.cl)
                qidx.push_back(p);
        }
        jrecs[p] = b.wj;
        if (b.cl) {
            ClusterJob &J = cjobs[p];
            J.A = w.W;
            J.m = w.m;
            J.n = w.n;
            J.pre = b.pre ? 1 : 0;
            J.tau = b.pre ? b.q.tau : nullptr;
            J.perm = b.pre ? b.q.perm : nullptr;
            J.X = b.wj.W;
            J.V = b.wj.Vw;
            J.bar = w.bar;
        }
    }
    QrWork *dq = reinterpret_cast<QrWork *>(base + o_qrec);
    SvdWork *dj = reinterpret_cast<SvdWork *>(base + o_jrec);
    int *dbegin = reinterpret_cast<int *>(base + o_begin);
    {
        long long want = 0;
        for (int p : qidx)
            want += qgrids[p];
        if (want > qbudget)
            for (int p : qidx)
                qgrids[p] = std::max(1, int(qgrids[p] * (long long)qbudget / want));
    }
    if (jacobi_events && jacobi_events[0])
        cudaEventRecord(static_cast<cudaEvent_t>(jacobi_events[0]), st);
    // cluster kernel: one launch per cluster size, one cluster per problem
    size_t cjobs_used = 0;
    for (int CL = 1; e == cudaSuccess && CL <= kClMaxCtas; ++CL) {
        std::vector<ClusterJob> jobs;
        size_t smem = 0;
        int pp = 1;
        for (int p = 0; p < np; ++p)
            if (P[p].cl == CL) {
                jobs.push_back(cjobs[p]);
                const ClLayout L = cl_layout(P[p].w.m, P[p].w.n, P[p].pre, CL);
                smem = std::max(smem, L.total);
                pp = std::max(pp, L.PP);
            }
        if (jobs.empty())
            continue;
        ClusterJob *dj2 = reinterpret_cast<ClusterJob *>(base + o_cjob) + cjobs_used;
        cjobs_used += jobs.size();
        cudaMemcpyAsync(dj2, jobs.data(), sizeof(ClusterJob) * jobs.size(),
                        cudaMemcpyHostToDevice, st);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(unsigned(CL * int(jobs.size())));
        // a warp per pair of a round, at least four (the QR's two scalar
        // warps and the column warps); fewer threads leave room on the SMs
        // for other work (the next walk launch) beside the cluster
        cfg.blockDim = dim3(pp <= 4 ? 128u : unsigned(kClThreads));
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = unsigned(CL);
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, svd_cluster_kernel, const_cast<const ClusterJob *>(dj2), CL);
        ++launches;
    }
    {
        // the FP32-preconditioned problems: column order by norm, QR without
        // pivoting; the others: QR with column pivoting
        std::vector<int> piv, srt;
        for (int p : qidx)
            (P[p].mixed ? srt : piv).push_back(p);
        for (int p = 0; e == cudaSuccess && p < int(srt.size()); ++p) {
            const QrWork &q = P[srt[p]].q;
            qr_col_norms_kernel<<<sms * 2, 256, 0, st>>>(q);
            sort_columns_kernel<<<(q.n + 255) / 256, 256, size_t(q.n) * sizeof(double), st>>>(q);
            launches += 2;
        }
        if (e == cudaSuccess && !srt.empty()) {
            int sbps = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sbps, qrs_kernel, kQrsThreads, 0);
            const int sbudget = std::max(1, sbps) * sms;
            std::vector<int> sgrids(qgrids);  // the problems' CTAs within this kernel's budget
            long long want = 0;
            for (int p : srt)
                want += sgrids[p];
            if (want > sbudget)
                for (int p : srt)
                    sgrids[p] = std::max(1, int(sgrids[p] * (long long)sbudget / want));
            e = launch_groups(reinterpret_cast<const void *>(qrs_kernel), kQrsThreads, sbudget,
                              srt, sgrids, qrecs, dq, dbegin, st, &launches);
        }
        if (e == cudaSuccess && !piv.empty())
            e = launch_groups(reinterpret_cast<const void *>(qrcp_kernel), kQrThreads, qbudget,
                              piv, qgrids, qrecs, dq + srt.size(), dbegin + srt.size() + 1, st,
                              &launches);
    }
    for (int p = 0; e == cudaSuccess && p < np; ++p)
        if (P[p].pre && !P[p].cl) {
            SvdProb &b = P[p];
            build_x_kernel<<<sms * 4, 256, 0, st>>>(b.q, b.mixed ? b.X0 : b.wj.W, b.wj.Vw);
            ++launches;
            if (b.mixed) {
                to32_kernel<<<sms * 4, 256, 0, st>>>(b.X0, size_t(b.pc.m) * b.pc.n, b.pc.X);
                ++launches;
            } else if (b.lean) {  // the squared column norms the lean sweeps carry
                column_sq_norms_kernel<<<sms * 2, 256, 0, st>>>(b.wj);
                ++launches;
            }
        }
    // FP32 preconditioning sweeps: cooperative launches of the problems'
    // CTAs, one per block width; then J from each problem's G products
    {
        std::vector<Pc32Job> recs(np);
        for (int p = 0; p < np; ++p)
            if (P[p].mixed)
                recs[p] = P[p].pc;
        const void *sk = reinterpret_cast<const void *>(&pc32_sweeps_kernel);
        for (int bw = 4; e == cudaSuccess && bw <= kPc32MaxB; bw += 4) {
            std::vector<int> idx;
            std::vector<int> grids(np, 0);
            int nmax = 0;
            for (int p = 0; p < np; ++p)
                if (P[p].mixed && P[p].pc.b == bw) {
                    idx.push_back(p);
                    grids[p] = P[p].pc.C;
                    nmax = std::max(nmax, P[p].pc.n);
                }
            if (idx.empty())
                continue;
            const size_t smem = pc32_smem(nmax);
            int bps = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, sk, 32 * bw, smem);
            e = launch_groups(sk, 32 * bw, std::max(1, bps) * sms, idx, grids, recs,
                              reinterpret_cast<Pc32Job *>(base + o_pcrec), dbegin + 2 * np + 3,
                              st, &launches, smem);
        }
    }
    if (e == cudaSuccess) {  // every problem's J in one launch
        std::vector<Pc32Job> jobs;
        std::vector<int> begin(1, 0);
        size_t smem = 0;
        for (int p = 0; p < np; ++p)
            if (P[p].mixed) {
                jobs.push_back(P[p].pc);
                begin.push_back(begin.back() + (P[p].pc.n + kRpRows - 1) / kRpRows);
                smem = std::max(smem, pc32_replay_smem(P[p].pc.n));
            }
        if (!jobs.empty()) {
            Pc32Job *dj3 = reinterpret_cast<Pc32Job *>(base + o_rprec);
            int *db3 = reinterpret_cast<int *>(dj3 + np);
            cudaMemcpyAsync(dj3, jobs.data(), sizeof(Pc32Job) * jobs.size(),
                            cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(db3, begin.data(), sizeof(int) * begin.size(), cudaMemcpyHostToDevice,
                            st);
            pc32_replay_kernel<<<begin.back(), 256, smem, st>>>(dj3, db3, int(jobs.size()));
            ++launches;
        }
    }
    // two Newton-Schulz steps Q <- Q - Q (Q^T Q - I) / 2 from Q = J, then the
    // FP64 sweeps' start X Q: Q^T Q in FP64 (its departure from I, about
    // 1e-4 and then 1e-8, must be exact to FP64 rounding), the correction
    // products in FP32 (their rounding, scaled by that departure, leaves Q
    // orthogonal to about 1e-15), X Q in FP64 (a right-multiplicative
    // rounding: relative accuracy kept).  M sits in V's place (free until
    // the left vectors); J2 holds Q after one step, then X Q.
    {
        std::vector<GemmJob> s1, c1, s2, c2, xq;
        for (int p = 0; p < np; ++p)
            if (P[p].mixed) {
                SvdProb &b = P[p];
                const int n = b.w.n;
                double *J = b.pc.J, *J2 = b.wj.W, *M = b.wj.Vw;
                s1.push_back(gemm_syrk(n, n, J, M));             // M = J^T J
                c1.push_back(gemm_ns(n, J, M, J, J2));           // J2 = J - J (M - I) / 2
                s2.push_back(gemm_syrk(n, n, J2, M));            // M = J2^T J2
                c2.push_back(gemm_ns(n, J2, M, J2, J));          // Q = J2 - J2 (M - I) / 2
                xq.push_back(gemm_nn(n, n, n, b.X0, J, J2));     // X Q
            }
        GemmJob *dg = reinterpret_cast<GemmJob *>(base + o_gemm);
        if (e == cudaSuccess) e = gemm_batch(st, kGemmSyrk, s1, dg, &launches);
        if (e == cudaSuccess) e = gemm_batch(st, kGemmNsCorrection, c1, dg, &launches);
        if (e == cudaSuccess) e = gemm_batch(st, kGemmSyrk, s2, dg, &launches);
        if (e == cudaSuccess) e = gemm_batch(st, kGemmNsCorrection, c2, dg, &launches);
        if (e == cudaSuccess) e = gemm_batch(st, kGemmNN, xq, dg, &launches);
        for (int p = 0; e == cudaSuccess && p < np; ++p)
            if (P[p].mixed) {
                column_sq_norms_kernel<<<sms * 2, 256, 0, st>>>(P[p].wj);
                ++launches;
            }
    }
    // Jacobi: one cooperative launch per class of rows per thread (and per
    // group of co-resident problems); the CTAs are shared in proportion to
    // the pairs when the batch is larger than the GPU
    // Without V: four pairs per CTA when the batch has pairs for more than
    // three CTAs of one pair per SM and its sweeps are FP64 ones alone (ten
    // or so sweeps: the FP64 units bound them), else a CTA per pair (a lone
    // problem, or the two or three sweeps after FP32 ones: the round's
    // critical path bounds them)
    long long lean_pairs = 0;
    bool any_mixed = false;
    for (int p = 0; p < np; ++p)
        if (P[p].lean) {
            lean_pairs += P[p].wj.n_pad / 2;
            any_mixed = any_mixed || P[p].mixed;
        }
    const bool grouped = !any_mixed && lean_pairs > 3LL * sms;
    for (int cls = 0; cls < 11; ++cls) {
        if (e != cudaSuccess)
            break;
        static const int kRpts[7] = {1, 2, 3, 4, 5, 6, 8};
        static const int kRpls[4] = {8, 16, 24, 32};
        // classes: 0-6 with V (rows per thread), 7-10 without V (rows per
        // lane of the canonical order): grouped or a CTA per pair
        const bool lean = cls >= 7;
        const bool group = lean && grouped;
        const int rpt = lean ? kRpls[cls - 7] : kRpts[cls];
        std::vector<int> idx;
        for (int p = 0; p < np; ++p)
            if (!P[p].cl && P[p].lean == lean &&
                (lean ? rpl_of(P[p].wj.m) : rpt_of(P[p].wj.m)) == rpt)
                idx.push_back(p);
        if (idx.empty())
            continue;
        long long cls_pairs = 0;
        for (int p : idx)
            cls_pairs += P[p].wj.n_pad / 2;
        const bool dense = lean && !group && cls_pairs > 10LL * sms;
        const void *jk = group ? jacobi_group_kernel_rpl(rpt)
                               : lean ? jacobi_lean_kernel_rpl(rpt, dense) : jacobi_kernel_rpt(rpt);
        const int threads = group ? kGroupThreads : kPairThreads;
        int bps = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, jk, threads, 0);
        const int budget = std::max(1, bps) * sms;
        long long want = 0;
        for (int p : idx) {
            // a CTA per pair (per four pairs without V) if they fit
            const int half = P[p].wj.n_pad / 2;
            jgrids[p] = std::min(group ? (half + kGroupPairs - 1) / kGroupPairs : half, budget);
            want += jgrids[p];
        }
        if (want > budget)
            for (int p : idx)
                jgrids[p] = std::max(1, int(jgrids[p] * (long long)budget / want));
        e = launch_groups(jk, threads, budget, idx, jgrids, jrecs, dj, dbegin + np + 2, st,
                          &launches);
    }
    if (jacobi_events && jacobi_events[1])
        cudaEventRecord(static_cast<cudaEvent_t>(jacobi_events[1]), st);
    // left vectors without V: L = W P X_final (an FP64 GEMM of the saved W
    // with the row-permuted final X; its columns are sigma^2 times the unit
    // left vectors, scaled in finalize)
    {
        std::vector<GemmJob> lv;
        for (int p = 0; e == cudaSuccess && p < np; ++p)
            if (P[p].lean) {
                SvdProb &b = P[p];
                const int m = b.w.m, n = b.w.n;
                fold_scales_kernel<<<sms * 4, 256, 0, st>>>(b.wj);  // X = d_j xt_j
                permute_rows_kernel<<<sms * 4, 256, 0, st>>>(b.wj.W, b.q.perm, n, b.wj.Vw);
                launches += 2;
                lv.push_back(gemm_nn(m, n, n, b.W0, b.wj.Vw, b.Lb));
            }
        if (e == cudaSuccess)
            e = gemm_batch(st, kGemmNN, lv, reinterpret_cast<GemmJob *>(base + o_gemm), &launches);
    }
    if (e == cudaSuccess) {  // left vectors of every other preconditioned problem
        std::vector<LeftJob> jobs;
        int ncols = 0;
        for (int p : pidx) {
            if (P[p].lean)
                continue;
            jobs.push_back(LeftJob{P[p].q, P[p].wj.Vw, P[p].Lb, ncols});
            ncols += P[p].w.n;
        }
        if (!jobs.empty()) {
            LeftJob *dl = reinterpret_cast<LeftJob *>(base + o_left);
            cudaMemcpyAsync(dl, jobs.data(), sizeof(LeftJob) * jobs.size(),
                            cudaMemcpyHostToDevice, st);
            // two warps (columns) per block: the columns spread over the SMs'
            // sub-partitions (each warp's dependent FP64 chain of n reflectors
            // holds its sub-partition's FP64 unit; two per SM would queue)
            form_left_kernel<<<std::max(1, std::min((ncols + 1) / 2, sms * 16)), 64, 0, st>>>(
                dl, int(jobs.size()), ncols);
            ++launches;
        }
    }
    for (int p = 0; e == cudaSuccess && p < np; ++p) {
        SvdProb &b = P[p];
        column_norms_kernel<<<sms, 256, 0, st>>>(b.wj, b.sv);
        if (b.pre)
            finalize_pre_kernel<<<sms, 256, 0, st>>>(b.Lb, b.wj.W, b.q.perm, b.sv, b.w.m, b.w.n,
                                                     b.transposed, b.lean ? 1 : 0, b.U, b.S,
                                                     b.V);
        else
            finalize_kernel<<<sms, 256, 0, st>>>(b.w, b.sv, b.transposed, b.U, b.S, b.V);
        launches += 2;
    }
    if (e == cudaSuccess)
        e = cudaGetLastError();
    wos::count_launches(ctx, launches);
    wos_status status = wos::cuda_status(e);
    if (status == WOS_OK && sweeps) {
        std::vector<unsigned> hb(size_t(np) * 14, 0u);
        for (int p = 0; p < np; ++p) {
            cudaMemcpyAsync(hb.data() + p * 14, P[p].w.bar, 7 * 4, cudaMemcpyDeviceToHost, st);
            if (P[p].pre)
                cudaMemcpyAsync(hb.data() + p * 14 + 7, P[p].q.bar, 7 * 4, cudaMemcpyDeviceToHost,
                                st);
            if (P[p].mixed)  // the FP32 sweeps' barrier status in place of q.bar[6]
                cudaMemcpyAsync(hb.data() + p * 14 + 13, P[p].pc.bar + 5, 4,
                                cudaMemcpyDeviceToHost, st);
        }
        e = cudaStreamSynchronize(st);
        status = wos::cuda_status(e);
        for (int p = 0; p < np; ++p) {
            sweeps[p] = int32_t(hb[p * 14 + 6]);
            if (status == WOS_OK && hb[p * 14 + 7 + 5] != 0u)
                status = wos_status(hb[p * 14 + 7 + 5]);
            if (status == WOS_OK && hb[p * 14 + 5] != 0u)
                status = wos_status(hb[p * 14 + 5]);
            if (status == WOS_OK && P[p].mixed && hb[p * 14 + 13] != 0u)
                status = wos_status(hb[p * 14 + 13]);
        }
    }
    cudaFreeAsync(base, st);
    return status;
}

wos_status svd_prob(const wos_svd_problem &in, SvdProb *b)
{
    if (!in.counts || !in.gamma1 || !in.sigma || !in.U || !in.S || !in.V || in.M_D < 1 ||
        in.M_tot < 1 || in.N < 1)
        return WOS_INVALID_ARG;
    b->counts = in.counts;
    b->M_D = in.M_D;
    b->M_tot = in.M_tot;
    b->N = in.N;
    b->nu = in.nu;
    b->sigma = in.sigma;
    b->U = in.U;
    b->S = in.S;
    b->V = in.V;
    b->L = split(in.gamma1, in.M_tot);
    b->M_1 = int(b->L.g1.size());
    if (b->M_1 < 1)
        return WOS_INVALID_ARG;
    b->transposed = b->M_D < b->M_1;
    return WOS_OK;
}

}  // namespace

extern "C" wos_status wos_op_svd(wos_context *ctx, const uint32_t *counts, int32_t M_D,
                                 int32_t M_tot, uint32_t N, const uint8_t *gamma1,
                                 const double *nu, const double *sigma, double *U,
                                 double *S, double *V, int32_t *sweeps, void *stream)
{
    if (!ctx)
        return WOS_INVALID_ARG;
    wos_svd_problem in = {counts, M_D, M_tot, N, gamma1, nu, sigma, U, S, V};
    std::vector<SvdProb> P(1);
    wos_status st = svd_prob(in, &P[0]);
    if (st != WOS_OK)
        return st;
    cudaSetDevice(wos::ctx_device(ctx));
    return svd_batch(ctx, P, sweeps, static_cast<cudaStream_t>(stream));
}

extern "C" wos_status wos_op_svd_batched(wos_context *ctx, int32_t n,
                                         const wos_svd_problem *problems, int32_t *sweeps,
                                         void *stream, void *const *jacobi_events)
{
    if (!ctx || n < 1 || !problems)
        return WOS_INVALID_ARG;
    std::vector<SvdProb> P(n);
    for (int q = 0; q < n; ++q) {
        wos_status st = svd_prob(problems[q], &P[q]);
        if (st != WOS_OK)
            return st;
    }
    cudaSetDevice(wos::ctx_device(ctx));
    return svd_batch(ctx, P, sweeps, static_cast<cudaStream_t>(stream), jacobi_events);
}

extern "C" wos_status wos_reconstruct(wos_context *ctx, const double *U, const double *S,
                                      const double *V, int32_t M_D, int32_t k,
                                      const uint32_t *counts, int32_t M_tot, uint32_t N,
                                      const uint8_t *gamma1, const double *nu,
                                      const double *sigma, const double *uD,
                                      const double *u0, int32_t r, double tikhonov_alpha,
                                      double *u_gamma1, double *uD_hat, void *stream)
{
    if (!ctx || !U || !S || !V || !counts || !gamma1 || !sigma || !uD || !u_gamma1 ||
        M_D < 1 || M_tot < 1 || N < 1 || k < 1 || r < 1 || r > k || tikhonov_alpha < 0)
        return WOS_INVALID_ARG;
    cudaSetDevice(wos::ctx_device(ctx));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Lists L = split(gamma1, M_tot);
    const int M_1 = int(L.g1.size()), M_0 = int(L.g0.size());
    if (M_1 < 1 || k > std::min(M_D, M_1))
        return WOS_INVALID_ARG;
    // scratch: f (M_tot), b (M_D), t (k), index lists
    size_t bytes = size_t(M_tot) * 8 + size_t(M_D) * 8 + size_t(k) * 8 +
                   size_t(M_tot) * 4 + 64;
    char *base = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&base), bytes, st);
    if (e != cudaSuccess)
        return wos::cuda_status(e);
    double *f = reinterpret_cast<double *>(base);
    double *b = f + M_tot;
    double *t = b + M_D;
    int *g1 = reinterpret_cast<int *>(t + k);
    int *g0 = g1 + M_1;
    cudaMemcpyAsync(g1, L.g1.data(), size_t(M_1) * 4, cudaMemcpyHostToDevice, st);
    if (M_0)
        cudaMemcpyAsync(g0, L.g0.data(), size_t(M_0) * 4, cudaMemcpyHostToDevice, st);
    int sms = wos::ctx_sm_count(ctx);
    const double invN = 1.0 / double(N);
    // b = uD - A u0full (u0full: u0 on Gamma_0, 0 on Gamma_1)
    cudaMemsetAsync(f, 0, size_t(M_tot) * 8, st);
    if (u0 && M_0)
        scatter_kernel<<<sms, 256, 0, st>>>(g0, M_0, u0, f);
    counts_matvec_kernel<<<sms * 2, 256, 0, st>>>(counts, M_D, M_tot, invN, f, uD, -1.0, b);
    tsvd_t_kernel<<<std::max(1, (r + 7) / 8), 256, 0, st>>>(U, S, M_D, k, r, nu, b,
                                                            tikhonov_alpha, t);
    tsvd_u_kernel<<<std::max(1, (M_1 + 255) / 256), 256, 0, st>>>(V, M_1, k, r, t, g1,
                                                                  sigma, u_gamma1);
    if (uD_hat) {
        scatter_kernel<<<sms, 256, 0, st>>>(g1, M_1, u_gamma1, f);
        counts_matvec_kernel<<<sms * 2, 256, 0, st>>>(counts, M_D, M_tot, invN, f, nullptr,
                                                      1.0, uD_hat);
    }
    wos::count_launches(ctx, 3 + ((u0 && M_0) ? 1 : 0) + (uD_hat ? 2 : 0));
    e = cudaGetLastError();
    cudaFreeAsync(base, st);
    return wos::cuda_status(e);
}
