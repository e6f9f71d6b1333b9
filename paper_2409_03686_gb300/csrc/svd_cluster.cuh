// svd_cluster.cuh -- the SVD of one small operator inside one thread-block
// cluster (included by wos_svd.cu after SvdWork, QrWork and the Jacobi
// helpers).
//
// Same mathematics as the grid-wide kernels of wos_svd.cu (Householder QR
// with column pivoting, Drmac & Veselic's preconditioning, one-sided
// Jacobi in the round-robin order with the relative rotation test and the
// early stop after a sweep of tiny angles), but the whole factorisation
// lives in the distributed shared memory of a cluster of up to 16 CTAs (one
// SM each): columns move between CTAs with shared::cluster stores and the
// rounds are ordered by hardware cluster barriers, so a round costs shared-
// memory latencies instead of L2 round trips, a release fence and flag
// polling.  Used when the worked matrix fits (n <= 256 columns).
//
//  * QR (preconditioned path): CTA c owns the physical columns j = c (mod
//    CL).  Per pivot k every CTA pushes its largest remaining squared norm to
//    every CTA (double buffered by pivot parity), one cluster barrier, every
//    CTA takes the same argmax pc (lowest index on ties), reads column pc from
//    its owner and forms the same reflector (xLARFG's beta, tau, v) in the
//    same arithmetic order; it then applies it to its own columns (one warp
//    per column) and downdates their norms (xLAQP2's test).  The owner writes
//    the reflector into column pc only after the next barrier, when nobody
//    reads the raw column any more.
//  * X = R^T goes to the Jacobi buffers: column i of X (row i of R) starts at
//    round-robin position i.
//  * Jacobi: one warp per pair; CTA c holds the pairs [c PP, (c + 1) PP) of
//    the round, each pair's two columns (X and V_X rows) in a slot of a
//    double-buffered array.  After rotating, the warp stores each column into
//    the slot of the position it takes in the next round (the circle method
//    moves every column but the first by one position), then the cluster
//    barrier.  Sweep statistics (rotations, and whether a rotated pair had
//    cos^2 > kLast^2: a comparison, no division on the FP64 pipe, which a
//    warp instruction occupies for 64 cycles whatever its active lanes) are
//    stored by every warp in its own CTA and read by every warp of the
//    cluster after the sweep's last barrier.
#pragma once

#include <cooperative_groups.h>

#include "svd_cluster_layout.h"

namespace cg = cooperative_groups;

struct ClusterJob {
    double *A;       // m x n column-major: W on entry; (pre) R and reflectors
    int m, n;        // worked orientation, m >= n
    int pre;         // 1: QR with pivoting, Jacobi on X = R^T
    double *tau;     // n reflector scalars (pre)
    int *perm;       // n: physical column of pivot k (pre)
    double *X;       // out: final columns of the matrix Jacobi worked on
                     // (n x n when pre, else m x n; may alias A when not pre)
    double *V;       // out: n x n accumulated rotations
    unsigned *bar;   // [5] status, [6] sweeps
};

// 64 registers a thread (8 bytes of spill): a 128-thread CTA then needs 8 K
// registers and fits on an SM beside four 56-register walk blocks.
__global__ void __maxnreg__(64)
svd_cluster_kernel(const ClusterJob *jobs, int CL)
{
    cg::cluster_group cluster = cg::this_cluster();
    const ClusterJob J = jobs[blockIdx.x / CL];
    const int c = int(cluster.block_rank());
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = int(blockDim.x), nw = T >> 5;  // 128 or 256 threads
    const int m = J.m, n = J.n, pre = J.pre;
    const ClLayout L = cl_layout(m, n, pre, CL);
    extern __shared__ __align__(16) unsigned char cl_smem[];
    unsigned char *sp = cl_smem;
    auto carve = [&](size_t b) { unsigned char *r = sp; sp += cl_align(b); return r; };
    double *pub_val = reinterpret_cast<double *>(carve(2 * 16 * 8));
    int *pub_idx = reinterpret_cast<int *>(carve(2 * 16 * 4));
    double *tau_all = reinterpret_cast<double *>(carve(size_t(n) * 8));
    int *perm_all = reinterpret_cast<int *>(carve(size_t(n) * 4));
    double *cn = reinterpret_cast<double *>(carve(size_t(L.cpc) * 8));
    double *cn0 = reinterpret_cast<double *>(carve(size_t(L.cpc) * 8));
    int *cflag = reinterpret_cast<int *>(carve(size_t(L.cpc) * 4));
    unsigned *swstat = reinterpret_cast<unsigned *>(carve(2 * kClWarps * 4));
    double *red = reinterpret_cast<double *>(carve(64 * 8));
    sp = cl_smem + L.small;
    double *qcol = reinterpret_cast<double *>(sp);
    double *vbuf = reinterpret_cast<double *>(sp + L.qcol);
    double *jb = reinterpret_cast<double *>(sp + L.qcol + L.vbuf);
    const int slot_len = L.nX + n;
    const size_t buf_len = size_t(2) * L.PP * slot_len;

    // ---- QR with column pivoting ------------------------------------------
    if (pre) {
        const int nown = c < n ? (n - c + CL - 1) / CL : 0;
        for (int t = warp; t < nown; t += nw) {
            const double *g = J.A + size_t(c + t * CL) * m;
            double *col = qcol + size_t(t) * m;
            double s = 0.0;
            for (int i = lane; i < m; i += 32) {
                const double v = g[i];
                col[i] = v;
                s = fma(v, v, s);
            }
            s = warp_sum(s);
            if (lane == 0) {
                cn[t] = s;
                cn0[t] = s;
                cflag[t] = 0;
            }
        }
        __syncthreads();
        int pend_t = -1, pend_k = 0;  // owner's reflector still to be stored
        double pend_beta = 0.0;
        for (int k = 0; k < n; ++k) {
            // push this CTA's largest remaining norm to every CTA
            if (tid < CL) {
                double bv = -1.0;
                int bi = -1;
                for (int t = 0; t < nown; ++t)
                    if (cflag[t] == 0 && cn[t] > bv) {
                        bv = cn[t];
                        bi = c + t * CL;
                    }
                double *rv = cluster.map_shared_rank(pub_val, tid);
                int *ri = cluster.map_shared_rank(pub_idx, tid);
                rv[(k & 1) * 16 + c] = bv;
                ri[(k & 1) * 16 + c] = bi;
            }
            cluster.sync();
            if (pend_t >= 0) {  // the previous pivot's reflector, now unread
                double *col = qcol + size_t(pend_t) * m;
                for (int i = pend_k + 1 + tid; i < m; i += T)
                    col[i] = vbuf[i];
                if (tid == 0)
                    col[pend_k] = pend_beta;
                pend_t = -1;
                __syncthreads();
            }
            // the same argmax in every CTA (largest norm, lowest column on ties)
            double bv = -1.0;
            int pc = 0x7fffffff;
            if (lane < CL) {
                const int i = pub_idx[(k & 1) * 16 + lane];
                const double v = pub_val[(k & 1) * 16 + lane];
                if (i >= 0) {
                    bv = v;
                    pc = i;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(FULL, bv, o);
                const int oi = __shfl_xor_sync(FULL, pc, o);
                if (ov > bv || (ov == bv && oi < pc)) {
                    bv = ov;
                    pc = oi;
                }
            }
            if (pc < 0 || pc >= n)
                pc = 0;  // unreachable: n - k columns remain
            const int owner = pc % CL, tp = pc / CL;
            const double *src = cluster.map_shared_rank(qcol + size_t(tp) * m, owner);
            for (int i = k + tid; i < m; i += T)
                vbuf[i] = src[i];
            __syncthreads();
            // reflector of rows k..m-1 (xLARFG), identical in every CTA.  A
            // warp instruction holds the FP64 pipe of its SM sub-partition
            // for 64 cycles whatever its active lanes, so the scalars are
            // formed by two warps (on two sub-partitions: warp 0 tau, warp 1
            // the scale), not by every thread.
            if (warp < 2) {
                double xn2 = 0.0;
                for (int i = k + 1 + lane; i < m; i += 32)
                    xn2 = fma(vbuf[i], vbuf[i], xn2);
                xn2 = warp_sum(xn2);
                const double alpha = vbuf[k];
                double tau = 0.0, beta = alpha, scal = 1.0;
                if (xn2 > 0.0) {
                    beta = -copysign(sqrt(fma(alpha, alpha, xn2)), alpha);
                    if (warp == 0)
                        tau = (beta - alpha) / beta;
                    else
                        scal = 1.0 / (alpha - beta);
                }
                if (lane == 0) {
                    if (warp == 0) {
                        red[0] = tau;
                        red[1] = beta;
                    } else {
                        red[2] = scal;
                    }
                }
            }
            __syncthreads();
            const double tau = red[0], beta = red[1], scal = red[2];
            if (tau != 0.0)
                for (int i = k + 1 + tid; i < m; i += T)
                    vbuf[i] *= scal;
            if (tid == 0) {
                tau_all[k] = tau;
                perm_all[k] = pc;
            }
            if (owner == c) {
                if (tid == 0)
                    cflag[tp] = k + 1;  // pivot k + 1 (>= 1: done)
                pend_t = tp;
                pend_k = k;
                pend_beta = beta;
            }
            __syncthreads();
            // apply H_k = I - tau v v^T (v_k = 1) to the remaining own columns
            for (int t = warp; t < nown; t += nw) {
                if (cflag[t] != 0)
                    continue;
                double *col = qcol + size_t(t) * m;
                if (tau != 0.0) {
                    double w = 0.0;
                    for (int i = k + 1 + lane; i < m; i += 32)
                        w = fma(vbuf[i], col[i], w);
                    w = warp_sum(w) + col[k];
                    const double tw = tau * w;
                    for (int i = k + 1 + lane; i < m; i += 32)
                        col[i] = fma(-tw, vbuf[i], col[i]);
                    __syncwarp();
                    if (lane == 0)
                        col[k] -= tw;
                    __syncwarp();
                }
                // norm of rows k+1..m-1: downdate |x|^2 - r^2, or recompute
                // when cancellation has eaten half the digits (xLAQP2's test
                // (1 - r^2/|x|^2) |x|^2 / |x_0|^2 <= tol3z, multiplied out:
                // no division on the FP64 pipe)
                const double r = col[k], cv = cn[t];
                double f = 0.0;
                bool recompute = false;
                if (cv > 0.0) {
                    f = fmax(fma(-r, r, cv), 0.0);
                    recompute = f <= kTol3z * cn0[t];
                }
                if (recompute) {
                    double s = 0.0;
                    for (int i = k + 1 + lane; i < m; i += 32)
                        s = fma(col[i], col[i], s);
                    s = warp_sum(s);
                    if (lane == 0) {
                        cn[t] = s;
                        cn0[t] = s;
                    }
                } else if (lane == 0) {
                    cn[t] = f;
                }
                __syncwarp();
            }
            __syncthreads();
        }
        cluster.sync();
        if (pend_t >= 0) {
            double *col = qcol + size_t(pend_t) * m;
            for (int i = pend_k + 1 + tid; i < m; i += T)
                col[i] = vbuf[i];
            if (tid == 0)
                col[pend_k] = pend_beta;
        }
        __syncthreads();
        // factors out (R and reflectors in place, tau, perm)
        for (int t = warp; t < nown; t += nw) {
            double *g = J.A + size_t(c + t * CL) * m;
            const double *col = qcol + size_t(t) * m;
            for (int i = lane; i < m; i += 32)
                g[i] = col[i];
        }
        if (c == 0)
            for (int k = tid; k < n; k += T) {
                J.tau[k] = tau_all[k];
                J.perm[k] = perm_all[k];
            }
        // X = R^T into buffer 0: own column j (pivot kj) is row kj of X's
        // columns: X[kj][i] = R[i][kj] = A[i][j] for i <= kj, else 0
        for (int t = warp; t < nown; t += nw) {
            const int kj = cflag[t] - 1;
            const double *col = qcol + size_t(t) * m;
            for (int i = lane; i < n; i += 32) {
                int cta, slot;
                cl_where(i, L, cta, slot);
                double *dst = cluster.map_shared_rank(jb + size_t(slot) * slot_len, cta);
                dst[kj] = i <= kj ? col[i] : 0.0;
            }
        }
    }
    // own slots: V = I (and X = W on the direct path; zeros for the dummy)
    for (int s = warp; s < 2 * L.PP; s += nw) {
        const int pr = c * L.PP + (s >> 1);
        if (pr >= L.half)
            continue;
        const int pos = (s & 1) ? L.n_pad - 1 - pr : pr;  // = column at round 0
        double *x = jb + size_t(s) * slot_len;
        if (!pre)
            for (int i = lane; i < L.nX; i += 32)
                x[i] = pos < n ? J.A[size_t(pos) * m + i] : 0.0;
        else if (pos >= n)
            for (int i = lane; i < L.nX; i += 32)
                x[i] = 0.0;
        for (int i = lane; i < n; i += 32)
            x[L.nX + i] = (i == pos) ? 1.0 : 0.0;
    }
    cluster.sync();

    // ---- one-sided Jacobi ---------------------------------------------------
    const int pr = c * L.PP + warp;
    const bool has_pair = warp < L.PP && pr < L.half;
    const int pos_t = pr, pos_b = L.n_pad - 1 - pr;
    int cta_t = 0, slot_t = 0, cta_b = 0, slot_b = 0;
    if (has_pair) {
        cl_where(cl_next(pos_t, L.n_pad), L, cta_t, slot_t);
        cl_where(cl_next(pos_b, L.n_pad), L, cta_b, slot_b);
    }
    int cur = 0, sweeps = 0;
    bool converged = false;
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        unsigned my_rot = 0;
        bool my_big = false;  // a rotated pair had cos^2 > kLast^2
        for (int r = 0; r < L.n_pad - 1; ++r) {
            if (has_pair) {
                const double *xt = jb + cur * buf_len + size_t(2 * warp) * slot_len;
                const double *xb = xt + slot_len;
                const int a = cl_column(pos_t, r, L.n_pad);
                const int b = cl_column(pos_b, r, L.n_pad);
                const bool real = (a < n) && (b < n);
                // rows in chunks of four per lane, loads first (one warp per
                // sub-partition: nothing else hides the shared-memory latency)
                double tt = 0.0, bb = 0.0, tb = 0.0;
                if (real)
                    for (int i0 = lane; i0 < L.nX; i0 += 32 * kClChunk) {
                        double x[kClChunk], y[kClChunk];
#pragma unroll
                        for (int u = 0; u < kClChunk; ++u) {
                            const int i = i0 + 32 * u;
                            x[u] = i < L.nX ? xt[i] : 0.0;
                            y[u] = i < L.nX ? xb[i] : 0.0;
                        }
#pragma unroll
                        for (int u = 0; u < kClChunk; ++u) {
                            tt = fma(x[u], x[u], tt);
                            bb = fma(y[u], y[u], bb);
                            tb = fma(x[u], y[u], tb);
                        }
                    }
                const double red3 = warp_sum3(tt, bb, tb, lane);
                tt = __shfl_sync(FULL, red3, 0);
                bb = __shfl_sync(FULL, red3, 8);
                tb = __shfl_sync(FULL, red3, 16);
                // p = the lower column index of the pair
                const bool top_is_p = a < b;
                const double al = top_is_p ? tt : bb, be = top_is_p ? bb : tt;
                double cs = 1.0, sn = 0.0;
                const double ab = al * be, g2 = tb * tb;
                bool rotate = real && al != 0.0 && be != 0.0 && g2 > (kTol * kTol) * ab;
                if (rotate) {
                    jacobi_rotation(al, be, tb, cs, sn);
                    my_big = my_big || g2 > (kLast * kLast) * ab;  // no division
                    ++my_rot;
                }
                // x_p' = c x_p - s x_q, x_q' = s x_p + c x_q, written to the
                // slots the two columns take in the next round
                const double ss = top_is_p ? sn : -sn;
                double *dt = cluster.map_shared_rank(
                    jb + (cur ^ 1) * buf_len + size_t(slot_t) * slot_len, cta_t);
                double *db = cluster.map_shared_rank(
                    jb + (cur ^ 1) * buf_len + size_t(slot_b) * slot_len, cta_b);
                for (int i0 = lane; i0 < slot_len; i0 += 32 * kClChunk) {
                    double x[kClChunk], y[kClChunk];
#pragma unroll
                    for (int u = 0; u < kClChunk; ++u) {
                        const int i = i0 + 32 * u;
                        x[u] = i < slot_len ? xt[i] : 0.0;
                        y[u] = i < slot_len ? xb[i] : 0.0;
                    }
                    if (rotate) {
#pragma unroll
                        for (int u = 0; u < kClChunk; ++u) {
                            const double a2 = cs * x[u] - ss * y[u];
                            y[u] = ss * x[u] + cs * y[u];
                            x[u] = a2;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kClChunk; ++u) {
                        const int i = i0 + 32 * u;
                        if (i < slot_len) {
                            dt[i] = x[u];
                            db[i] = y[u];
                        }
                    }
                }
            }
            cur ^= 1;
            cluster.sync();
        }
        // every warp publishes its rotations and flag in its own CTA (plain
        // stores, double buffered by sweep parity); after the barrier every
        // warp reads all CTAs' entries and takes the same decision
        if (lane == 0)
            swstat[(sweep & 1) * kClWarps + warp] = (my_rot & 0x7fffffffu) |
                                                    (my_big ? 0x80000000u : 0u);
        cluster.sync();
        unsigned nrot = 0u, big = 0u;
        for (int e = lane; e < CL * nw; e += 32) {
            const unsigned v = *cluster.map_shared_rank(
                swstat + (sweep & 1) * kClWarps + (e % nw), e / nw);
            nrot += v & 0x7fffffffu;
            big |= v >> 31;
        }
        nrot = __reduce_add_sync(FULL, nrot);
        big = __reduce_or_sync(FULL, big);
        sweeps = sweep + 1;
        if (nrot == 0u || big == 0u) {
            converged = true;
            break;
        }
    }

    // ---- results: position i holds column i at the start of a sweep --------
    for (int s = warp; s < 2 * L.PP; s += nw) {
        const int p2 = c * L.PP + (s >> 1);
        if (p2 >= L.half)
            continue;
        const int pos = (s & 1) ? L.n_pad - 1 - p2 : p2;
        if (pos >= n)
            continue;
        const double *x = jb + cur * buf_len + size_t(s) * slot_len;
        for (int i = lane; i < L.nX; i += 32)
            J.X[size_t(pos) * L.nX + i] = x[i];
        for (int i = lane; i < n; i += 32)
            J.V[size_t(pos) * n + i] = x[L.nX + i];
    }
    if (c == 0 && tid == 0) {
        J.bar[6] = unsigned(sweeps);
        if (!converged)
            J.bar[5] = unsigned(WOS_NO_CONVERGENCE);
    }
    // no CTA may leave while others can still read its shared memory
    cluster.sync();
}
