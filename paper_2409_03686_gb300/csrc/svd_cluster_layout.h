// svd_cluster_layout.h -- the data layout of the cluster SVD kernel
// (svd_cluster.cuh), host- and device-callable so that the host picks the
// shared memory of a launch and the tests check the column movement.
//
// One-sided Jacobi in the round-robin order (the circle method): n_pad
// columns (n rounded up to even) sit at positions 0..n_pad-1; round r pairs
// position pr with position n_pad - 1 - pr (pr < n_pad / 2); between rounds
// position 0 keeps its column and every other column moves one position down
// (position 1 to n_pad - 1), so that n_pad - 1 rounds meet every pair of
// columns once.  Pair pr lives in CTA pr / PP of the cluster, its top
// column in slot 2 (pr mod PP), its bottom column in the next slot.
#pragma once

#include <cstddef>

#ifdef __CUDACC__
#define CL_HD __host__ __device__
#else
#define CL_HD
#endif

constexpr int kClThreads = 256;
constexpr int kClWarps = kClThreads / 32;
constexpr int kClMaxCtas = 16;
constexpr int kClMaxN = 2 * kClMaxCtas * kClWarps;  // 256 columns
constexpr int kClChunk = 4;                          // rows per lane per chunk

// Shared-memory layout of one CTA (bytes, 16-byte aligned pieces).
struct ClLayout {
    int CL, PP, cpc, nX, n_pad, half;
    size_t small, qcol, vbuf, jb, total;
};

CL_HD inline size_t cl_align(size_t b) { return (b + 15) / 16 * 16; }

CL_HD inline ClLayout cl_layout(int m, int n, int pre, int CL)
{
    ClLayout L;
    L.CL = CL;
    L.n_pad = n + (n & 1) < 2 ? 2 : n + (n & 1);
    L.half = L.n_pad / 2;
    L.PP = (L.half + CL - 1) / CL;
    L.cpc = pre ? (n + CL - 1) / CL : 0;
    L.nX = pre ? n : m;
    // small: pub_val[2][16] double, pub_idx[2][16] int, tau_all[n] double,
    // perm_all[n] int, cn[cpc], cn0[cpc] double, flags[cpc] int (done, or
    // pivot position + 1), sweep statistics of the warps [2][kClWarps],
    // scalar scratch
    size_t s = 0;
    s += cl_align(2 * 16 * 8) + cl_align(2 * 16 * 4);
    s += cl_align(size_t(n) * 8) + cl_align(size_t(n) * 4);
    s += 2 * cl_align(size_t(L.cpc) * 8) + cl_align(size_t(L.cpc) * 4);
    s += cl_align(2 * kClWarps * 4) + cl_align(64 * 8);
    L.small = s;
    L.qcol = pre ? cl_align(size_t(L.cpc) * m * 8) : 0;
    L.vbuf = pre ? cl_align(size_t(m) * 8) : 0;
    L.jb = cl_align(size_t(2) * 2 * L.PP * (L.nX + n) * 8);
    L.total = L.small + L.qcol + L.vbuf + L.jb;
    return L;
}

// Column at position pos in round r.
CL_HD inline int cl_column(int pos, int r, int n_pad)
{
    return pos == 0 ? 0 : 1 + (pos - 1 + r) % (n_pad - 1);
}

// CTA and slot of position pos: pair pr = pos (top) or n_pad - 1 - pos
// (bottom); CTA pr / PP, slot 2 (pr mod PP) + (bottom).
CL_HD inline void cl_where(int pos, const ClLayout &L, int &cta, int &slot)
{
    const bool top = pos < L.half;
    const int pr = top ? pos : L.n_pad - 1 - pos;
    cta = pr / L.PP;
    slot = 2 * (pr - cta * L.PP) + (top ? 0 : 1);
}

// Position in the next round of the column at position pos.
CL_HD inline int cl_next(int pos, int n_pad)
{
    return pos == 0 ? 0 : (pos == 1 ? n_pad - 1 : pos - 1);
}
