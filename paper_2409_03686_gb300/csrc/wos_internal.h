// wos_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "wos.h"
#include "wos_device.cuh"

namespace wos {

wos_status cuda_status(cudaError_t e);
int ctx_device(const wos_context *c);
int ctx_sm_count(const wos_context *c);
void count_launches(wos_context *c, int n);
int ctx_max_smem(const wos_context *c);
int ctx_svd_path(const wos_context *c);  // WOS_SVD_AUTO / _GRID / _CLUSTER
// Stream i (< kClassStreams) of the context for a batched build's kernel
// classes, created non-blocking on first use; null if creation failed.
constexpr int kClassStreams = 18;
cudaStream_t ctx_class_stream(wos_context *c, int i);
// Launch fields of opts replaced by the context's tuned configuration for the
// class (precision, dim, kind) when they are all zero.
void apply_tuning(const wos_context *c, int precision, int dim, int kind, wos_opts *o);

// descriptor handling shared by the entry points (wos_api.cu)
wos_status validate(const wos_domain *d, const wos_partition *p);
int32_t num_elements(const wos_domain &d, const wos_partition &p);
template <typename Real>
void fill_geom(const wos_domain &d, const wos_partition &p, Geom<Real> &g);
wos_status setup_S(int d, const double *K, double *S);
double fp32_floor(const wos_domain &d);
// Mapped walks: whether the domain is a polytope the kernel can map (box,
// convex counter-clockwise polygon of <= kMaxPlanes edges, no holes); its
// faces in y = S^{-1} x, S and S^{-1}; the FP32 floor in y.
bool mapped_supported(const wos_domain &d);
template <typename Real>
void set_mapped(const wos_domain &d, const double *S, Geom<Real> &g);
double fp32_floor_mapped(const wos_domain &d, const double *S);
// Mapped walks on a disc / ball minus holes: S and lambda_min(S)^2 for the
// quadric bound of the step radius (walk_dist, kQuadric kinds).
template <typename Real>
void set_quadric(const wos_domain &d, const double *S, Geom<Real> &g);

// Argument checks of an operator build (wos_build_operator and its
// no-allocation variant): *o = opts (or zeros), S = (K / lambda_max)^{1/2};
// returns the first error (WOS_INVALID_ARG, WOS_COUNT_OVERFLOW,
// WOS_K_NOT_SPD, WOS_EPS_BELOW_FP32_FLOOR).
wos_status validate_build(const wos_context *ctx, const wos_domain *domain, const double *K,
                          const double *points, int32_t M_D,
                          const wos_partition *partition, uint32_t N, double eps,
                          const wos_opts *opts, const uint32_t *counts, wos_opts *o,
                          double *S);
// Enqueues the FP64 inside test of the points (device, M_D x dim) on
// `stream`: an outside point sets work[5] = M_D - (its index), the largest
// such value, and work[0] past every tile, so the walk kernel launched next
// on the stream with this work array runs no walk.  work[0] and work[5]
// must be zero before.
cudaError_t launch_point_check(const wos_domain &d, const wos_partition &part,
                               const double *points, int32_t M_D,
                               unsigned long long *work, cudaStream_t stream);

// Points the geometry at a Voronoi candidate grid already on the device.
template <typename Real, typename Grid>
void set_voronoi_grid(const Grid &G, const int32_t *dstart, const int32_t *dcand,
                      Geom<Real> &g)
{
    g.vcell = dstart;
    g.vcand = dcand;
    for (int a = 0; a < 3; ++a) {
        g.vg[a] = G.g[a];
        g.vlo[a] = Real(G.lo[a]);
    }
    g.vinv_h = Real(1.0 / G.h);
}

}  // namespace wos
