// wos_api.cu -- host side of the C ABI declared in include/wos.h: argument
// validation, instance set-up (paper Sec. 4.2: K_s = K / lambda_max(K),
// S = K_s^{1/2}), launch configuration of the persistent walk kernel and the
// context object.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "wos.h"
#include "voronoi_grid.h"
#include "wos_internal.h"
#include "walk_launch.cuh"

using namespace wos;

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct wos_context {
    std::atomic<uint64_t> launches{0};
    std::mutex tune_mu;
    std::map<int, wos_tuning> tuned;  // key: precision, dim, kernel kind
    int device = 0;
    int sm_count = 0;
    int max_smem_optin = 0;
    std::atomic<int> svd_path{WOS_SVD_AUTO};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // streams of the batched build's kernel classes (created on first use)
    std::mutex class_mu;
    cudaStream_t class_streams[wos::kClassStreams] = {};
};

namespace wos {

wos_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess)
        return WOS_OK;
    if (e == cudaErrorMemoryAllocation)
        return WOS_OOM;
    return WOS_CUDA_ERROR;
}

int ctx_device(const wos_context *c) { return c->device; }
void count_launches(wos_context *c, int n) { c->launches += uint64_t(n); }
int ctx_sm_count(const wos_context *c) { return c->sm_count; }
int ctx_max_smem(const wos_context *c) { return c->max_smem_optin; }
int ctx_svd_path(const wos_context *c) { return c->svd_path.load(); }

cudaStream_t ctx_class_stream(wos_context *c, int i)
{
    std::lock_guard<std::mutex> lock(c->class_mu);
    if (!c->class_streams[i] &&
        cudaStreamCreateWithFlags(&c->class_streams[i], cudaStreamNonBlocking) != cudaSuccess)
        c->class_streams[i] = nullptr;
    return c->class_streams[i];
}

static int tune_key(int precision, int dim, int kind) { return (precision << 8) | (dim << 4) | kind; }

void apply_tuning(const wos_context *c, int precision, int dim, int kind, wos_opts *o)
{
    if (o->block_size || o->blocks_per_sm || o->tile_walks || o->hist_slots ||
        o->refill_min || o->tiles_per_warp || o->group_blocks)
        return;
    wos_context *cc = const_cast<wos_context *>(c);
    std::lock_guard<std::mutex> lock(cc->tune_mu);
    auto it = cc->tuned.find(tune_key(precision, dim, kind));
    if (it == cc->tuned.end())
        return;
    o->block_size = it->second.block_size;
    o->blocks_per_sm = it->second.blocks_per_sm;
    o->tiles_per_warp = it->second.tiles_per_warp;
    o->hist_slots = it->second.hist_slots;
    o->refill_min = it->second.refill_min;
    o->group_blocks = it->second.group_blocks;
}

}  // namespace wos

extern "C" wos_status wos_create(int32_t device, wos_context **out)
{
    if (!out)
        return WOS_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n)
        return WOS_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess)
        return WOS_CUDA_ERROR;
    wos_context *c = new (std::nothrow) wos_context();
    if (!c)
        return WOS_OOM;
    c->device = device;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&c->max_smem_optin,
                           cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (cudaEventCreate(&c->ev0) != cudaSuccess ||
        cudaEventCreate(&c->ev1) != cudaSuccess) {
        delete c;
        return WOS_CUDA_ERROR;
    }
    *out = c;
    return WOS_OK;
}

extern "C" wos_status wos_destroy(wos_context *c)
{
    if (!c)
        return WOS_INVALID_ARG;
    cudaSetDevice(c->device);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    for (cudaStream_t st : c->class_streams)
        if (st)
            cudaStreamDestroy(st);
    delete c;
    return WOS_OK;
}

extern "C" uint64_t wos_kernel_launches(const wos_context *c)
{
    return c ? c->launches.load() : 0;
}

extern "C" wos_status wos_set_svd_path(wos_context *c, int32_t path)
{
    if (!c || path < WOS_SVD_AUTO || path > WOS_SVD_FP64_SWEEPS)
        return WOS_INVALID_ARG;
    c->svd_path.store(path);
    return WOS_OK;
}

extern "C" const char *wos_status_string(wos_status s)
{
    switch (s) {
    case WOS_OK: return "ok";
    case WOS_INVALID_ARG: return "invalid argument";
    case WOS_K_NOT_SPD: return "K is not symmetric positive definite";
    case WOS_POINT_OUTSIDE: return "observation point outside the domain";
    case WOS_EPS_BELOW_FP32_FLOOR: return "eps below the FP32 safety floor";
    case WOS_COUNT_OVERFLOW: return "walk ids or counts overflow";
    case WOS_STEP_CAP_HIT: return "some walks reached the step cap";
    case WOS_DEVICE_TIMEOUT: return "device-side wait timed out";
    case WOS_OOM: return "device out of memory";
    case WOS_CUDA_ERROR: return "CUDA runtime error";
    case WOS_NO_CONVERGENCE: return "Jacobi SVD did not converge";
    case WOS_TRUNCATION_IN_CLUSTER: return "truncation inside a singular-value cluster";
    case WOS_NOT_READY: return "not ready";
    }
    return "unknown status";
}

// ---------------------------------------------------------------------------
// descriptors
// ---------------------------------------------------------------------------
namespace wos {

static int32_t outer_elements(const wos_domain &d, const wos_partition &p)
{
    if (d.outer_kind == WOS_OUTER_SPHERE)
        return d.dim == 2 ? p.outer_m : p.outer_nb * p.outer_ns;
    if (d.outer_kind == WOS_OUTER_BOX && d.dim == 3)
        return 6 * p.face_n1 * p.face_n2;
    int ne = d.outer_kind == WOS_OUTER_BOX ? 4 : d.n_vertices;
    int64_t s = 0;
    for (int e = 0; e < ne; ++e)
        s += p.edge_m[e];
    return int32_t(s);
}

static int32_t hole_elements(const wos_domain &d, const wos_partition &p, int h)
{
    return d.dim == 2 ? p.hole_m[h] : p.hole_nb[h] * p.hole_ns[h];
}

wos_status validate(const wos_domain *dp, const wos_partition *pp)
{
    if (!dp || !pp)
        return WOS_INVALID_ARG;
    const wos_domain &d = *dp;
    const wos_partition &p = *pp;
    if (d.dim != 2 && d.dim != 3)
        return WOS_INVALID_ARG;
    if (d.n_holes < 0 || d.n_holes > WOS_MAX_HOLES)
        return WOS_INVALID_ARG;
    for (int h = 0; h < d.n_holes; ++h)
        if (!(d.hole_radius[h] > 0.0))
            return WOS_INVALID_ARG;
    bool cells = p.voronoi_n <= 0;
    switch (d.outer_kind) {
    case WOS_OUTER_SPHERE:
        if (!(d.radius > 0.0))
            return WOS_INVALID_ARG;
        if (cells && d.dim == 2 && p.outer_m < 1)
            return WOS_INVALID_ARG;
        if (cells && d.dim == 3 && (p.outer_nb < 1 || p.outer_ns < 1))
            return WOS_INVALID_ARG;
        break;
    case WOS_OUTER_BOX:
        for (int a = 0; a < d.dim; ++a)
            if (!(d.half[a] > 0.0))
                return WOS_INVALID_ARG;
        if (cells && d.dim == 2)
            for (int e = 0; e < 4; ++e)
                if (p.edge_m[e] < 1)
                    return WOS_INVALID_ARG;
        if (cells && d.dim == 3 && (p.face_n1 < 1 || p.face_n2 < 1))
            return WOS_INVALID_ARG;
        break;
    case WOS_OUTER_POLYGON: {
        if (d.dim != 2 || d.n_vertices < 3 || d.n_vertices > WOS_MAX_VERTICES)
            return WOS_INVALID_ARG;
        double area2 = 0.0;
        for (int e = 0; e < d.n_vertices; ++e) {
            int e1 = (e + 1) % d.n_vertices;
            double ax = d.vertices[2 * e], ay = d.vertices[2 * e + 1];
            double bx = d.vertices[2 * e1], by = d.vertices[2 * e1 + 1];
            if (ax == bx && ay == by)
                return WOS_INVALID_ARG;
            area2 += ax * by - bx * ay;
            if (cells && p.edge_m[e] < 1)
                return WOS_INVALID_ARG;
        }
        if (!(area2 > 0.0))
            return WOS_INVALID_ARG;  // vertices must be counter-clockwise
        break;
    }
    default:
        return WOS_INVALID_ARG;
    }
    if (cells)
        for (int h = 0; h < d.n_holes; ++h)
            if (hole_elements(d, p, h) < 1 || (d.dim == 3 && (p.hole_nb[h] < 1 || p.hole_ns[h] < 1)))
                return WOS_INVALID_ARG;
    if (!cells && !p.voronoi_sites)
        return WOS_INVALID_ARG;
    return WOS_OK;
}

int32_t num_elements(const wos_domain &d, const wos_partition &p)
{
    if (p.voronoi_n > 0)
        return p.voronoi_n;
    int64_t s = outer_elements(d, p);
    for (int h = 0; h < d.n_holes; ++h)
        s += hole_elements(d, p, h);
    return s > INT32_MAX / 2 ? -1 : int32_t(s);
}

template <typename Real>
void fill_geom(const wos_domain &d, const wos_partition &p, Geom<Real> &g)
{
    std::memset(&g, 0, sizeof(g));
    g.dim = d.dim;
    g.outer_kind = d.outer_kind;
    g.n_holes = d.n_holes;
    g.M_tot = num_elements(d, p);
    g.vn = p.voronoi_n > 0 ? p.voronoi_n : 0;
    for (int a = 0; a < 3; ++a) {
        g.c[a] = Real(d.center[a]);
        g.h[a] = Real(d.half[a]);
    }
    g.R = Real(d.radius);
    const double inv2pi = 0.15915494309189533577;
    g.outer_m = p.outer_m;
    g.outer_t0 = Real(p.outer_theta0 * inv2pi);
    g.nb = p.outer_nb;
    g.ns = p.outer_ns;
    g.n1 = p.face_n1;
    g.n2 = p.face_n2;
    int ne = 0;
    if (d.outer_kind == WOS_OUTER_POLYGON) {
        ne = d.n_vertices;
        g.n_vert = ne;
        for (int e = 0; e < ne; ++e) {
            int e1 = (e + 1) % ne;
            double ax = d.vertices[2 * e], ay = d.vertices[2 * e + 1];
            double bx = d.vertices[2 * e1], by = d.vertices[2 * e1 + 1];
            g.vx[e] = Real(ax);
            g.vy[e] = Real(ay);
            g.ex[e] = Real(bx - ax);
            g.ey[e] = Real(by - ay);
            g.il2[e] = Real(1.0 / ((bx - ax) * (bx - ax) + (by - ay) * (by - ay)));
        }
    } else if (d.outer_kind == WOS_OUTER_BOX && d.dim == 2) {
        ne = 4;
    }
    int32_t off = 0;
    for (int e = 0; e < ne; ++e) {
        g.edge_m[e] = p.edge_m[e];
        g.edge_off[e] = off;
        off += p.edge_m[e];
    }
    off = outer_elements(d, p);
    for (int h = 0; h < d.n_holes; ++h) {
        for (int a = 0; a < 3; ++a)
            g.hc[h][a] = Real(d.hole_center[h][a]);
        g.hr[h] = Real(d.hole_radius[h]);
        g.hole_m[h] = p.hole_m[h];
        g.hole_t0[h] = Real(p.hole_theta0[h] * inv2pi);
        g.hole_nb[h] = p.hole_nb[h];
        g.hole_ns[h] = p.hole_ns[h];
        g.hole_off[h] = off;
        off += hole_elements(d, p, h);
    }
    if (d.n_holes > 0) {
        g.amid = Real(0.5 * (d.radius + d.hole_radius[0]));
        g.ahalf = Real(0.5 * (d.radius - d.hole_radius[0]));
    }
}

template void fill_geom<float>(const wos_domain &, const wos_partition &, Geom<float> &);
template void fill_geom<double>(const wos_domain &, const wos_partition &, Geom<double> &);

// Symmetric eigen-decomposition of a d x d matrix (d <= 3) by cyclic Jacobi
// rotations: A = Q diag(w) Q^T.
static void sym_eig(int d, const double *A, double *w, double *Q)
{
    double a[9];
    std::memcpy(a, A, sizeof(double) * d * d);
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j)
            Q[i * d + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < d; ++i)
            for (int j = i + 1; j < d; ++j)
                off += a[i * d + j] * a[i * d + j];
        if (off == 0.0)
            break;
        for (int pp = 0; pp < d; ++pp)
            for (int q = pp + 1; q < d; ++q) {
                double apq = a[pp * d + q];
                if (apq == 0.0)
                    continue;
                double theta = (a[q * d + q] - a[pp * d + pp]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) /
                           (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < d; ++k) {  // A <- A J
                    double akp = a[k * d + pp], akq = a[k * d + q];
                    a[k * d + pp] = c * akp - s * akq;
                    a[k * d + q] = s * akp + c * akq;
                }
                for (int k = 0; k < d; ++k) {  // A <- J^T A
                    double apk = a[pp * d + k], aqk = a[q * d + k];
                    a[pp * d + k] = c * apk - s * aqk;
                    a[q * d + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < d; ++k) {  // Q <- Q J
                    double qkp = Q[k * d + pp], qkq = Q[k * d + q];
                    Q[k * d + pp] = c * qkp - s * qkq;
                    Q[k * d + q] = s * qkp + c * qkq;
                }
            }
    }
    for (int i = 0; i < d; ++i)
        w[i] = a[i * d + i];
}

wos_status setup_S(int d, const double *K, double *S)
{
    if (!K)
        return WOS_INVALID_ARG;
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double x = K[i * d + j], y = K[j * d + i];
            if (!std::isfinite(x) ||
                std::fabs(x - y) > 1e-12 * (std::fabs(x) + std::fabs(y) + 1e-300))
                return WOS_K_NOT_SPD;
        }
    double w[3], Q[9];
    sym_eig(d, K, w, Q);
    double lmax = w[0];
    for (int i = 1; i < d; ++i)
        lmax = std::max(lmax, w[i]);
    for (int i = 0; i < d; ++i)
        if (!(w[i] > 1e-12 * lmax))
            return WOS_K_NOT_SPD;
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double acc = 0.0;
            for (int k = 0; k < d; ++k)
                acc += Q[i * d + k] * std::sqrt(w[k] / lmax) * Q[j * d + k];
            S[i * d + j] = acc;
        }
    return WOS_OK;
}

double fp32_floor(const wos_domain &d)
{
    double m = 0.0;
    auto upd = [&](double v) { m = std::max(m, std::fabs(v)); };
    if (d.outer_kind == WOS_OUTER_SPHERE)
        for (int a = 0; a < d.dim; ++a) {
            upd(d.center[a] - d.radius);
            upd(d.center[a] + d.radius);
        }
    else if (d.outer_kind == WOS_OUTER_BOX)
        for (int a = 0; a < d.dim; ++a) {
            upd(d.center[a] - d.half[a]);
            upd(d.center[a] + d.half[a]);
        }
    else
        for (int e = 0; e < 2 * d.n_vertices; ++e)
            upd(d.vertices[e]);
    return 128.0 * std::ldexp(1.0, -24) * m;
}

// Faces a.x <= c of the box or convex polygon D (outward unit a).
static int polytope_faces(const wos_domain &d, double (*a)[3], double *c)
{
    int nf = 0;
    if (d.outer_kind == WOS_OUTER_BOX) {
        for (int ax = 0; ax < d.dim; ++ax)
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                for (int b = 0; b < 3; ++b)
                    a[nf][b] = b == ax ? double(sgn) : 0.0;
                c[nf++] = sgn * d.center[ax] + d.half[ax];
            }
        return nf;
    }
    const int nv = d.n_vertices;
    for (int e = 0; e < nv; ++e) {
        const double *v0 = d.vertices + 2 * e, *v1 = d.vertices + 2 * ((e + 1) % nv);
        const double tx = v1[0] - v0[0], ty = v1[1] - v0[1], L = std::hypot(tx, ty);
        a[nf][0] = ty / L;
        a[nf][1] = -tx / L;
        a[nf][2] = 0.0;
        c[nf++] = a[e][0] * v0[0] + a[e][1] * v0[1];
    }
    return nf;
}

bool mapped_supported(const wos_domain &d)
{
    if (d.outer_kind == WOS_OUTER_SPHERE)
        return true;  // a disc / ball minus any holes: the quadric bound
    if (d.n_holes != 0)
        return false;
    if (d.outer_kind == WOS_OUTER_BOX)
        return true;
    if (d.outer_kind != WOS_OUTER_POLYGON || d.dim != 2 || d.n_vertices > kMaxPlanes)
        return false;
    const int nv = d.n_vertices;
    for (int e = 0; e < nv; ++e) {  // convex, counter-clockwise: left turns only
        const double *p0 = d.vertices + 2 * e, *p1 = d.vertices + 2 * ((e + 1) % nv),
                     *p2 = d.vertices + 2 * ((e + 2) % nv);
        const double cr = (p1[0] - p0[0]) * (p2[1] - p1[1]) - (p1[1] - p0[1]) * (p2[0] - p1[0]);
        if (!(cr > 0.0))
            return false;
    }
    return true;
}

// Inverse of a symmetric positive definite d x d matrix (d <= 3), by
// cofactors.
static void inverse(int dim, const double *S, double *Si)
{
    if (dim == 2) {
        const double det = S[0] * S[3] - S[1] * S[2];
        Si[0] = S[3] / det; Si[1] = -S[1] / det; Si[2] = -S[2] / det; Si[3] = S[0] / det;
        return;
    }
    double cof[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
            cof[i * 3 + j] = S[i1 * 3 + j1] * S[i2 * 3 + j2] - S[i1 * 3 + j2] * S[i2 * 3 + j1];
        }
    const double det = S[0] * cof[0] + S[1] * cof[1] + S[2] * cof[2];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Si[i * 3 + j] = cof[j * 3 + i] / det;
}

// A face a.x <= c becomes (S a).y <= c in y = S^{-1} x (S symmetric),
// normalised to a unit normal.
template <typename Real>
void set_mapped(const wos_domain &d, const double *S, Geom<Real> &g)
{
    const int dim = d.dim;
    double a[kMaxPlanes][3], c[kMaxPlanes], Si[9] = {0};
    const int nf = polytope_faces(d, a, c);
    inverse(dim, S, Si);
    g.mapped = 1;
    g.np = nf;
    for (int f = 0; f < kMaxPlanes; ++f) {
        double m[3] = {0.0, 0.0, 0.0}, L = 0.0;
        if (f < nf) {
            for (int i = 0; i < dim; ++i) {
                for (int j = 0; j < dim; ++j)
                    m[i] += S[i * dim + j] * a[f][j];
                L += m[i] * m[i];
            }
            L = std::sqrt(L);
        }
        for (int i = 0; i < 3; ++i)
            g.pn[f][i] = f < nf ? Real(m[i] / L) : Real(0);
        g.pd[f] = f < nf ? Real(c[f] / L) : Real(0);
    }
    for (int i = 0; i < 9; ++i) {
        g.mS[i] = i < dim * dim ? Real(S[i]) : Real(0);
        g.mSinv[i] = i < dim * dim ? Real(Si[i]) : Real(0);
    }
}

template <typename Real>
void set_quadric(const wos_domain &d, const double *S, Geom<Real> &g)
{
    const int dim = d.dim;
    double w[3], Q[9];
    sym_eig(dim, S, w, Q);
    double mu = w[0];
    for (int a = 1; a < dim; ++a)
        mu = std::min(mu, w[a]);
    g.mapped = 2;
    for (int i = 0; i < 9; ++i)
        g.mS[i] = i < dim * dim ? Real(S[i]) : Real(0);
    g.qmu2 = Real(mu * mu);
}

template void set_quadric<float>(const wos_domain &, const double *, Geom<float> &);
template void set_quadric<double>(const wos_domain &, const double *, Geom<double> &);
template void set_mapped<float>(const wos_domain &, const double *, Geom<float> &);
template void set_mapped<double>(const wos_domain &, const double *, Geom<double> &);

// The floor of the unmapped walks over the coordinates y = S^{-1} x of D's
// corners (the walk's own coordinates).
double fp32_floor_mapped(const wos_domain &d, const double *S)
{
    const int dim = d.dim;
    double Si[9] = {0}, m = 0.0;
    inverse(dim, S, Si);
    auto corner = [&](const double *x) {
        for (int i = 0; i < dim; ++i) {
            double y = 0.0;
            for (int j = 0; j < dim; ++j)
                y += Si[i * dim + j] * x[j];
            m = std::max(m, std::fabs(y));
        }
    };
    if (d.outer_kind == WOS_OUTER_BOX) {
        for (int q = 0; q < (1 << dim); ++q) {
            double x[3];
            for (int a = 0; a < dim; ++a)
                x[a] = d.center[a] + (((q >> a) & 1) ? d.half[a] : -d.half[a]);
            corner(x);
        }
    } else {
        for (int v = 0; v < d.n_vertices; ++v)
            corner(d.vertices + 2 * v);
    }
    return 128.0 * std::ldexp(1.0, -24) * m;
}

}  // namespace wos

extern "C" wos_status wos_conductivity_sqrt(int32_t dim, const double *K, double *S)
{
    if ((dim != 2 && dim != 3) || !K || !S)
        return WOS_INVALID_ARG;
    return setup_S(dim, K, S);
}

extern "C" int32_t wos_num_elements(const wos_domain *d, const wos_partition *p)
{
    if (validate(d, p) != WOS_OK)
        return -1;
    return num_elements(*d, *p);
}

extern "C" double wos_fp32_eps_floor(const wos_domain *d)
{
    return d ? fp32_floor(*d) : 0.0;
}

// ---------------------------------------------------------------------------
// sigma(omega_j) of extrinsic Voronoi cells (App. A, Ex. A.2) whose sites lie
// on the circles / spheres of the domain (the outer sphere and the holes);
// each of those surfaces is shared among its own sites (a site belongs to the
// circle or sphere it lies on, within 1e-9 of its radius).
//   2-D: the cell of a site on a circle of radius r is the arc between the
//        bisectors of its two angular neighbours (the perpendicular bisector
//        of two points of a circle passes through its centre), of length
//        r (theta_next - theta_prev) / 2; a lone site owns the whole circle.
//   3-D: the cell of a site s on a sphere is {x : x.s >= x.s' for every other
//        site s' of the sphere}, an intersection of hemispheres.  In the
//        central (gnomonic) projection onto the plane tangent at s every
//        great circle is a line, so the cell is a convex polygon, built by
//        clipping a square by one half-plane per other site; its area is
//        the sum of the spherical triangles (s, v_k, v_{k+1}), each from
//        tan(E / 2) = a.(b x c) / (1 + a.b + b.c + c.a) (Van Oosterom &
//        Strackee, IEEE Trans. Biomed. Eng. 30, 1983).  A cell reaching
//        89.9 degrees from its site is not representable: WOS_INVALID_ARG.
// Identical sites: the lowest index owns the cell, the others get 0 (the
// classifier's tie rule).  Outer boxes and polygons: WOS_INVALID_ARG.
// ---------------------------------------------------------------------------
namespace {

// A vertex of the clipped polygon and the line of the edge that starts at
// it (line index into the caller's table).
struct P2 {
    double a, b;
    int next;
};
struct Line {
    double A, B, C;  // A a + B b = C
};

// Keeps the part of the convex polygon with A a + B b <= C, line j of the
// table (Sutherland & Hodgman, one edge).
void clip_half_plane(std::vector<P2> &poly, const Line &ln, int j, std::vector<P2> &tmp)
{
    tmp.clear();
    const size_t n = poly.size();
    for (size_t k = 0; k < n; ++k) {
        const P2 u = poly[k], v = poly[(k + 1) % n];
        const double fu = ln.A * u.a + ln.B * u.b - ln.C, fv = ln.A * v.a + ln.B * v.b - ln.C;
        if (fu <= 0.0)
            tmp.push_back(u);
        if ((fu < 0.0 && fv > 0.0) || (fu > 0.0 && fv < 0.0)) {
            const double t = fu / (fu - fv);
            const P2 x{u.a + t * (v.a - u.a), u.b + t * (v.b - u.b), fu < 0.0 ? j : u.next};
            tmp.push_back(x);
        }
    }
    poly.swap(tmp);
}

double spherical_cell_area(const double *u0, const std::vector<const double *> &others,
                           bool *ok)
{
    // tangent basis e1, e2 of the plane at u0
    double t[3] = {0, 0, 0};
    int ax = 0;
    for (int a = 1; a < 3; ++a)
        if (std::fabs(u0[a]) < std::fabs(u0[ax]))
            ax = a;
    t[ax] = 1.0;
    double e1[3], e2[3];
    const double td = t[0] * u0[0] + t[1] * u0[1] + t[2] * u0[2];
    for (int a = 0; a < 3; ++a)
        e1[a] = t[a] - td * u0[a];
    const double n1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int a = 0; a < 3; ++a)
        e1[a] /= n1;
    e2[0] = u0[1] * e1[2] - u0[2] * e1[1];
    e2[1] = u0[2] * e1[0] - u0[0] * e1[2];
    e2[2] = u0[0] * e1[1] - u0[1] * e1[0];
    const double L = 1.0e3;  // tan(89.94 degrees)
    // lines 0..3: the square's sides; 4 + q: the bisector of other site q
    std::vector<Line> lines = {{0, -1, L}, {1, 0, L}, {0, 1, L}, {-1, 0, L}};
    std::vector<P2> poly = {{-L, -L, 0}, {L, -L, 1}, {L, L, 2}, {-L, L, 3}}, tmp;
    for (const double *uj : others) {
        // x = u0 + a e1 + b e2 is in the cell when x.(u0 - uj) >= 0
        const Line ln{e1[0] * uj[0] + e1[1] * uj[1] + e1[2] * uj[2],
                      e2[0] * uj[0] + e2[1] * uj[1] + e2[2] * uj[2],
                      1.0 - (u0[0] * uj[0] + u0[1] * uj[1] + u0[2] * uj[2])};
        lines.push_back(ln);
        clip_half_plane(poly, ln, int(lines.size()) - 1, tmp);
        if (poly.empty())
            return 0.0;
    }
    // every vertex again as the intersection of the lines of its two edges
    // (the clipping interpolated along edges whose far ends can lie 1e3 away)
    const size_t n = poly.size();
    for (size_t k = 0; k < n; ++k) {
        const Line &l1 = lines[poly[(k + n - 1) % n].next], &l2 = lines[poly[k].next];
        const double det = l1.A * l2.B - l1.B * l2.A;
        if (det != 0.0) {
            poly[k].a = (l1.C * l2.B - l1.B * l2.C) / det;
            poly[k].b = (l1.A * l2.C - l1.C * l2.A) / det;
        }
    }
    double area = 0.0;
    std::vector<std::array<double, 3>> v(n);
    for (size_t k = 0; k < n; ++k) {
        if (std::fabs(poly[k].a) >= 0.5 * L || std::fabs(poly[k].b) >= 0.5 * L)
            *ok = false;
        double x[3];
        for (int a = 0; a < 3; ++a)
            x[a] = u0[a] + poly[k].a * e1[a] + poly[k].b * e2[a];
        const double nx = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        for (int a = 0; a < 3; ++a)
            v[k][a] = x[a] / nx;
    }
    for (size_t k = 0; k < n; ++k) {
        const double *b = v[k].data(), *c = v[(k + 1) % n].data();
        const double bc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2],
                              b[0] * c[1] - b[1] * c[0]};
        const double num = u0[0] * bc[0] + u0[1] * bc[1] + u0[2] * bc[2];
        const double den = 1.0 + (u0[0] * b[0] + u0[1] * b[1] + u0[2] * b[2]) +
                           (b[0] * c[0] + b[1] * c[1] + b[2] * c[2]) +
                           (c[0] * u0[0] + c[1] * u0[1] + c[2] * u0[2]);
        area += 2.0 * std::atan2(num, den);
    }
    return std::fabs(area);
}

wos_status voronoi_cell_measures(const wos_domain &d, const wos_partition &p, double *out)
{
    if (d.outer_kind != WOS_OUTER_SPHERE)
        return WOS_INVALID_ARG;
    const int dim = d.dim, ns = p.voronoi_n;
    const int ncomp = 1 + d.n_holes;
    auto centre = [&](int c) { return c == 0 ? d.center : d.hole_center[c - 1]; };
    auto radius = [&](int c) { return c == 0 ? d.radius : d.hole_radius[c - 1]; };
    std::vector<int> owner(ns, -1);
    std::vector<double> u(size_t(ns) * 3, 0.0);  // unit vector from the centre
    for (int j = 0; j < ns; ++j) {
        const double *x = p.voronoi_sites + size_t(j) * dim;
        for (int c = 0; c < ncomp && owner[j] < 0; ++c) {
            const double *cc = centre(c);
            const double r = radius(c);
            double v[3] = {0, 0, 0}, n2 = 0.0;
            for (int a = 0; a < dim; ++a) {
                v[a] = x[a] - cc[a];
                n2 += v[a] * v[a];
            }
            const double nv = std::sqrt(n2);
            if (std::fabs(nv - r) <= 1e-9 * std::max(r, 1.0) && nv > 0.0) {
                owner[j] = c;
                for (int a = 0; a < dim; ++a)
                    u[size_t(j) * 3 + a] = v[a] / nv;
            }
        }
        if (owner[j] < 0)
            return WOS_INVALID_ARG;  // a site on no circle / sphere of D
    }
    const double pi = 3.14159265358979323846;
    for (int c = 0; c < ncomp; ++c) {
        std::vector<int> idx;
        for (int j = 0; j < ns; ++j)
            if (owner[j] == c)
                idx.push_back(j);
        if (idx.empty())
            continue;
        const double r = radius(c);
        // identical sites: the lowest index keeps the cell
        std::vector<char> dup(ns, 0);
        for (size_t a = 0; a < idx.size(); ++a)
            for (size_t b = 0; b < a; ++b) {
                const double *ua = &u[size_t(idx[a]) * 3], *ub = &u[size_t(idx[b]) * 3];
                if (ua[0] == ub[0] && ua[1] == ub[1] && ua[2] == ub[2]) {
                    dup[idx[a]] = 1;
                    break;
                }
            }
        std::vector<int> live;
        for (int j : idx) {
            if (dup[j])
                out[j] = 0.0;
            else
                live.push_back(j);
        }
        if (dim == 2) {
            if (live.size() == 1) {
                out[live[0]] = 2 * pi * r;
                continue;
            }
            std::vector<std::pair<double, int>> ang;
            for (int j : live)
                ang.push_back({std::atan2(u[size_t(j) * 3 + 1], u[size_t(j) * 3]), j});
            std::sort(ang.begin(), ang.end());
            const size_t n = ang.size();
            for (size_t k = 0; k < n; ++k) {
                double nxt = ang[(k + 1) % n].first - ang[k].first;
                double prv = ang[k].first - ang[(k + n - 1) % n].first;
                if (k + 1 == n)
                    nxt += 2 * pi;
                if (k == 0)
                    prv += 2 * pi;
                out[ang[k].second] = r * 0.5 * (nxt + prv);
            }
        } else {
            bool ok = true;
            std::vector<const double *> others;
            for (int j : live) {
                others.clear();
                for (int q : live)
                    if (q != j)
                        others.push_back(&u[size_t(q) * 3]);
                out[j] = r * r * spherical_cell_area(&u[size_t(j) * 3], others, &ok);
            }
            if (!ok)
                return WOS_INVALID_ARG;
        }
    }
    return WOS_OK;
}

}  // namespace

extern "C" wos_status wos_element_measures(const wos_domain *dp,
                                           const wos_partition *pp, double *out)
{
    wos_status st = validate(dp, pp);
    if (st != WOS_OK)
        return st;
    if (!out)
        return WOS_INVALID_ARG;
    if (pp->voronoi_n > 0)
        return voronoi_cell_measures(*dp, *pp, out);
    const wos_domain &d = *dp;
    const wos_partition &p = *pp;
    const double pi = 3.14159265358979323846;
    int32_t q = 0;
    if (d.outer_kind == WOS_OUTER_SPHERE) {
        if (d.dim == 2)
            for (int j = 0; j < p.outer_m; ++j)
                out[q++] = 2 * pi * d.radius / p.outer_m;
        else
            for (int j = 0; j < p.outer_nb * p.outer_ns; ++j)
                out[q++] = 4 * pi * d.radius * d.radius / (p.outer_nb * p.outer_ns);
    } else if (d.outer_kind == WOS_OUTER_BOX && d.dim == 3) {
        for (int f = 0; f < 6; ++f) {
            int ax = f % 3, b0 = ax == 0 ? 1 : 0, b1 = ax == 2 ? 1 : 2;
            double a = (2 * d.half[b0] / p.face_n1) * (2 * d.half[b1] / p.face_n2);
            for (int j = 0; j < p.face_n1 * p.face_n2; ++j)
                out[q++] = a;
        }
    } else {
        double len[WOS_MAX_VERTICES];
        int ne;
        if (d.outer_kind == WOS_OUTER_BOX) {
            ne = 4;
            len[0] = len[2] = 2 * d.half[0];
            len[1] = len[3] = 2 * d.half[1];
        } else {
            ne = d.n_vertices;
            for (int e = 0; e < ne; ++e) {
                int e1 = (e + 1) % ne;
                len[e] = std::hypot(d.vertices[2 * e1] - d.vertices[2 * e],
                                    d.vertices[2 * e1 + 1] - d.vertices[2 * e + 1]);
            }
        }
        for (int e = 0; e < ne; ++e)
            for (int j = 0; j < p.edge_m[e]; ++j)
                out[q++] = len[e] / p.edge_m[e];
    }
    for (int h = 0; h < d.n_holes; ++h) {
        double r = d.hole_radius[h];
        if (d.dim == 2)
            for (int j = 0; j < p.hole_m[h]; ++j)
                out[q++] = 2 * pi * r / p.hole_m[h];
        else {
            int n = p.hole_nb[h] * p.hole_ns[h];
            for (int j = 0; j < n; ++j)
                out[q++] = 4 * pi * r * r / n;
        }
    }
    return WOS_OK;
}

extern "C" wos_status wos_check_points(const wos_domain *dp, const double *pts,
                                       int32_t M_D, int32_t *bad)
{
    wos_partition dummy;
    std::memset(&dummy, 0, sizeof(dummy));
    dummy.voronoi_n = 1;
    double site[3] = {0, 0, 0};
    dummy.voronoi_sites = site;
    wos_status st = validate(dp, &dummy);
    if (st != WOS_OK || (M_D > 0 && !pts) || M_D < 0)
        return WOS_INVALID_ARG;
    Geom<double> g;
    fill_geom(*dp, dummy, g);
    for (int32_t i = 0; i < M_D; ++i) {
        double r = dp->dim == 2 ? domain_dist<double, 2>(g, pts + 2 * i)
                                : domain_dist<double, 3>(g, pts + 3 * i);
        bool inside = r > 0.0;
        if (inside && dp->outer_kind == WOS_OUTER_POLYGON) {
            // the polygon distance is unsigned: add a crossing-number test
            double x = pts[2 * i], y = pts[2 * i + 1];
            bool in = false;
            int n = dp->n_vertices;
            for (int e = 0; e < n; ++e) {
                int e1 = (e + 1) % n;
                double ax = dp->vertices[2 * e], ay = dp->vertices[2 * e + 1];
                double bx = dp->vertices[2 * e1], by = dp->vertices[2 * e1 + 1];
                if ((ay > y) != (by > y) && x < ax + (y - ay) * (bx - ax) / (by - ay))
                    in = !in;
            }
            inside = in;
        }
        if (!inside) {
            if (bad)
                *bad = i;
            return WOS_POINT_OUTSIDE;
        }
    }
    return WOS_OK;
}

// ---------------------------------------------------------------------------
// observation points inside D, checked on the device before the walks
// ---------------------------------------------------------------------------
namespace {

// The test of wos_check_points in FP64 on the device: dist(x, dD) > 0 and,
// for a polygon (unsigned distance), an odd crossing number.  An outside
// point records M_D - i in work[5] (the largest value marks the lowest
// index) and takes every tile of the walk queue (work[0]), so that the walk
// kernel after it on the stream runs no walk at all instead of walking from
// outside D until the step cap.
template <int DIM>
__global__ void point_check_kernel(const __grid_constant__ Geom<double> g, const double *pts,
                                   int32_t M_D, unsigned long long *work)
{
    const int32_t i = int32_t(blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= M_D)
        return;
    const double *x = pts + size_t(i) * DIM;
    bool inside = domain_dist<double, DIM>(g, x) > 0.0;
    if (inside && DIM == 2 && g.outer_kind == kPolygon) {
        bool in = false;
        for (int e = 0; e < g.n_vert; ++e) {
            const int e1 = e + 1 < g.n_vert ? e + 1 : 0;
            const double ax = g.vx[e], ay = g.vy[e], bx = g.vx[e1], by = g.vy[e1];
            if ((ay > x[1]) != (by > x[1]) && x[0] < ax + (x[1] - ay) * (bx - ax) / (by - ay))
                in = !in;
        }
        inside = in;
    }
    if (!inside) {
        atomicMax(work + 5, (unsigned long long)(M_D - i));
        atomicExch(work, 1ull << 62);
    }
}

}  // namespace

namespace wos {

cudaError_t launch_point_check(const wos_domain &d, const wos_partition &part,
                               const double *points, int32_t M_D,
                               unsigned long long *work, cudaStream_t stream)
{
    Geom<double> g;
    std::memset(&g, 0, sizeof(g));
    fill_geom(d, part, g);
    const unsigned blocks = unsigned((M_D + 127) / 128);
    if (d.dim == 2)
        point_check_kernel<2><<<blocks, 128, 0, stream>>>(g, points, M_D, work);
    else
        point_check_kernel<3><<<blocks, 128, 0, stream>>>(g, points, M_D, work);
    return cudaGetLastError();
}

wos_status validate_build(const wos_context *ctx, const wos_domain *domain, const double *K,
                          const double *points, int32_t M_D,
                          const wos_partition *partition, uint32_t N, double eps,
                          const wos_opts *opts, const uint32_t *counts, wos_opts *o,
                          double *S)
{
    if (!ctx)
        return WOS_INVALID_ARG;
    wos_status st = validate(domain, partition);
    if (st != WOS_OK)
        return st;
    std::memset(o, 0, sizeof(*o));
    if (opts)
        *o = *opts;
    const uint32_t k1 = o->k1 ? o->k1 : N;
    if (M_D < 1 || N < 1 || !points || !counts || !(eps > 0.0) || o->k0 >= k1 || k1 > N)
        return WOS_INVALID_ARG;
    if (o->precision != WOS_FP32 && o->precision != WOS_FP64)
        return WOS_INVALID_ARG;
    if (o->block_size && (o->block_size % 32 != 0 || o->block_size > 256))
        return WOS_INVALID_ARG;
    if (o->hist_slots < -1 || o->hist_slots > 2)
        return WOS_INVALID_ARG;
    if (num_elements(*domain, *partition) < 1)
        return WOS_INVALID_ARG;
    // walk ids i * N + k must fit 64 bits (always true for int32 M_D)
    if (uint64_t(M_D) * uint64_t(N) > (1ull << 63))
        return WOS_COUNT_OVERFLOW;
    st = setup_S(domain->dim, K, S);
    if (st != WOS_OK)
        return st;
    if (o->mapped != 0 && (o->mapped != 1 || !mapped_supported(*domain)))
        return WOS_INVALID_ARG;
    // the polytope walks run in y = S^{-1} x, the others in x
    const bool in_y = o->mapped && domain->outer_kind != WOS_OUTER_SPHERE;
    if (o->precision == WOS_FP32 &&
        eps < (in_y ? fp32_floor_mapped(*domain, S) : fp32_floor(*domain)))
        return WOS_EPS_BELOW_FP32_FLOOR;
    return WOS_OK;
}

}  // namespace wos

// ---------------------------------------------------------------------------
// the walk launch
// ---------------------------------------------------------------------------
namespace {

template <typename Real>
__global__ void convert_points_kernel(const double *in, int n, Real *out)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n)
        out[q] = Real(in[q]);
}

template <typename Real>
wos_status build_impl(wos_context *ctx, const wos_domain &d,
                      const wos_partition &part, const double *S,
                      const double *points, int32_t M_D, uint32_t N, double eps,
                      uint64_t seed, const wos_opts &o_in, uint32_t *counts,
                      uint32_t *unterm, wos_stats *stats, cudaStream_t stream)
{
    WalkParams<Real> *pp = new (std::nothrow) WalkParams<Real>();
    if (!pp)
        return WOS_OOM;
    WalkParams<Real> &p = *pp;
    std::memset(&p, 0, sizeof(p));
    const int dim = d.dim;
    wos_opts o = o_in;
    apply_tuning(ctx, sizeof(Real) == sizeof(double) ? WOS_FP64 : WOS_FP32, dim,
                 walk_kind(d, part, o.mapped != 0), &o);
    fill_inst<Real>(d, part, S, points, M_D, N, eps, o.stream_id, o.k0, o.k1, o.step_cap,
                    counts, unterm, &p.one, o.mapped != 0);
    philox_round_keys(seed, p.rk);
    p.trace_elem = o.trace_elem;
    p.trace_steps = o.trace_steps;
    p.trace_x = o.trace_x;
    const int32_t M = p.one.g.M_tot;

    const uint64_t per_point = uint64_t(p.one.k1 - p.one.k0);
    WalkPlan plan;
    wos_status pst = plan_walk_any<Real>(dim, walk_kind(d, part, o.mapped != 0), M, o,
                                         ctx->sm_count,
                                         ctx->max_smem_optin, per_point, M_D, &plan);
    if (pst != WOS_OK) {
        delete pp;
        return pst;
    }
    apply_plan(plan, &p);
    p.refill_min = refill_min_of(o);
    p.group_blocks = group_blocks_of<Real>(o, dim);
    const void *kfn = plan.kfn;
    const int grid = plan.grid, block = plan.block, nslot = plan.nslot;
    const size_t smem = plan.smem;
    const uint64_t tw = plan.tile_w;

    // per-call scratch: work counters, statistics, Voronoi sites and (FP32
    // walks) the points in walk precision, so that no walk converts FP64
    size_t site_bytes = part.voronoi_n > 0 ? size_t(part.voronoi_n) * dim * sizeof(Real) : 0;
    site_bytes = (site_bytes + 255) / 256 * 256;
    VoronoiGrid vgrid;
    const bool has_grid = part.voronoi_n > 0 && build_voronoi_grid(d, part, &vgrid);
    const size_t gstart_bytes = has_grid ? (vgrid.start.size() * 4 + 255) / 256 * 256 : 0;
    const size_t grid_bytes = has_grid ? gstart_bytes + (vgrid.cand.size() * 4 + 255) / 256 * 256 : 0;
    const bool convert = sizeof(Real) != sizeof(double);
    size_t pts_bytes = convert ? size_t(M_D) * dim * sizeof(Real) : 0;
    size_t scratch_bytes = 256 + site_bytes + grid_bytes + pts_bytes;
    void *scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, scratch_bytes, stream);
    if (e != cudaSuccess) { delete pp; return cuda_status(e); }
    p.work = reinterpret_cast<unsigned long long *>(scratch);
    if (site_bytes) {
        std::vector<Real> sites(size_t(part.voronoi_n) * dim);
        for (size_t q = 0; q < sites.size(); ++q)
            sites[q] = Real(part.voronoi_sites[q]);
        Real *dsites = reinterpret_cast<Real *>(static_cast<char *>(scratch) + 256);
        cudaMemcpyAsync(dsites, sites.data(), sites.size() * sizeof(Real),
                        cudaMemcpyHostToDevice, stream);
        p.one.g.vsites = dsites;
    }
    if (has_grid) {
        char *gbase = static_cast<char *>(scratch) + 256 + site_bytes;
        int32_t *dstart = reinterpret_cast<int32_t *>(gbase);
        int32_t *dcand = reinterpret_cast<int32_t *>(gbase + gstart_bytes);
        cudaMemcpyAsync(dstart, vgrid.start.data(), vgrid.start.size() * 4,
                        cudaMemcpyHostToDevice, stream);
        if (!vgrid.cand.empty())
            cudaMemcpyAsync(dcand, vgrid.cand.data(), vgrid.cand.size() * 4,
                            cudaMemcpyHostToDevice, stream);
        set_voronoi_grid(vgrid, dstart, dcand, p.one.g);
    }
    cudaMemsetAsync(scratch, 0, 64, stream);
    e = launch_point_check(d, part, points, M_D, p.work, stream);
    count_launches(ctx, 1);
    if (e != cudaSuccess) {
        cudaFreeAsync(scratch, stream);
        delete pp;
        return cuda_status(e);
    }
    if (convert) {
        Real *dpts = reinterpret_cast<Real *>(static_cast<char *>(scratch) + 256 + site_bytes +
                                              grid_bytes);
        int n = M_D * dim;
        convert_points_kernel<Real><<<(n + 255) / 256, 256, 0, stream>>>(points, n, dpts);
        count_launches(ctx, 1);
        p.one.points_r = dpts;
    }
    if (!o.accumulate) {
        cudaMemsetAsync(counts, 0, size_t(M_D) * M * 4, stream);
        if (unterm)
            cudaMemsetAsync(unterm, 0, size_t(M_D) * 4, stream);
    }
    if (stats)
        cudaEventRecord(ctx->ev0, stream);
    if (o.kernel_events[0])
        cudaEventRecord(static_cast<cudaEvent_t>(o.kernel_events[0]), stream);
    void *args[] = {pp};
    e = cudaLaunchKernel(kfn, dim3(grid), dim3(block), args, smem, stream);
    count_launches(ctx, 1);
    if (o.kernel_events[1])
        cudaEventRecord(static_cast<cudaEvent_t>(o.kernel_events[1]), stream);
    if (stats)
        cudaEventRecord(ctx->ev1, stream);
    wos_status st = cuda_status(e);
    if (st == WOS_OK && stats) {
        unsigned long long w[6] = {0, 0, 0, 0, 0, 0};
        cudaMemcpyAsync(w, scratch, sizeof(w), cudaMemcpyDeviceToHost, stream);
        e = cudaStreamSynchronize(stream);
        st = cuda_status(e);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
        stats->steps = w[1];
        stats->walks = w[2];
        stats->unterminated = w[3];
        stats->max_steps = uint32_t(w[4]);
        stats->grid = grid;
        stats->block = block;
        stats->tile_walks = int32_t(tw);
        stats->hist_slots = nslot;
        stats->kernel_ms = ms;
        if (st == WOS_OK && w[5] > 0)
            st = WOS_POINT_OUTSIDE;
        else if (st == WOS_OK && w[3] > 0)
            st = WOS_STEP_CAP_HIT;
    }
    cudaFreeAsync(scratch, stream);
    delete pp;
    return st;
}

}  // namespace

extern "C" wos_status wos_build_operator(wos_context *ctx, const wos_domain *domain,
                                         const double *K, const double *points,
                                         int32_t M_D, const wos_partition *partition,
                                         uint32_t N, double eps, uint64_t seed,
                                         const wos_opts *opts, uint32_t *counts,
                                         uint32_t *unterminated, wos_stats *stats,
                                         void *stream)
{
    wos_opts o;
    double S[9];
    const wos_status st = validate_build(ctx, domain, K, points, M_D, partition, N, eps, opts,
                                         counts, &o, S);
    if (st != WOS_OK)
        return st;
    cudaSetDevice(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (o.precision == WOS_FP64)
        return build_impl<double>(ctx, *domain, *partition, S, points, M_D, N, eps,
                                  seed, o, counts, unterminated, stats, s);
    return build_impl<float>(ctx, *domain, *partition, S, points, M_D, N, eps, seed,
                             o, counts, unterminated, stats, s);
}

extern "C" wos_status wos_truncation_gap(const double *S, int32_t k, int32_t r)
{
    if (!S || k < 1 || r < 1 || r > k)
        return WOS_INVALID_ARG;
    if (r == k)
        return WOS_OK;
    if (!(S[r] > 0.0))
        return WOS_OK;
    return S[r - 1] / S[r] >= 1.5 ? WOS_OK : WOS_TRUNCATION_IN_CLUSTER;
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
extern "C" wos_status wos_autotune_reset(wos_context *ctx)
{
    if (!ctx)
        return WOS_INVALID_ARG;
    std::lock_guard<std::mutex> lock(ctx->tune_mu);
    ctx->tuned.clear();
    return WOS_OK;
}

extern "C" wos_status wos_autotune(wos_context *ctx, const wos_problem *sp, uint64_t seed,
                                   int32_t precision, uint64_t sample_walks, wos_tuning *out,
                                   void *stream)
{
    if (!ctx || !sp || !out || sample_walks < 1 ||
        (precision != WOS_FP32 && precision != WOS_FP64))
        return WOS_INVALID_ARG;
    wos_status st = validate(sp->domain, sp->partition);
    if (st != WOS_OK)
        return st;
    if (sp->M_D < 1 || sp->N < 1 || !sp->points || !sp->counts)
        return WOS_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the sample: the first points, about sample_walks walks in all
    const int32_t md = std::min<int32_t>(sp->M_D, 256);
    const uint32_t nn = uint32_t(std::max<uint64_t>(
        1, std::min<uint64_t>(sp->N, sample_walks / uint64_t(md))));
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess)
        return WOS_CUDA_ERROR;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return WOS_CUDA_ERROR;
    }
    auto trial = [&](const wos_opts &cand, float *ms) -> wos_status {
        wos_opts o = cand;
        o.precision = precision;
        o.stream_id = sp->stream_id;
        o.step_cap = sp->step_cap;
        o.kernel_events[0] = e0;
        o.kernel_events[1] = e1;
        wos_status r = wos_build_operator(ctx, sp->domain, sp->K, sp->points, md, sp->partition,
                                          nn, sp->eps, seed, &o, sp->counts, nullptr, nullptr,
                                          stream);
        if (r != WOS_OK && r != WOS_STEP_CAP_HIT)
            return r;
        if (cudaStreamSynchronize(s) != cudaSuccess)
            return WOS_CUDA_ERROR;
        cudaEventElapsedTime(ms, e0, e1);
        return WOS_OK;
    };
    wos_opts best;
    std::memset(&best, 0, sizeof(best));
    best.block_size = 256;
    best.tiles_per_warp = 16;
    best.refill_min = 1;
    best.group_blocks = 0;  // the default for the class
    float best_ms = 0.f, ms = 0.f;
    int trials = 0;
    st = trial(best, &ms);  // warm-up
    if (st == WOS_OK)
        st = trial(best, &best_ms);
    const float default_ms = best_ms;
    trials = 1;
    auto consider = [&](int field, int value) {
        if (st != WOS_OK)
            return;
        wos_opts c = best;
        int *f = field == 0 ? &c.block_size : field == 1 ? &c.blocks_per_sm
               : field == 2 ? &c.tiles_per_warp : field == 3 ? &c.hist_slots
               : field == 4 ? &c.refill_min : &c.group_blocks;
        if (*f == value)
            return;
        *f = value;
        wos_status r = trial(c, &ms);
        ++trials;
        if (r == WOS_INVALID_ARG)
            return;  // configuration does not fit this device
        if (r != WOS_OK) {
            st = r;
            return;
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    };
    for (int v : {128}) consider(0, v);
    for (int v : {3, 2}) consider(1, v);
    for (int v : {4, 64}) consider(2, v);
    for (int v : {-1}) consider(3, v);
    for (int v : {4, 8}) consider(4, v);
    for (int v : {2, 4, 8}) consider(5, v);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != WOS_OK)
        return st;
    std::memset(out, 0, sizeof(*out));
    out->block_size = best.block_size;
    out->blocks_per_sm = best.blocks_per_sm;
    out->tiles_per_warp = best.tiles_per_warp;
    out->hist_slots = best.hist_slots;
    out->refill_min = best.refill_min;
    out->group_blocks = best.group_blocks;
    out->trials = trials;
    out->best_ms = best_ms;
    out->default_ms = default_ms;
    std::lock_guard<std::mutex> lock(ctx->tune_mu);
    ctx->tuned[tune_key(precision, sp->domain->dim, walk_kind(*sp->domain, *sp->partition))] =
        *out;
    return WOS_OK;
}
