/*
 * wos_oracle.h -- the FP64 CPU oracle's own declarations.
 *
 * TEST INFRASTRUCTURE ONLY (see wos_oracle.c).  Nothing in the CUDA
 * library includes this header; the library declares its own types.
 */
#ifndef WOS_ORACLE_H
#define WOS_ORACLE_H

#include <stdint.h>

#define ORC_MAX_VERTS 64
#define ORC_MAX_HOLES 16
#define ORC_MAX_PLANES 64

enum { ORC_OUTER_SPHERE = 1, ORC_OUTER_BOX = 2, ORC_OUTER_POLYGON = 3 };

/* Domain D = outer body minus disjoint closed holes (discs / balls), and
 * the partition of dD into elements (cells of App. A, Ex. A.2 / A.3).
 * Element order: outer elements first, then hole 0, hole 1, ... */
typedef struct {
    int32_t dim;        /* 2 or 3 */
    int32_t outer_kind; /* ORC_OUTER_* */
    double center[3];   /* sphere / box centre */
    double radius;      /* sphere radius */
    double half[3];     /* box half-extents */
    int32_t n_vertices; /* polygon, counter-clockwise */
    double vertices[2 * ORC_MAX_VERTS];
    int32_t n_holes;
    double hole_center[ORC_MAX_HOLES][3];
    double hole_radius[ORC_MAX_HOLES];
    /* partition of the outer component */
    int32_t outer_m;      /* 2-D circle: arcs */
    double outer_theta0;  /* 2-D circle: start angle of arc 0 */
    int32_t edge_m[ORC_MAX_VERTS]; /* polygon / 2-D box: cells per edge */
    int32_t outer_nb, outer_ns;    /* 3-D sphere: z-bands x phi-sectors */
    int32_t face_n1, face_n2;      /* 3-D box: cells per face */
    /* partition of each hole */
    int32_t hole_m[ORC_MAX_HOLES];
    double hole_theta0[ORC_MAX_HOLES];
    int32_t hole_nb[ORC_MAX_HOLES];
    int32_t hole_ns[ORC_MAX_HOLES];
    /* extrinsic Voronoi sites (voronoi_n > 0 replaces the cells above) */
    int32_t voronoi_n;
    const double *voronoi_sites; /* voronoi_n x dim */
} orc_domain;

typedef struct {
    orc_domain dom;
    double S[9];        /* (K / lambda_max)^{1/2}, row-major d x d */
    double eps;         /* stopping shell width */
    uint64_t seed;      /* Philox key */
    uint32_t stream;    /* fourth Philox counter word */
    uint32_t N;         /* walks per point (walk id = i * N + k) */
    uint32_t step_cap;  /* walks reaching it are left unterminated */
    int32_t words_per_uniform; /* 1: 23-bit, 2: 53-bit uniforms */
    /* mapped = 1: walk-on-spheres in y = S^{-1} x, whose domain S^{-1} D is a
     * convex polytope: dist_y(y) = min_f (plane_d[f] - plane_n[f] . y);
     * mapped = 2: D a disc / ball minus disc / ball holes; the chain moves by
     * the radius of orc_quadric_radius (a lower bound of dist_y) */
    int32_t mapped;
    int32_t n_planes;
    double plane_n[ORC_MAX_PLANES][3];
    double plane_d[ORC_MAX_PLANES];
    double Sinv[9];     /* row-major d x d */
    double mu2;         /* lambda_min(S)^2 (mapped = 2) */
} orc_instance;

double orc_quadric_radius(const orc_instance *I, const double *x);

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]);
double orc_dist(const orc_domain *D, const double *x);
int orc_classify(const orc_domain *D, const double *x);
int orc_num_elements(const orc_domain *D);
int orc_outer_elements(const orc_domain *D);
int orc_hole_elements(const orc_domain *D, int h);
int orc_walk(const orc_instance *I, const double *x0, uint64_t walk,
             double *x_exit, uint32_t *nsteps);
int orc_walk_batch(const orc_instance *I, const double *x0,
                   const uint64_t *walks, int64_t n, double *x_exit,
                   int32_t *elem, uint32_t *nsteps);
int orc_build_counts(const orc_instance *I, const double *points, int32_t M_D,
                     uint32_t k0, uint32_t k1, uint32_t *counts,
                     uint32_t *unterminated, uint64_t *total_steps,
                     int32_t nthreads);
int orc_jacobi_svd(int32_t m, int32_t n, const double *B, double *U,
                   double *S, double *V, int32_t *sweeps);
int orc_setup_S(int32_t d, const double *K, double *S, double *lam_max);

#endif
