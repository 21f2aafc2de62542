/*
 * oracle.h -- single-threaded CPU oracle for 3D-BBS (arxiv 2310.10023).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
 * and its Python binding) may include, link, load or call this code; only
 * the tests, the smoke check and the benchmark's CPU-baseline leg do.  It
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * What it computes, and where the paper defines it:
 *   - angular step delta(r)                              Sec. III-B, Eq. (2)
 *   - rotational step delta'(r_l), divisions a           Sec. III-D, Eq. (12), (14)
 *   - initial translation set                            Sec. III-B, Eq. (3)-(5)
 *   - per-level sparse hash voxel maps with dilation     Sec. III-C, Eq. (10)
 *   - node score = upper bound                           Sec. III-C, Eq. (11)
 *   - roto-translational branching                       Sec. III-D, Eq. (13)
 *   - best-first batched branch-and-bound                Sec. III-E, Algorithm 2
 *   - exhaustive search over the leaf set                Sec. III-B, Eq. (1)
 *
 * Floating point: the grid and the rotation matrices are FP64; the rotated
 * point and its floor are FP32 with a fixed operation order and no FMA
 * (compiled with -ffp-contract=off), because that FP32 value decides the
 * integer voxel key and both sides must take that decision in the same
 * precision.  Scores are exact integer counts.
 */
#ifndef BBS_ORACLE_H
#define BBS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* flag bits (numerically equal to the library's, defined independently) */
#define ORC_TRANSLATION_ONLY   0x1u  /* every level uses the level-0 angle grid, a = 1 */
#define ORC_LEAF_UNDILATED     0x2u  /* level 0 map is the plain occupancy, no dilation */
#define ORC_PRUNE_GE           0x4u  /* reserved: Algorithm 2's '<' pruning (not implemented) */
#define ORC_ANGLE_LOWER_EDGE   0x8u  /* angle of index c is W_min + c*delta' (not the segment centre) */
#define ORC_CHILD_LITERAL      0x10u /* rotational children a*c + j literally (Eq. (13)), not by segment nesting */
/* exact-bound mode (map flag): levels l >= 1 store {v - j, j in [-e, 1+e]^3},
 * e in 1..15 in bits 12..15, so that a node's score bounds every leaf below
 * it under rotation as well (see orc_exact_dilation) */
#define ORC_EXACT_BOUND        0x20u
/* depth-first batched order (Table I's DFS strategy): deepest level first,
 * then highest score (orc_localize only) */
#define ORC_SEARCH_DFS         0x40u
#define ORC_EXACT_E(flags)     ((int)(((flags) >> 12) & 15u))

#define ORC_MAX_LEVELS 16

/* return codes (numerically equal to the library's) */
#define ORC_OK          0
#define ORC_NOT_FOUND   1
#define ORC_EINVAL     -1
#define ORC_ENOMEM     -2
#define ORC_EKEYRANGE  -5

typedef struct {
    /* translation search range (m) and roll / pitch / yaw ranges (rad) */
    double lo[3], hi[3];
    double ang_lo[3], ang_hi[3];
} orc_ranges;

typedef struct {
    int    levels;          /* L; l_max = L - 1                              */
    double r;               /* finest voxel size (the float r widened)       */
    double d_max;           /* maximum scan range used by Eq. (2)            */
    uint32_t flags;
    double ang_lo[3], ang_range[3];
    double  delta[ORC_MAX_LEVELS];           /* delta(r_l), Eq. (2), clamped        */
    int64_t N[ORC_MAX_LEVELS][3];            /* angle segments per axis             */
    double  dprime[ORC_MAX_LEVELS][3];       /* delta'(r_l), Eq. (12)               */
    int64_t a[ORC_MAX_LEVELS][3];            /* divisions from level l to l-1, Eq. (14); a[0] unused */
    int64_t wmin[3], wmax[3];                /* initial translation indices at l_max, Eq. (3)-(5)    */
} orc_grid;

typedef struct orc_maps orc_maps;

typedef struct {
    int32_t status, found, best_score, num_points;
    int32_t node[7];
    double  pose[6];
    int64_t nodes_scored, probes, iterations, peak_frontier, parents_branched;
    double  ms_total;
    /* Sec. IV-A's check of the approximate rotational bound: of the children
     * scored while branching (initial set excluded), those scoring above
     * their parent, and the sum over them of (child - parent) / child */
    int64_t children_scored, bound_violations;
    double  bound_excess;
} orc_result;

/* ---- grid ------------------------------------------------------------- */
double orc_delta(double r, double d_max);
double orc_scan_dmax(const float* scan_xyz, int64_t k);
int  orc_grid_build(double r, int levels, double d_max, const orc_ranges* rg,
                    uint32_t flags, orc_grid* g);
double orc_angle(const orc_grid* g, int level, int axis, int64_t c);
/* The extra dilation e that makes every node's score an upper bound on its
 * leaves' scores under this grid for scan points of norm at most
 * scan_norm_max (exact-bound mode); -1 when no e can (the literal Eq. (13)
 * children) */
int orc_exact_dilation(const orc_grid* g, double scan_norm_max);
/* A = fl32(R(alpha, beta, gamma) / r) row-major, R = Rz(gamma) Ry(beta) Rx(alpha) */
void orc_rotation(const orc_grid* g, int level, int64_t ia, int64_t ib, int64_t ig, float A[9]);
int64_t orc_num_children(const orc_grid* g, const int32_t node[7]);
void orc_child_range(const orc_grid* g, int level, int axis, int64_t c, int64_t* lo, int64_t* hi);

/* ---- maps ------------------------------------------------------------- */
int  orc_maps_build(const float* xyz, int64_t n, float r, int levels, uint32_t flags,
                    orc_maps** out);
void orc_maps_free(orc_maps* m);
int  orc_maps_levels(const orc_maps* m);
int64_t orc_maps_count(const orc_maps* m, int level);
int64_t orc_maps_table_size(const orc_maps* m, int level);
int64_t orc_maps_collisions(const orc_maps* m, int level);
/* writes count*3 int32 keys in table order; returns the number written */
int64_t orc_maps_keys(const orc_maps* m, int level, int32_t* out, int64_t cap);
int  orc_maps_contains(const orc_maps* m, int level, int32_t vx, int32_t vy, int32_t vz);
void orc_maps_bbox(const orc_maps* m, double lo[3], double hi[3]);

/* ---- scores ------------------------------------------------------------ */
/* Eq. (11): number of scan points whose voxel key at the node's level is occupied */
int32_t orc_score(const orc_maps* m, const orc_grid* g, const float* scan, int64_t k,
                  const int32_t node[7]);
int  orc_score_nodes(const orc_maps* m, const orc_grid* g, const float* scan, int64_t k,
                     const int32_t* nodes, int64_t n, int32_t* scores);
/* all children of a parent in canonical order (alpha, beta, gamma, x, y, z);
 * writes up to cap nodes (7 ints each); returns the number of children */
int64_t orc_children(const orc_grid* g, const int32_t parent[7], int32_t* out_nodes, int64_t cap);

/* ---- search ------------------------------------------------------------ */
int  orc_localize(const orc_maps* m, const float* scan, int64_t k, const orc_ranges* rg,
                  double score_frac, int64_t batch, double d_max, uint32_t flags,
                  int64_t max_frontier, orc_result* res);
/* threads of the OpenMP build (n > 0 sets them); 1 for the plain build */
int  orc_threads(int n);
/* exhaustive max over the leaf set (all leaf translations of the grid's window,
 * all level-0 rotations); returns the max score, lexmin argmax in best_node */
int  orc_brute_force(const orc_maps* m, const orc_grid* g, const float* scan, int64_t k,
                     int32_t* best_score, int32_t best_node[7]);

#ifdef __cplusplus
}
#endif
#endif
