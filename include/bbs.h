/*
 * bbs.h -- C ABI of libbbs: GPU (sm_103a) batched best-first branch-and-bound
 * scan matching for global localization, after 3D-BBS (Aoki et al.,
 * arxiv 2310.10023).
 *
 * Problem (Sec. III-A): given a map point cloud M = {m_n} and a LiDAR scan
 * S = {s_k}, find the pose x = [x, y, z, roll, pitch, yaw] maximizing the
 * number of transformed scan points that fall into occupied map voxels
 * (Eq. (1), (11)).  The search is a tree over a pose grid (Sec. III-B/D),
 * explored best-first in batches (Sec. III-E, Algorithm 2); each node's score
 * is an exact integer count against a per-level dilated sparse hash voxel
 * map (Sec. III-C, Eq. (10)).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Return value: BBS_OK (0), BBS_NOT_FOUND (1: no leaf reached the score
 *   threshold, so Algorithm 2 has no match to return), or a negative
 *   error code.  Errors never abort the process; bbs_last_error() gives a
 *   thread-local description of the last failure on the calling thread.
 * - Point clouds are K x 3 float32, row-major (x, y, z), metres.
 * - is_device != 0: every pointer argument of the call (clouds, nodes,
 *   scores) is CUDA device memory on the current device; otherwise host
 *   memory.  The library only reads inputs during the call and never keeps
 *   a pointer to caller memory; results go to caller memory.
 * - Nodes are int32 x 7: (c_x, c_y, c_z, c_alpha, c_beta, c_gamma, c_l) as in
 *   Sec. III-C: translation index c at level l means a translation of
 *   c * 2^l * r metres; angle indices are segment indices of the level's
 *   roll / pitch / yaw grid (Eq. (12)); c_l is the level (0 = leaf).
 * - Work runs on opts->cuda_stream (NULL: the legacy default stream).  Calls
 *   return after their work completes on that stream.
 * - Thread safety: distinct handles are independent; one bbs_maps may be
 *   shared read-only by concurrent calls.
 */
#ifndef BBS_H
#define BBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define BBS_OK          0
#define BBS_NOT_FOUND   1
#define BBS_EINVAL     -1   /* bad argument: non-finite input, r <= 0, levels outside 1..16, ... */
#define BBS_ENOMEM     -2   /* device memory or frontier capacity exhausted                       */
#define BBS_ECUDA      -3   /* a CUDA runtime call failed                                         */
#define BBS_ETIMEOUT   -4   /* a bounded device wait or the iteration limit ran out               */
#define BBS_EKEYRANGE  -5   /* a voxel key or translation index beyond +-2^20 fine voxels         */
#define BBS_ECORRUPT   -6   /* an internal consistency check failed                               */
#define BBS_ECANCELED  -7   /* the request was cancelled (server)                                 */
#define BBS_PENDING     2   /* server: the request is queued or running                           */

/* ---- flags (bbs_build_maps and bbs_opts.flags) ------------------------- */
/* every level uses the level-0 angle grid and only translations branch
 * (Table I configurations (d)-(f)); the bound is then exact */
#define BBS_TRANSLATION_ONLY  0x1u
/* level 0 stores the plain occupancy without the dilation of Sec. III-C
 * (pass to bbs_build_maps) */
#define BBS_LEAF_UNDILATED    0x2u
/* reserved for Algorithm 2's '<' pruning; rejected with BBS_EINVAL */
#define BBS_PRUNE_GE          0x4u
/* angle of segment index c is W_min + c * delta' instead of the centre
 * W_min + (c + 1/2) * delta' */
#define BBS_ANGLE_LOWER_EDGE  0x8u
/* rotational children a*c + j literally as printed in Eq. (13) instead of
 * the finer segments whose centres lie inside the parent's segment */
#define BBS_CHILD_LITERAL     0x10u
/* exact-bound mode (pass BBS_EXACT_BOUND_E(e) to bbs_build_maps, e in 1..15):
 * every level above the leaves also stores the keys within e voxels around
 * its dilation ({v - j, j in [-e, 1 + e]^3} instead of {0,1}^3), which covers
 * the displacement of any scan point between a node's rotation and any leaf
 * rotation below it; each node's score then bounds its leaves' scores and the
 * search returns the exhaustive optimum under roto-translational branching
 * too.  bbs_localize refuses (BBS_EINVAL) a scan whose grid needs more than e
 * (bbs_exact_dilation gives the need; e = 3 suffices for the workloads here)
 * or the BBS_CHILD_LITERAL reading, under which no e bounds the children */
#define BBS_EXACT_BOUND       0x20u
#define BBS_EXACT_BOUND_E(e)  (BBS_EXACT_BOUND | ((uint32_t)(e) << 12))
/* depth-first batched order (Table I's DFS search strategy), for
 * bbs_localize_hostqueue: the frontier is kept per level and taken deepest
 * level first, then highest score, in whole (level, score) buckets until the
 * popped parents have b children; the best leaf found at the start of a round
 * sets best and the match (lexmin among its score) and every node at or below
 * best goes.  With an exact bound the score equals the best-first one; the
 * match may differ among equal scores.  bbs_localize and the server refuse it
 * (BBS_EINVAL). */
#define BBS_SEARCH_DFS        0x40u
/* time every launch of the scoring kernel with CUDA events on the call's
 * stream (bbs_result.score_ms); off by default */
#define BBS_TIME_KERNELS      0x100u
/* drive every search iteration from the host (one synchronization per
 * iteration) instead of the device-side loop of a captured CUDA graph;
 * results are identical, only the overhead differs */
#define BBS_HOST_DRIVEN       0x200u

#define BBS_MAX_LEVELS 16

typedef struct bbs_maps bbs_maps;      /* opaque: device-resident hash pyramid */

/* Search ranges (Sec. III-B, III-D): translation box [lo, hi] in metres and
 * roll / pitch / yaw ranges [ang_lo, ang_hi] in radians (index 0, 1, 2).  The
 * paper's defaults are the map's bounding box (bbs_maps_bbox), roll and pitch
 * (-0.02, 0.02) and yaw (0, 2 pi). */
typedef struct {
    double lo[3], hi[3];
    double ang_lo[3], ang_hi[3];
} bbs_ranges;

/* Search options; a zero field takes its default. */
typedef struct {
    double   score_frac;    /* threshold = ceil(score_frac * K); default 0.95 (Sec. IV)       */
    int64_t  batch;         /* b: children popped per iteration; default 10000 (Sec. IV)     */
    double   d_max;         /* maximum scan range for Eq. (2); default max_k |s_k|           */
    uint32_t flags;         /* BBS_* flags                                                   */
    void*    cuda_stream;   /* cudaStream_t to run on; NULL = legacy default stream          */
    int64_t  max_frontier;  /* largest frontier in nodes: the arrays start at up to 2^24 and  */
                            /* double as the search needs; default 2^30; BBS_ENOMEM beyond  */
} bbs_opts;

/* Result of a localization.  pose = x_c of the matched leaf (Sec. III-B):
 * translation c * r metres, angles of the level-0 grid. */
typedef struct {
    int32_t status;         /* same as the return value                                       */
    int32_t found;          /* 1 if a leaf reached the threshold                              */
    int32_t best_score;     /* score of the match, or threshold - 1 when not found            */
    int32_t num_points;     /* K                                                              */
    int32_t node[7];        /* matched leaf node                                              */
    double  pose[6];        /* x, y, z (m), roll, pitch, yaw (rad)                            */
    int64_t nodes_scored;   /* children and initial nodes scored                              */
    int64_t probes;         /* nodes_scored * K: point-probes                                 */
    int64_t iterations;     /* batched BnB iterations (Algorithm 2 batches)                   */
    int64_t peak_frontier;  /* largest frontier size seen                                     */
    int64_t parents_branched;
    double  ms_to_optimum;  /* call start to the end of the iteration that set the match      */
    double  ms_total;       /* call start to return                                           */
    /* phases after Table III: 0 set source point cloud (upload, d_max, grid,
     * rotation tables), 1 initial nodes calculation, 2 find best score,
     * 3 pop remaining queue, 4 result read-back */
    double  phase_ms[5];
    int64_t gathers;        /* brick probes issued by the scoring kernel: items x K           */
    int64_t launches;       /* kernels this call launched                                     */
    int64_t score_launches; /* launches of the scoring kernel                                 */
    double  score_ms;       /* their summed device time (BBS_TIME_KERNELS), else 0            */
    int64_t h2d_bytes;      /* host-to-device bytes the call copied                           */
    int64_t d2h_bytes;      /* device-to-host bytes the call copied                           */
    /* Sec. IV-A's check of the approximate rotational bound: children scored
     * while branching (the initial set excluded), those scoring above their
     * parent, and the sum over them of (child - parent) / child */
    int64_t children_scored;
    int64_t bound_violations;
    double  bound_excess;
    /* scan points the scoring kernel rotated: the tasks of a run share one
     * rotation (one evaluation of Eq. (11)'s R s per point for the run);
     * gathers / rotations is the average number of tasks sharing one */
    int64_t rotations;
} bbs_result;

/* bbs_pose_matrix -- the rigid transform of a result pose (x, y, z, roll,
 * pitch, yaw; Sec. III-A names the angles): R = Rz(yaw) Ry(pitch) Rx(roll),
 * row-major 3 x 3 in FP64, the composition the pose grid's rotations use,
 * and t = (x, y, z).  A scan point s maps to R s + t.  Host memory; feeds
 * bbs_gicp's (R0, t0).  BBS_EINVAL for a NULL argument or a non-finite pose. */
int  bbs_pose_matrix(const double pose[6], double R[9], double t[3]);

/* ---- maps: Sec. III-C ---------------------------------------------------
 * bbs_build_maps -- build the per-level voxel maps H^l on the current device.
 *   xyz, n    : map cloud (n x 3 float32), host or device per is_device.
 *   r         : finest voxel size r (m), > 0.  Level l has voxel size 2^l r.
 *   levels    : L in 1..16 (l_max = L - 1).
 *   flags     : BBS_LEAF_UNDILATED or 0.
 *   stream    : cudaStream_t or NULL.
 *   out       : receives the handle; owned by the caller until bbs_free_maps.
 * Level l holds every voxel floor(u / 2^l) - j, j in {0,1}^3, for each map
 * point's fine key u = floor(fl32(m * fl32(1/r))) (the dilation of the last
 * paragraph of Sec. III-C; level 0 undilated with BBS_LEAF_UNDILATED).
 * Errors: BBS_EINVAL (non-finite point, r <= 0, bad levels, n < 0),
 * BBS_EKEYRANGE (a fine key with |u| > 2^20 - 4), BBS_ENOMEM, BBS_ECUDA. */
int  bbs_build_maps(const float* xyz, int64_t n, int is_device, float r, int levels,
                    uint32_t flags, void* cuda_stream, bbs_maps** out);
void bbs_free_maps(bbs_maps* maps);

/* Map bounding box of the input cloud (the paper's default translation range). */
int  bbs_maps_bbox(const bbs_maps* maps, double lo[3], double hi[3]);

/* Statistics of level `level`: stored voxels |H^l|, buckets (4^3-voxel
 * bricks) in use, buckets in the table (T_l; for a dense level every brick of
 * its box and one zero brick), longest probe sequence, and the fraction of buckets not in their
 * home slot (the collision rate of Sec. III-C; 0 for a dense level). */
int  bbs_maps_info(const bbs_maps* maps, int level, int64_t* n_voxels, int64_t* n_buckets,
                   int64_t* table_size, int32_t* max_probe, double* collision_rate);

/* Layout of level `level`'s table: BBS_LAYOUT_WIDE, BBS_LAYOUT_COMPACT,
 * BBS_LAYOUT_DENSE or BBS_LAYOUT_BYTES (see bbs_set_probe_layout).  BBS_EINVAL for a bad handle
 * or level. */
#define BBS_LAYOUT_WIDE    0
#define BBS_LAYOUT_COMPACT 1
#define BBS_LAYOUT_DENSE   2
#define BBS_LAYOUT_BYTES   3
int  bbs_maps_layout(const bbs_maps* maps, int level, int32_t* layout);

/* bbs_maps_device -- the CUDA device holding the maps' tables (the device
 * current when bbs_build_maps ran).  BBS_EINVAL for a NULL argument. */
int  bbs_maps_device(const bbs_maps* maps, int32_t* device);

/* Target load (buckets in use / buckets) of the hashed level tables built by
 * later bbs_build_maps calls in this process (byte grids and dense bricks
 * have none); default 0.25.  Sec. III-C enlarges
 * T_l until few keys collide; the load trades the collision rate (probe
 * length) against the table's footprint in L2.  BBS_EINVAL outside
 * (0.01, 0.9]. */
int  bbs_set_load_factor(double load);

/* Bucket layout of the tables built by later bbs_build_maps calls in this
 * process (scores never depend on it):
 *   0 (default)  byte grid -- one byte per key of the level's key box holding
 *                the 8 child bits of that key (Eq. (13) children), one 1-byte
 *                load per query -- where the box spans at most 2^24 4^3-key
 *                bricks, at most 64 x the occupied bricks + 2^16, and under
 *                2^20 keys per axis; else compact -- a 32-bit key relative to
 *                the box, one 16-byte load per probe -- where the box fits
 *                8192 x 8192 x 4092 keys; else wide (64-bit key, 32-byte
 *                probe);
 *   1            always wide;
 *   2            hashed only: compact where it fits, else wide;
 *   3            dense bricks where the box qualifies: every brick of the
 *                box at a computed index, no key, one 16-byte load per query;
 *                else hashed;
 *   4            byte grid where the box qualifies, else hashed.
 * BBS_EINVAL for any other value. */
int  bbs_set_probe_layout(int layout);

/* Launch shape of the search, for every engine and launch made after the
 * call (results never depend on it).  Zero fields take the defaults:
 *   launch_tasks  most rotational-child tasks per scoring launch, 1..2^19
 *                 (default 2^19); a round with more is scored in several
 *                 launches planned on the host;
 *   static_pm     per-mille of a launch's (task, 512-point block) slices split
 *                 evenly over the scoring CTAs before the rest is handed out
 *                 in shrinking grabs, 1..1000 (default 750; a launch of fewer
 *                 than 256 slices per CTA is split statically);
 *   grab_min      smallest grab in slices, 1..2^20 (default 16);
 *   ctas_per_sm   scoring CTAs per SM, 1..4 (default 4);
 *   frontier_log2 the frontier arrays of later bbs_localize and
 *                 bbs_localize_many calls start at 2^frontier_log2 nodes,
 *                 10..30, and double as a search needs (default: up to 2^24
 *                 nodes plus room for one round).
 * NULL restores every default.  BBS_EINVAL for a field out of range. */
typedef struct {
    int64_t launch_tasks;
    int32_t static_pm;
    int32_t grab_min;
    int32_t ctas_per_sm;
    int32_t frontier_log2;
} bbs_tuning;
int  bbs_set_tuning(const bbs_tuning* t);
/* The tuning in effect (defaults filled in). */
int  bbs_get_tuning(bbs_tuning* t);

/* bbs_launch_log -- the scoring launches of the last search call on this
 * thread that ran with BBS_TIME_KERNELS: per launch its units (rotational
 * children x scan points, each unit scoring 8 translational children) and
 * its device milliseconds between CUDA events on the call's stream.  units
 * and ms: host arrays of cap entries; *n receives the count (a size query
 * with cap = 0 returns BBS_OK when the log is empty, else BBS_EINVAL with *n
 * set).  The paper has no counterpart: it serves the roofline measurement. */
int  bbs_launch_log(int64_t* units, double* ms, int64_t cap, int64_t* n);

/* All voxel keys of level `level` (n_voxels x 3 int32) into the host buffer
 * out (capacity cap keys); *n receives the count.  BBS_EINVAL if cap is short. */
int  bbs_maps_keys(const bbs_maps* maps, int level, int32_t* out, int64_t cap, int64_t* n);

/* The extra dilation the exact-bound mode needs for this scan and search
 * ranges (*e; -1 when no dilation can give the bound): over the levels
 * l >= 1, ceil((theta_l d / r + 2) / 2^l), where theta_l sums, over the three
 * axes and the levels 1..l, half a segment (a whole one with
 * BBS_ANGLE_LOWER_EDGE) -- how far a leaf's angles can lie from a level-l
 * node's -- and d is the larger of the scan's largest point norm and d_max. */
int  bbs_exact_dilation(const bbs_maps* maps, const float* scan_xyz, int64_t k, int is_device,
                        const bbs_ranges* ranges, const bbs_opts* opts, int32_t* e);

/* ---- pose grid: Sec. III-B Eq. (2)-(5), Sec. III-D Eq. (12)-(14) --------
 * Fills, for one (map, scan, ranges, opts) tuple and one level:
 *   dims[0..2]  : angle segments N_l for roll, pitch, yaw,
 *   dims[3..5]  : divisions a_l (Eq. (14); 1 at level 0),
 *   dims[6..11] : initial translation indices w_min[3], w_max[3] (Eq. (3)-(5)),
 * and, if A_out is not NULL, the N_alpha N_beta N_gamma scaled rotation
 * matrices A = fl32(R(alpha, beta, gamma) / r), R = Rz(gamma) Ry(beta) Rx(alpha),
 * row-major 9 floats each, rotation index (i_a N_b + i_b) N_g + i_g, into the
 * host buffer A_out (capacity cap matrices).  *n_rot receives N_a N_b N_g. */
int  bbs_pose_grid(const bbs_maps* maps, const float* scan_xyz, int64_t k, int is_device,
                   const bbs_ranges* ranges, const bbs_opts* opts, int level, int64_t* dims,
                   float* A_out, int64_t cap, int64_t* n_rot);

/* ---- scores: Sec. III-C Eq. (11) ------------------------------------------
 * bbs_score_batch -- score(c) = #{k : key_{c_l}(T_{x_c} s_k) in H^{c_l}} for n
 * caller nodes.  nodes: n x 7 int32; scores: n int32 (both host or both
 * device, per is_device).  The fine key of s under node c is
 * u = floor(fl32(A s)) with FP32 products and sums in the order
 * ((A_i0 s_x + A_i1 s_y) + A_i2 s_z), no FMA; the level key is
 * floor((u + c 2^l) / 2^l).  Errors: BBS_EINVAL for a node outside the grid
 * (level, angle index) or with |c 2^l| > 2^20, or bad scan points. */
int  bbs_score_batch(const bbs_maps* maps, const float* scan_xyz, int64_t k, int is_device,
                     const bbs_ranges* ranges, const bbs_opts* opts, const int32_t* nodes,
                     int64_t n, int32_t* scores);

/* bbs_score_children -- branch (Eq. (13)) and score every child of n parent
 * nodes with the fused branch-and-score kernel of the search.  Writes, per
 * parent in order, its children in the order (alpha, beta, gamma, x, y, z)
 * into child_nodes (cap x 7 int32) and child_scores (cap int32); *n_children
 * receives the total.  Leaves (level 0) have no children.  Pointers follow
 * is_device; the output buffers may be NULL with cap = 0 (a size query:
 * *n_children is set and BBS_EINVAL returned when there are children).
 * BBS_EINVAL if cap is short, an output buffer is NULL, or a parent is
 * outside the grid. */
int  bbs_score_children(const bbs_maps* maps, const float* scan_xyz, int64_t k, int is_device,
                        const bbs_ranges* ranges, const bbs_opts* opts, const int32_t* parents,
                        int64_t n, int32_t* child_nodes, int32_t* child_scores, int64_t cap,
                        int64_t* n_children);

/* ---- scores without allocation ---------------------------------------------
 * bbs_score_batch_noalloc -- the scores of bbs_score_batch for callers that
 * cannot allocate memory while they run: real-time control loops that must
 * not touch an allocator after start-up (unbounded latency, fragmentation),
 * frameworks that own all device memory through their own pool, and servers
 * that budget every byte up front.  The paper has no counterpart.
 *   scan_xyz, nodes, scores : DEVICE memory on the maps' device (k x 3 float32,
 *                             n x 7 int32, n int32), as in bbs_score_batch;
 *                             any other pointer is BBS_EINVAL (checked with
 *                             cudaPointerGetAttributes, which allocates nothing).
 * It calls no cudaMalloc/cudaFree and no allocating routine; its scratch
 * (the packed scan and the angle cosines/sines) is one file-scope device
 * array of 3 MiB + 4 KiB that every GPU loading the library keeps until the
 * process exits.  Limits: k <= BBS_NOALLOC_MAX_POINTS and at most
 * BBS_NOALLOC_MAX_ANGLES angle segments summed over levels and axes, both
 * BBS_EINVAL beyond.  Bad arguments and k above the maximum are refused before
 * any GPU work; the angle-segment limit and non-finite or too large scan
 * coordinates are found after the scan has been packed into the array.  All
 * calls share the array and it keeps the last call's contents (the status
 * words are cleared at the start of each call), so calls that overlap on the
 * GPU race; a process-wide lock held until each call's final stream
 * synchronization keeps calls through this library from overlapping.  The
 * call synchronizes its stream (the scan's d_max is read back before the pose
 * grid is formed).  The first call on a device looks up the array's device
 * address with that device current; make it before any stream capture.
 * Same errors as bbs_score_batch. */
#define BBS_NOALLOC_MAX_POINTS 131072
#define BBS_NOALLOC_MAX_ANGLES 65536
int  bbs_score_batch_noalloc(const bbs_maps* maps, const float* scan_xyz, int64_t k,
                             const bbs_ranges* ranges, const bbs_opts* opts, const int32_t* nodes,
                             int64_t n, int32_t* scores);

/* ---- search: Sec. III-E, Algorithm 2 ---------------------------------------
 * bbs_localize -- global localization of one scan.  Canonical batched
 * best-first iteration: best = ceil(theta K) - 1; the frontier F holds scored
 * nodes bucketed by score; each iteration pops whole top buckets until the
 * popped parents have at least b children, a bucket at or below best clears
 * F, a bucket holding a leaf sets best and the match (lexicographic minimum
 * leaf of that bucket) and clears F; the popped parents are branched
 * (Eq. (13)) and children scoring above best join F.  ranges NULL: map
 * bounding box, roll/pitch (-0.02, 0.02), yaw (0, 2 pi).  opts may be NULL.
 * K is at most 2^24 - 2 (BBS_EINVAL beyond).
 * Returns BBS_OK, BBS_NOT_FOUND, or an error (also in out->status). */
int  bbs_localize(const bbs_maps* maps, const float* scan_xyz, int64_t k, int is_device,
                  const bbs_ranges* ranges, const bbs_opts* opts, bbs_result* out);

/* bbs_localize with the frontier kept on the host, as Algorithm 2 lays it
 * out (Sec. III-E): a host priority structure; per batch the popped parents'
 * rotational children are copied to the GPU, scored by the same kernels, and
 * their children's scores copied back for the host to keep those above best.
 * Same canonical iteration, so the same results as bbs_localize; it measures
 * what keeping the frontier on the device buys.  With BBS_SEARCH_DFS in
 * opts->flags it runs the depth-first order instead (Table I's DFS). */
int  bbs_localize_hostqueue(const bbs_maps* maps, const float* scan_xyz, int64_t k, int is_device,
                            const bbs_ranges* ranges, const bbs_opts* opts, bbs_result* out);

/* ---- local fine registration (GICP) after the BnB result --------------------
 *
 * Sec. IV seeds a generalized-ICP refinement with the BnB estimate; the
 * paper fixes none of its internals, so these are the library's readings:
 * the target is the map cloud grouped by fine voxel key
 * u = floor(fl32(x fl32(1/r))) (the level-0 quantization), voxel u standing
 * for the centroid of its points (sums of rint((x - u r) 2^32) in integers:
 * exact and independent of order); a scan point p = R s + t corresponds to
 * the nearest centroid of the occupied voxels of the 3 x 3 x 3 block around
 * floor(p / r) (ties to the first in (dx, dy, dz) order), kept within tau;
 * covariances are normalized, r^2 (S / tr S + eps I) with S the sample
 * covariance of the centroids of the block around the target voxel, or of
 * the scan points within rho of the scan point (r^2 I when S = 0);
 * Gauss-Newton on sum d^T (C_t + R C_s R^T)^-1 d, d = centroid - p, with
 * steps p -> Exp(w) p + v, until |w| < eps_rot and |v| < eps_trans or
 * max_iters linearizations.  Transformed coordinates and distances are
 * formed in FP64 with every operation rounded on its own. */
typedef struct bbs_gicp_target bbs_gicp_target;   /* opaque: device-resident voxel centroids */

/* Build the target from a map cloud (n x 3 float, host or device) at voxel
 * size r.  BBS_EINVAL (n < 1, r <= 0, non-finite point), BBS_EKEYRANGE (a key
 * beyond +-2^20), BBS_ENOMEM, BBS_ECUDA. */
int  bbs_gicp_target_build(const float* xyz, int64_t n, int is_device, float r, void* cuda_stream,
                           bbs_gicp_target** out);
void bbs_gicp_target_free(bbs_gicp_target* target);
/* occupied voxels, hash table slots, longest probe */
int  bbs_gicp_target_info(const bbs_gicp_target* target, int64_t* n_voxels, int64_t* table_size,
                          int32_t* max_probe);

typedef struct {
    int32_t max_iters;      /* linearizations (0: 30)                            */
    int32_t pad;
    double  tau;            /* correspondence distance, m (0: r)                 */
    double  rho;            /* source neighbourhood radius, m (0: 2 r)           */
    double  cov_eps;        /* covariance regularization (0: 1e-3)               */
    double  eps_rot;        /* convergence on the step's rotation, rad (0: 1e-6) */
    double  eps_trans;      /* and translation, m (0: 1e-6)                      */
    void*   cuda_stream;
} bbs_gicp_opts;

typedef struct {
    int32_t status;           /* BBS_OK or an error                              */
    int32_t converged;        /* the last step was below both tolerances         */
    int32_t iterations;       /* linearizations made                             */
    int32_t correspondences;  /* kept at the last linearization (< 6 stops)      */
    double  cost;             /* sum d^T M d at the last linearization           */
    double  R[9], t[3];       /* refined pose: map point = R scan point + t      */
    double  pose[6];          /* x, y, z, roll, pitch, yaw of (R, t), R = Rz Ry Rx */
    double  ms;               /* wall time of the call                           */
} bbs_gicp_result;

/* Refine the pose (R0 row-major, t0) of a scan (k x 3 float, host or
 * device).  BBS_EINVAL for k < 1, NULL arguments or non-finite options. */
int  bbs_gicp(const bbs_gicp_target* target, const float* scan_xyz, int64_t k, int is_device, const double R0[9],
              const double t0[3], const bbs_gicp_opts* opts, bbs_gicp_result* out);

/* One linearization at (R, t): H (6 x 6 row-major, parameters w then v),
 * g = sum J^T M d, cost, correspondences kept; with voxels (k x 3 int32) and
 * found (k bytes) both non-NULL, each point's nearest block voxel and
 * whether it was kept (host memory). */
int  bbs_gicp_linearize(const bbs_gicp_target* target, const float* scan_xyz, int64_t k, int is_device,
                        const double R[9], const double t[3], const bbs_gicp_opts* opts, double H[36], double g[6],
                        double* cost, int64_t* n, int32_t* voxels, uint8_t* found);

/* ---- measurement ----------------------------------------------------------
 * bbs_bench_gather -- device time (ms, CUDA events on cuda_stream) of
 * `gathers` random 32-byte bucket reads, issued as the scoring kernel's probes
 * issue them, over a table of table_bytes (rounded down to a power of two
 * buckets, at least 1 KiB).  Small tables stay in L2 and give the L2 gather
 * roofline; tables well above L2 give the HBM one.  The call allocates and
 * frees its own table. */
int  bbs_bench_gather(int64_t table_bytes, int64_t gathers, void* cuda_stream, double* ms_out);

/* bbs_localize_many -- n independent localizations against one map, advanced
 * together: every iteration pops one canonical batch from each live search
 * and scores the children of all of them in shared launches (the scans may
 * have different sizes).  scans[i] points to ks[i] x 3 float32 (host or
 * device per is_device); out[i] receives scan i's result, identical to what
 * bbs_localize returns for it alone (same best score, match, iterations and
 * nodes scored; times and launch counts are those of the shared run).  The
 * frontier capacity opts->max_frontier is shared by all n searches.  At most
 * 256 searches advance together (n <= 4096): the others take the slots of
 * searches that finish, between iterations.  Returns BBS_OK when every search
 * ran (each out[i].status tells found / not found), or an error for the whole
 * call. */
int  bbs_localize_many(const bbs_maps* maps, int n, const float* const* scans, const int64_t* ks,
                       int is_device, const bbs_ranges* ranges, const bbs_opts* opts, bbs_result* out);

/* ---- serving: continuous batching --------------------------------------------
 * A server owns a worker thread, a CUDA stream and a search engine on the
 * device current at bbs_server_create.  Requests (a map handle, a host scan
 * that is copied at submission, ranges, options) queue up; between search
 * iterations the worker admits them in arrival order into free search slots
 * while the device-memory budget allows (the shared frontier pool is charged
 * once; each admitted search its scan, rotation tables and frontier arrays),
 * so a request that arrives while others run joins the next iteration and
 * shares its launches.  Finished searches release their slot and memory
 * immediately.  Each result equals what bbs_localize returns for the same
 * request alone (times excepted: ms_total is submission to result).
 * Requests whose memory estimate exceeds the whole budget finish at once
 * with BBS_ENOMEM.  opts->cuda_stream and BBS_TIME_KERNELS are ignored. */
typedef struct bbs_server bbs_server;

typedef struct {
    size_t  mem_budget;     /* device bytes for the pool plus admitted searches; 0 = 8 GiB  */
    int32_t max_active;     /* searches advanced together; 0 = 32, at most 256              */
    int64_t max_frontier;   /* shared frontier pool in nodes; 0 = 2^24                      */
} bbs_server_opts;

typedef struct {
    int64_t submitted, completed, active, queued, rejected;
    int64_t peak_active;               /* most searches advanced in one iteration            */
    double  p50_ms, p99_ms, mean_ms;   /* submission-to-result latency of completed requests */
    double  throughput_rps;            /* completed / (last completion - first submission)   */
    double  probes_per_s;              /* point-probes of completed requests over that span  */
    size_t  mem_in_use, mem_budget;
} bbs_server_counters;

int  bbs_server_create(const bbs_server_opts* opts, bbs_server** out);
/* queue a request; *ticket identifies it.  BBS_OK once queued. */
int  bbs_server_submit(bbs_server* server, const bbs_maps* maps, const float* scan_xyz, int64_t k,
                       const bbs_ranges* ranges, const bbs_opts* opts, uint64_t* ticket);
/* wait up to wait_ms (0: do not wait, negative: until done) for a ticket.
 * Returns BBS_PENDING while queued or running; otherwise the request's status
 * (BBS_OK, BBS_NOT_FOUND or an error), with its result in *out, and forgets
 * the ticket: a later poll of it (or of a ticket never issued) returns
 * BBS_EINVAL at once.  The maps handle of a request must stay alive until its
 * result has been polled. */
int  bbs_server_poll(bbs_server* server, uint64_t ticket, int wait_ms, bbs_result* out);
/* cancel a queued or running request; its result reports BBS_ECANCELED */
int  bbs_server_cancel(bbs_server* server, uint64_t ticket);
int  bbs_server_stats(bbs_server* server, bbs_server_counters* out);
/* stops the worker after its current iteration; unfinished requests are dropped */
void bbs_server_destroy(bbs_server* server);

/* Thread-local description of the last error on this thread ("" if none). */
const char* bbs_last_error(void);

/* Library version string. */
const char* bbs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BBS_H */
