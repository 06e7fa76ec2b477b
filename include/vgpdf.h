/*
 * vgpdf.h -- C ABI of the GB300 library for batched local Gaussian-process distance fields
 * (the data-parallel hot path of VDB-GPDF, Wu, Le Gentil and Vidal-Calleja, arXiv 2407.09649).
 *
 * The library keeps a sparse voxel map on one GPU: a hash of 8^3-voxel leaves replacing the
 * paper's OpenVDB trees (Sec. III-B).  Three entry points carry the method:
 *
 *   vgp_build_frame              L-GPDF of one frame (Sec. IV-A/B): voxelise the points,
 *                                one GP per occupied leaf trained on voxel centres, distance
 *                                and variance inferred at every testing voxel;
 *   vgp_fuse                     probabilistic fusion of a frame into the global grid
 *                                (Sec. IV-C, Eqs. 7-8, or Eq. 9);
 *   vgp_query_distance_gradient  G-GPDF queries (Sec. IV-D): per query leaf a GP over the
 *                                surface points of its 27-leaf neighbourhood, trained lazily
 *                                for the leaves that queries touch; distance, gradient and
 *                                variance at arbitrary points.
 *
 * plus vgp_query_backward (derivatives of the distance w.r.t. query and surface points),
 * vgp_gp_batch (independent GP instances given directly) and grid export/import.
 *
 * Every GP uses the unscaled SE kernel k(x, x') = exp(-|x - x'|^2 / (2 l^2)) (Sec. III-A),
 * A = K + sigma^2 I, alpha = A^-1 1 (Eq. 1), latent variance u = 1 - k^T A^-1 k (Eq. 2, read
 * as the standard GP posterior), latent gradient (Eq. 5), reverting d = sqrt(-2 l^2 log o)
 * (Eq. 3), distance variance v = Lambda^2 u, Lambda = -l^2 / (o d) (Eq. 4), and the
 * chain-rule distance gradient grad d = -l^2 grad o / (o d).
 *
 * Conventions, for every function below:
 *   - Pointers named *_dev are device memory on the map's GPU, owned by the caller, which
 *     must keep them alive until the stream has passed the call.  Host pointers are named
 *     without that suffix.  The library owns vgp_map and vgp_frame and their device memory.
 *   - Point arrays are float32, row-major [n][3] (x, y, z in metres, world frame).
 *   - Calls enqueue work on `stream` (a cudaStream_t; NULL is the legacy default stream)
 *     and return once it is enqueued.  Some calls read a few sizes back from the GPU and so
 *     synchronise the stream part-way (noted per call).  Read outputs after a stream sync
 *     or vgp_sync().
 *   - Return value: VGP_OK (0) or a negative VGP_ERR_* code; vgp_last_error() then gives a
 *     thread-local message.  On error, outputs are unspecified and the map stays usable
 *     unless the code is VGP_ERR_CUDA.
 *   - A map and its frames may be used from one host thread at a time.
 *   - Per-query status: VGP_ST_OK, VGP_ST_NO_SUPPORT (no surface point within the leaf
 *     search radius), VGP_ST_CLAMPED (o <= 0 or log o below the floor: d = d_max),
 *     VGP_ST_BAD_INPUT (non-finite or out-of-range coordinate), VGP_ST_FACTOR_FAIL
 *     (non-positive Cholesky pivot).  For NO_SUPPORT, BAD_INPUT and FACTOR_FAIL:
 *     d = +inf, grad = 0, var = +inf.  For CLAMPED: d = d_max, grad = 0, var = +inf.
 *     For o >= 1 (on or inside the surface): status OK, d = 0, grad = 0.
 */
#ifndef VGPDF_H
#define VGPDF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vgp_map vgp_map;
typedef struct vgp_frame vgp_frame;
typedef struct vgp_mesh vgp_mesh;
typedef void* vgp_stream; /* cudaStream_t */

enum {
    VGP_OK = 0,
    VGP_ERR_ARG = -1,        /* invalid argument or unsupported size */
    VGP_ERR_OOM = -2,        /* device or host allocation failed */
    VGP_ERR_CUDA = -3,       /* a CUDA call failed (message has the CUDA error) */
    VGP_ERR_TABLE_FULL = -4, /* a hash table ran out of slots (bounded probe) */
    VGP_ERR_TIMEOUT = -5,    /* a bounded device-side loop hit its limit */
    VGP_ERR_STATE = -6       /* call out of order (e.g. query before set_surface) */
};

enum { VGP_FP64 = 0, VGP_MIXED = 1 };          /* precision */
enum { VGP_FUSE_INVVAR = 0, VGP_FUSE_TSDF = 1 }; /* fusion rule: Eq. 8 or Eq. 9 */
enum { VGP_LAUNCH_BATCHED = 0, VGP_LAUNCH_PER_INSTANCE = 1, VGP_LAUNCH_GRAPH = 2 };
enum {
    VGP_ST_OK = 0,
    VGP_ST_NO_SUPPORT = 1,
    VGP_ST_CLAMPED = 2,
    VGP_ST_BAD_INPUT = 3,
    VGP_ST_FACTOR_FAIL = 4
};

/*
 * Map parameters.  Defaults (vgp_default_params): voxel 0.1 m, l = 0.3 m (about three
 * voxels, Sec. V: l spanning 2-4 voxels), sigma_occ = 0.01 (std of the latent occupancy
 * noise; sigma^2 is added to diag K, Eq. 1), d_max = 10 m, d_var_floor = 1e-3 m,
 * max_pts_leaf = 64, max_pts_group = 1024, max_leaf_search = 8, fusion = VGP_FUSE_INVVAR,
 * precision = VGP_MIXED.
 *
 *   voxel_size       voxel edge (m); leaves are 8^3 voxels (Sec. III-B).
 *   lengthscale      SE kernel length scale l (m).
 *   sigma_occ        latent noise std (unitless occupancy).
 *   d_max            distance cap: log o is floored at -d_max^2 / (2 l^2) (footnote of
 *                    Sec. III-A: the occupancy is capped; the cap value is ours).
 *   d_var_floor      lower bound on d inside Lambda (m).
 *   max_pts_leaf     L-GPDF training cap per leaf: a leaf with n > cap occupied voxels keeps
 *                    the voxels of rank floor(k n / cap), k = 0..cap-1, in bit order
 *                    (bit = x + 8 y + 64 z of the in-leaf offset).  1..512.
 *   max_pts_group    G-GPDF cap per neighbourhood: keeps the points nearest to the centre
 *                    leaf's centre (FP64 squared distance, ties to the lower point index).
 *                    1..1024.
 *   max_leaf_search  Chebyshev radius (in leaves) of the fallback search when a query's
 *                    27-leaf neighbourhood is empty.  0..16.
 *   fusion           VGP_FUSE_INVVAR (Eqs. 7-8) or VGP_FUSE_TSDF (Eq. 9, weight 1 - v).
 *   precision        VGP_FP64: every step in FP64.  VGP_MIXED: kernel values, latent mean
 *                    and gradient in FP32 (shifted by the nearest training point so they
 *                    cannot underflow); Cholesky, triangular solves, variance and the
 *                    reverting log in FP64.
 *   profile          0 (default) or 1: record CUDA events around the GP solve kernels and
 *                    report their time in vgp_stats.t_solve_ms (adds one stream sync per call).
 *   normal_steps     K in [0, 16] (default 3): with a sensor origin, vgp_build_frame also tests
 *                    the voxels round(s + k n), k = +-1..+-K, along each surface voxel's normal.
 *   emulate_fp64     1: instances with N > 32 (A in global memory) are factorised in blocks of
 *                    32 columns whose trailing updates run on the bf16 tensor cores to FP64
 *                    accuracy: each row of the block is cut into seven balanced base-256 digit
 *                    slices (55 bits under a power-of-two row scale), the slice products
 *                    accumulate exactly in FP32, and each update is packed exactly into an
 *                    integer and added to the not yet factorised matrix, held as 64-bit
 *                    integers round(v 2^61) (error of the order of the FP64 rounding of the
 *                    update).  In mixed precision their K entries are float-pair values (error
 *                    below 2^-45 k (1 + r^2 / 2l^2)), and off-lattice distance instances take
 *                    the latent variance from the Schur complement of the matrix with up to
 *                    1024 query rows appended.  Same results up to rounding; 0 keeps every
 *                    update on the FP64 tensor path.  Uses a per-CTA workspace of about
 *                    0.5 KB per matrix row and 8 bytes per lower-triangle entry.
 *   launch           VGP_LAUNCH_BATCHED (default): all GP instances of a call run in a few
 *                    persistent launches, one per size bucket, largest first.
 *                    VGP_LAUNCH_PER_INSTANCE: one kernel launch per instance, in instance
 *                    order (the plain comparison form; same arithmetic, no batching).
 *                    VGP_LAUNCH_GRAPH: the batched form with the size histogram, bucket
 *                    plan and ordering computed on the device, so that the whole solve of a
 *                    call (eight kernels) is captured as a CUDA graph on a stream the map
 *                    owns and replayed through a cached executable graph, updated in place
 *                    from call to call; the launch shapes are sized for the largest
 *                    instance the call can hold (max_pts_leaf for frames, max_pts_group for
 *                    queries).  Same arithmetic and results as VGP_LAUNCH_BATCHED; the caller's
 *                    stream waits on the map's stream through events.  The backward pass and
 *                    the autotuner always launch directly.
 */
typedef struct {
    double voxel_size;
    double lengthscale;
    double sigma_occ;
    double d_max;
    double d_var_floor;
    int32_t max_pts_leaf;
    int32_t max_pts_group;
    int32_t max_leaf_search;
    int32_t fusion;
    int32_t precision;
    int32_t profile;     /* nonzero: time the solve kernels with CUDA events (vgp_stats) */
    int32_t launch;      /* VGP_LAUNCH_BATCHED (0), VGP_LAUNCH_PER_INSTANCE (1) or VGP_LAUNCH_GRAPH (2) */
    int32_t normal_steps;/* ray-cast testing points: voxels along each surface normal, each side */
    double sigma_prop;   /* noise std of the surface-property GP (Eq. 6); default 0.1 */
    int32_t n_props;     /* surface-property channels per point, 0..4; default 0 */
    int32_t emulate_fp64;/* 0 (default) or 1: see below */
} vgp_params;

/* Counters of the most recent call on a map (host copy; informational). */
typedef struct {
    int64_t n_points;     /* valid input points (frame or surface) */
    int64_t n_leaves;     /* occupied leaves (frame) or surface leaves */
    int64_t n_instances;  /* GP instances solved */
    int64_t n_train;      /* sum of N over instances */
    int64_t n_queries;    /* queries or testing voxels evaluated */
    int64_t n_groups;     /* distinct query leaves (G-GPDF) */
    int64_t bucket_count[5]; /* instances per size bucket: N<=32, <=64, <=128, <=256, >256 */
    double sum_n3;        /* sum of N^3 over instances */
    double sum_n2;        /* sum of N^2 over instances */
    double t_solve_ms;    /* GP solve kernels (factorise + evaluate), if params.profile */
    double t_bucket_ms[5];   /* the same per size bucket */
    int32_t cfg_threads[5];  /* launch shape used per bucket: threads per CTA ... */
    int32_t cfg_per_sm[5];   /* ... and cap on CTAs per SM (0: occupancy limit) */
    int64_t grid_leaves;  /* leaves in the global grid */
    int64_t grid_capacity_leaves;
    int32_t cfg_stage_panel; /* N > 224 bucket: panel column staged in shared memory (1) or read
                                through L1/L2, leaving room for two CTAs per SM (0) */
    int32_t reserved;
    int64_t graph_replays;        /* VGP_LAUNCH_GRAPH: executable-graph launches on this map ... */
    int64_t graph_instantiations; /* ... and graph instantiations (the rest were updates in place) */
    /* with params.profile (CUDA events on the call's stream, 0 otherwise): */
    double t_bin_ms;        /* the voxelise / bin kernel of build_frame or set_surface (S1) */
    double t_gather_ms;     /* the neighbourhood gather kernel of a G-GPDF query (S3) */
    double t_fuse_ms;       /* the fusion kernels of the latest vgp_fuse (S9) */
    int64_t n_candidates;   /* candidate points the gather scanned, summed over instances */
} vgp_stats;

/* Fill *p with the defaults listed above. */
void vgp_default_params(vgp_params* p);

/* Create a map on the current CUDA device.  Validates *p (VGP_ERR_ARG on a bad value). */
int vgp_create(const vgp_params* p, vgp_map** out);

/* Destroy a map (synchronises its device work first).  NULL is a no-op. */
int vgp_destroy(vgp_map* m);

/*
 * L-GPDF of one frame (Sec. IV-A, IV-B; Eqs. 1-4).
 *   pts_dev  [n][3] float32 world-frame points (device).  Non-finite points and points with
 *            |p / voxel_size| >= 2^20 - 64 are ignored.  n >= 0 (n == 0 gives an empty frame).
 *   origin   host pointer to the sensor origin (3 doubles, world frame), or NULL.
 * Voxelises with ijk = floor(p / voxel_size + 1/2) (IEEE FP64) and builds one GP per occupied
 * leaf on its (capped) voxel centres.  Testing voxels:
 *   - origin == NULL: every voxel of every occupied leaf and of its 26 neighbour leaves;
 *     distances unsigned;
 *   - origin given (Sec. IV-B): the occupied voxels; the voxels round(s + k n),
 *     k = +-1..+-normal_steps, along the normal n of each occupied voxel s (smallest-eigenvalue
 *     eigenvector of the scatter of the occupied voxels in its 3x3x3 block, at least 3, oriented
 *     towards the origin); and the voxels on the integer 3D Bresenham line from the origin's
 *     voxel to each occupied voxel that already hold a value in the map's global grid.
 *     Distances and gradients are signed: + on the sensor side (occupied, ray, k > 0),
 *     - for k < 0 (a voxel reached with both signs is +).
 * Each testing voxel uses the GP of its own leaf if that leaf holds one, else of the neighbour
 * leaf whose centre is nearest (ties to the first in (dz, dy, dx) order from -1 to 1), else the
 * nearest GP leaf within max_leaf_search (ties to the smaller key), else status NO_SUPPORT.
 * On success *out receives a new frame (free with vgp_frame_destroy).  Synchronises the
 * stream several times to size its buffers.
 */
int vgp_build_frame(vgp_map* m, const float* pts_dev, int64_t n, const double* origin, vgp_stream stream,
                    vgp_frame** out);

/*
 * vgp_build_frame with surface properties (Eq. 6).  props_dev [n][params.n_props] float32
 * (device) holds each point's properties (e.g. intensity, colour channels); NULL behaves as
 * vgp_build_frame.  Each occupied voxel's property is the mean over its points (FP64 sums, in
 * an unspecified order); each leaf gets a second GP on the same training voxels with noise
 * sigma_prop, and every testing voxel, through the same node as its distance, gets
 *   c = k^T (K + sigma_prop^2 I)^-1 y     (Eq. 6, per channel, FP64)
 *   w = 1 - k^T (K + sigma_prop^2 I)^-1 k (posterior variance, read as for Eq. 2, FP64)
 * read with vgp_frame_props; c = NaN and w = +inf where the distance has no GP node or the
 * factorisation failed.  VGP_ERR_ARG if props_dev is given and the map has n_props = 0.
 */
int vgp_build_frame_props(vgp_map* m, const float* pts_dev, const float* props_dev, int64_t n,
                          const double* origin, vgp_stream stream, vgp_frame** out);

/*
 * Views of a frame's testing-voxel results (device pointers, owned by the frame, valid until
 * vgp_frame_destroy).  Arrays have *n_test entries in one common (unspecified) order:
 *   keys    voxel key: ((i + 2^20) << 42) | ((j + 2^20) << 21) | (k + 2^20)
 *   d, v    distance (m) and distance variance (m^2), FP64
 *   grad    [n_test][3] distance gradient, FP64
 *   status  VGP_ST_*
 * Any output pointer may be NULL.
 */
int vgp_frame_results(const vgp_frame* f, int64_t* n_test, const uint64_t** keys,
                      const double** d, const double** v, const double** grad,
                      const uint8_t** status);

/*
 * Views of a frame's GP instances (device pointers, owned by the frame), one per occupied
 * leaf, in an unspecified common order:
 *   leaf_key  packed leaf key (as voxel keys, of the leaf coordinates floor(ijk / 8))
 *   n_occ     occupied voxels of the leaf before the cap
 *   inst_off  [n_leaves + 1] int64 offsets into X / alpha
 *   X         [n_train][3] FP64 training voxel centres, world frame, in bit order
 *   alpha     [n_train] FP64 (K + sigma^2 I)^-1 1 of each leaf's GP (Eq. 1)
 * Any output pointer may be NULL.
 */
int vgp_frame_instances(const vgp_frame* f, int64_t* n_leaves, int64_t* n_train,
                        const uint64_t** leaf_key, const int32_t** n_occ,
                        const int64_t** inst_off, const double** X, const double** alpha);

/*
 * Surface-property results of a frame built by vgp_build_frame_props (device pointers owned
 * by the frame, in the order of vgp_frame_results): c [n_test][n_props], w [n_test].
 * *n_props = 0 (and NULL pointers) for a frame without properties.
 */
int vgp_frame_props(const vgp_frame* f, int32_t* n_props, const double** c, const double** w);

/* Free a frame (waits for its stream).  NULL is a no-op. */
int vgp_frame_destroy(vgp_frame* f);

/*
 * Fuse a frame into the map's global grid (Sec. IV-C).  For each testing voxel with status
 * OK, finite d and finite v > 0 (and v < 1 for Eq. 9): a first visit stores D = d, V = v
 * (Eq. 9: V = 1 - v); later visits apply Eqs. 7-8 (D = a d + b D, a = V / (V + v),
 * b = v / (V + v), V = (1/V + 1/v)^-1) or Eq. 9.  Leaves that receive a voxel are marked
 * active (flag bit 0: touched by this fuse, bit 1: ever touched).  Grows the grid as needed
 * (may synchronise the stream).  The frame must come from the same map.
 * Surface properties (a frame with properties on a map with n_props > 0; the last sentence
 * of Sec. IV-C): where a voxel's distance is fused and its c is finite and w valid (finite,
 * > 0, and < 1 for Eq. 9), the properties C (all channels) and their variance W are fused by
 * the same rules with w in place of v; a voxel's first property takes C = c, W = w (Eq. 9:
 * 1 - w).  Voxels without a fused property hold C = W = NaN.
 */
int vgp_fuse(vgp_map* m, vgp_frame* f, vgp_stream stream);

/*
 * Copy the global grid to host arrays sorted by voxel key: keys, D, V, and the flags of
 * the voxel's leaf.  Call with keys == NULL to get the count in *n; otherwise *n is the
 * capacity of the arrays on input and the count on output (VGP_ERR_ARG if too small).
 * Synchronises the stream.
 */
int vgp_export_grid(vgp_map* m, int64_t* n, uint64_t* keys, double* D, double* V,
                    uint8_t* flags, vgp_stream stream);

/*
 * Fused surface properties in the order of vgp_export_grid: C [n][n_props], W [n] (NaN where
 * none was fused).  Count query and capacity rules as for vgp_export_grid; *n = 0 when the
 * map has n_props = 0.  Synchronises the stream.
 */
int vgp_export_props(vgp_map* m, int64_t* n, uint64_t* keys, double* C, double* W, vgp_stream stream);

/*
 * Set the fused surface properties of voxels already in the grid (after vgp_import_grid;
 * host arrays in the export format).  Keys not in the grid are skipped.  VGP_ERR_STATE if the
 * map has n_props = 0.  Synchronises the stream.
 */
int vgp_import_props(vgp_map* m, int64_t n, const uint64_t* keys, const double* C, const double* W,
                     vgp_stream stream);

/* Replace the global grid by host arrays in the export format (checkpoint / resume). */
int vgp_import_grid(vgp_map* m, int64_t n, const uint64_t* keys, const double* D,
                    const double* V, const uint8_t* flags, vgp_stream stream);

/*
 * G-GPDF training set (Sec. IV-D): bin surface points by leaf.  The map keeps its own copy
 * (float32) so pts_dev may be freed after the call.  Replaces any previous surface.
 * Synchronises the stream.
 */
int vgp_set_surface(vgp_map* m, const float* pts_dev, int64_t n, vgp_stream stream);

/*
 * Zero crossings and marching cubes over the fused grid (Sec. IV-D: after fusion the touched
 * leaves are active; marching cubes recovers the surface there and its zero crossings train
 * the G-GPDF).  The fused value D of a voxel sits at its centre ijk * voxel_size; a voxel is
 * inside when D < 0.
 *   - zero crossing: on every axis edge between two known neighbouring voxels a, b = a + e_axis
 *     whose insides differ, at p_axis = (a_axis + t) vs with t = D_a / (D_a - D_b), the other two
 *     coordinates a_k vs (round-to-nearest FP64, no contraction); rounded to float32 it belongs
 *     to the voxel it falls in (one of a, b).  Slot = 2 axis + (the other end is on the + side).
 *   - marching cubes: every cell whose lower corner lies in a selected leaf and whose 8 corners
 *     are known; per inside mask the triangles come from walking the cell's faces, ambiguous
 *     faces keeping diagonal inside corners apart (so a face is split alike from both cells and
 *     the mesh is closed where the grid is), loops fanned from their first edge in
 *     (lower corner, axis) order, normals towards increasing D.
 * active_only = 1 selects the leaves the latest vgp_fuse touched, 0 all leaves.  The handle
 * owns device arrays, read with the two accessors below (pointers valid until
 * vgp_mesh_destroy):
 *   crossings: xyz [n][3] float32, owner [n] voxel key, slot [n] uint8; grouped by leaf, in a
 *              leaf in voxel-bit then slot order; the order of the leaf groups is unspecified.
 *   triangles: xyz [n][3][3] FP64 vertices; edge_key [n][3] key of each vertex's edge lower
 *              voxel, edge_axis [n][3]; a leaf's triangles by lower-corner bit; leaf order
 *              unspecified.  Shared vertices repeat; (edge_key, edge_axis) identifies them.
 * want_triangles = 0 skips the triangles (n = 0).  An empty grid gives empty arrays.
 * Synchronises the stream.
 */
int vgp_extract_mesh(vgp_map* m, int active_only, int want_triangles, vgp_stream stream, vgp_mesh** out);
int vgp_mesh_crossings(const vgp_mesh* mesh, int64_t* n, const float** xyz_dev, const uint64_t** owner_dev,
                       const uint8_t** slot_dev);
int vgp_mesh_triangles(const vgp_mesh* mesh, int64_t* n, const double** xyz_dev, const uint64_t** edge_key_dev,
                       const uint8_t** edge_axis_dev);
void vgp_mesh_destroy(vgp_mesh* mesh);

/*
 * Surface properties on the mesh (Sec. IV-D: the reconstruction carries the fused properties):
 * at each crossing the fused C of the edge's two ends interpolated with the crossing's t,
 * C_a + t (C_b - C_a) (NaN unless both ends hold properties).  cross [n_crossings][n_props],
 * vert [n_triangles][3][n_props], device, owned by the handle; *n_props = 0 (NULL pointers)
 * when the map has none.
 */
int vgp_mesh_props(const vgp_mesh* mesh, int32_t* n_props, const double** cross_dev, const double** vert_dev);

/*
 * Host copy of the marching-cubes table the kernels use (no device work): tab [256][16] cell
 * edges, three per triangle, edge = 4 axis + bit_u + 2 bit_w with (u, w) = (axis + 1,
 * axis + 2) mod 3 the lower corner's other coordinates; ntri [256] triangles per inside mask
 * (corner c = x + 2 y + 4 z).
 */
void vgp_debug_mc_table(uint8_t* tab, uint8_t* ntri);

/*
 * G-GPDF training set from the map (Sec. IV-D): the map keeps the zero crossings per leaf.
 * This call drops the kept points that lie in leaves the latest vgp_fuse touched, appends the
 * zero crossings of those leaves (as vgp_extract_mesh with active_only = 1 lists them), and
 * trains the G-GPDF on the result as vgp_set_surface would (replacing any surface set
 * before).  Kept points keep their order; each touched leaf's crossings follow in voxel-bit,
 * slot order.  Synchronises the stream.
 */
int vgp_update_surface(vgp_map* m, vgp_stream stream);

/*
 * The map's kept G-GPDF training set: n points, device float32 [n][3] owned by the map and
 * valid until the next vgp_update_surface or vgp_destroy.
 */
int vgp_surface_points(vgp_map* m, int64_t* n, const float** xyz_dev);

/*
 * G-GPDF query (Sec. IV-D; Eqs. 1-5).  For each query point q_dev[i] (float32 [n][3]):
 * the query leaf M = floor(ijk / 8); the GP instance is the set of surface points in the
 * 27 leaves around M (or, if those are empty, around the nearest occupied leaf within
 * max_leaf_search: smallest integer leaf distance, ties to the smaller key), capped at
 * max_pts_group.  Outputs (device, caller-owned, each may be NULL except d_dev):
 *   d_dev      [n] FP64 distance (m)
 *   grad_dev   [n][3] FP64 distance gradient
 *   var_dev    [n] FP64 distance variance (m^2); computing it adds an FP64 triangular solve
 *              per query (NULL skips it)
 *   status_dev [n] VGP_ST_*
 * VGP_ERR_STATE before vgp_set_surface.  Synchronises the stream several times.
 */
int vgp_query_distance_gradient(vgp_map* m, const float* q_dev, int64_t n, double* d_dev,
                                double* grad_dev, double* var_dev, uint8_t* status_dev,
                                vgp_stream stream);

/*
 * G-GPDF as blended per-leaf GPs (Sec. IV-D, Eq. 10).  Every occupied surface leaf is one GP
 * node trained on its points (at most max_pts_leaf, those nearest the leaf centre, ties to the
 * lower index).  For each query, the n_nodes nodes nearest to it (FP64 squared distance to
 * the leaf centre, ties to the smaller key) among the occupied leaves in the 27-leaf
 * neighbourhood of its centre leaf (the centre rule of vgp_query_distance_gradient) each give
 * d_q, grad d_q, v_q (Eqs. 1-5); Eq. 10 is read as a smooth minimum:
 *   d = sum_q w_q d_q / sum_q w_q,  w_q = exp(-lambda (d_q - min_q d_q)),
 * over the nodes with status OK; grad d = the plain average of their gradients (the paper
 * averages the nodes' gradients); var = sum_q w_q v_q / sum_q w_q.  If no node is OK the
 * status is that of the nearest node.  n_nodes in [1, 27]; lambda > 0 (the paper uses 100
 * per metre).  Outputs as for vgp_query_distance_gradient (grad_dev, var_dev, status_dev may
 * be NULL).  Uses n * n_nodes pair buffers in the map's arena.  Synchronises the stream.
 */
int vgp_query_smooth(vgp_map* m, const float* q_dev, int64_t n, int32_t n_nodes, double lambda, double* d_dev,
                     double* grad_dev, double* var_dev, uint8_t* status_dev, vgp_stream stream);

/*
 * Autotuner of the GP solve launch shapes: plans the given queries against the current
 * surface (as vgp_query_distance_gradient does), then solves the batch twice with each of
 * seven candidate launch shapes (threads per CTA, CTAs per SM, panel staging for N > 224),
 * times each bucket with CUDA events (the faster of the two runs counts), and keeps the
 * fastest shape per bucket for later calls on this map (L-GPDF frames, queries, batches).  Outputs nothing else; the chosen shapes and bucket
 * times appear in vgp_stats.  VGP_ERR_STATE before vgp_set_surface.  Synchronises the stream.
 */
int vgp_autotune(vgp_map* m, const float* q_dev, int64_t n, vgp_stream stream);

/*
 * Set the GP solve launch shapes by hand (what vgp_autotune chooses): threads[5] per CTA for
 * the size buckets N > 224, 129..224, 65..128, 33..64, <= 32 (multiples of 32 in [32, 1024]),
 * per_sm[5] caps on CTAs per SM (0: the occupancy limit), stage_panel 1 or 0 for the N > 224
 * bucket (panel column staged in shared memory, or read through L1/L2 with room for two
 * CTAs per SM).  VGP_ERR_ARG on a bad value.  Results do not depend on the shapes.
 */
int vgp_set_launch(vgp_map* m, const int32_t* threads, const int32_t* per_sm, int32_t stage_panel);

/*
 * Backward pass of a scalar loss L through vgp_query_distance_gradient, with the discrete
 * choices (instances, caps) of the forward pass.  Given dL_dd_dev [n] FP64:
 *   dL_dq_dev  [n][3] FP64: dL/dd_i * grad d_i (may be NULL)
 *   dL_dX_dev  [n_surface][3] FP64, overwritten: derivative w.r.t. each surface point of the
 *              last vgp_set_surface, from differentiating alpha = A^-1 1 (Eq. 1) and k
 *              (may be NULL).
 * The factorisation and alpha are recomputed, not stored.  Results where the forward
 * output was clamped or invalid contribute zero.  Synchronises the stream.
 */
int vgp_query_backward(vgp_map* m, const float* q_dev, int64_t n, const double* dL_dd_dev,
                       double* dL_dq_dev, double* dL_dX_dev, vgp_stream stream);

/*
 * Independent GP instances given directly (no grid): instance I trains on
 * X_dev[inst_off[I] .. inst_off[I+1]) and answers Q_dev[q_off[I] .. q_off[I+1]).
 *   inst_off_dev, q_off_dev  [n_inst + 1] int64 device offsets (non-decreasing, from 0)
 *   X_dev, Q_dev             float32 [.][3] device points
 *   outputs as for vgp_query_distance_gradient, indexed like Q_dev (var_dev may be NULL).
 * Instances with N > 1024 are rejected (VGP_ERR_ARG).  Uses the map's parameters and
 * device arena.  Synchronises the stream.
 */
int vgp_gp_batch(vgp_map* m, int64_t n_inst, const int64_t* inst_off_dev, const float* X_dev,
                 const int64_t* q_off_dev, const float* Q_dev, double* d_dev, double* grad_dev,
                 double* var_dev, uint8_t* status_dev, vgp_stream stream);

/*
 * vgp_gp_batch_static -- vgp_gp_batch for callers that cannot allocate device memory.
 * The paper has no counterpart; this entry point exists for callers for whom a cudaMalloc
 * (or a stream-ordered allocation) is not allowed or not possible at call time: code running
 * under an externally owned memory budget, real-time loops that must never enter the
 * allocator, or hosts that give the library a fixed footprint.  It needs no vgp_map either.
 *
 * Same computation and outputs as vgp_gp_batch with the parameters *p (precision, l, sigma,
 * d_max, d_var_floor; grid fields unused), on the current device.  All scratch lives in one
 * statically sized device array of about 31 MiB, compiled into the library: every GPU on which
 * the library is loaded holds it until the process exits.  Limits (VGP_ERR_ARG beyond them,
 * before any result is written): at most 65536 instances and 262144 training points per call,
 * at most 64 points per instance.
 *
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current) and keeps it for the life of the process: make that first call
 * before any stream capture, and do not call this entry point on a device after a
 * cudaDeviceReset of it in the same process (the kept address no longer names the array).
 * Each call writes a 2 KB constant table into the array on the caller's stream (an
 * asynchronous copy from host memory, ordered before the kernels that read it).
 * VGP_ERR_ARG also for offsets that are negative, decrease, or run past the maximum.
 * The call reads two words back from the GPU, so it synchronises the stream.  Every call on a
 * device shares the same array and it keeps the last call's contents; the call clears what
 * must start at zero.  Calls whose GPU work overlaps (several streams or host threads at once)
 * race on the array and give wrong results: serialise them.  Outputs are complete once the
 * stream has passed the call.  Calls no cudaMalloc, cudaFree or allocating library routine.
 */
int vgp_gp_batch_static(const vgp_params* p, int64_t n_inst, const int64_t* inst_off_dev, const float* X_dev,
                        const int64_t* q_off_dev, const float* Q_dev, double* d_dev, double* grad_dev,
                        double* var_dev, uint8_t* status_dev, vgp_stream stream);

/*
 * Diagnostic view of the neighbourhood selection of vgp_query_distance_gradient (Sec. IV-D
 * with the cap and fallback rules of max_pts_group and max_leaf_search): plans the n queries
 * exactly as that call does (query leaves, centre leaves, capped 27-leaf neighbourhoods),
 * solves nothing, and copies the plan to HOST arrays.  Call it once with the four arrays NULL
 * to get *n_inst and *n_train, then again with arrays of those sizes (the plan is recomputed
 * and is the same):
 *   inst_key   [n_inst] centre leaf key of each instance (order unspecified)
 *   inst_off   [n_inst + 1] offsets of each instance's points in point_idx
 *   point_idx  [n_train] indices into the points of the last vgp_set_surface (order within an
 *              instance unspecified)
 *   q_inst     [n] instance of each query, negative when it has none (bad input or no
 *              support)
 * VGP_ERR_STATE before vgp_set_surface.  Synchronises the stream.
 */
int vgp_debug_query_plan(vgp_map* m, const float* q_dev, int64_t n, vgp_stream stream, int64_t* n_inst,
                         int64_t* n_train, uint64_t* inst_key, int64_t* inst_off, int64_t* point_idx,
                         int32_t* q_inst);

/*
 * Diagnostic view of the node selection of vgp_query_smooth (Sec. IV-D, Eq. 10): the node GPs
 * (occupied leaves around the queries' centre leaves, each capped to the max_pts_leaf points
 * nearest its centre) and the nodes each query blends, copied to HOST arrays; same two-call
 * protocol and array meanings as vgp_debug_query_plan, with
 *   node_key   [n_inst] leaf key of each node GP (order unspecified)
 *   pair_inst  [n][n_nodes] node of each query by rank (nearest first), -1 past the last node
 * n_nodes in [1, 27].  Synchronises the stream.
 */
int vgp_debug_smooth_plan(vgp_map* m, const float* q_dev, int64_t n, int32_t n_nodes, vgp_stream stream,
                          int64_t* n_inst, int64_t* n_train, uint64_t* node_key, int64_t* inst_off,
                          int64_t* point_idx, int32_t* pair_inst);

/* Counters of the most recent build_frame / set_surface / query / batch call. */
int vgp_get_stats(const vgp_map* m, vgp_stats* out);

/*
 * Diagnostic: out_dev[i] = e^(y_dev[i]) computed by the FP64 table-driven exponential that the
 * mixed path uses for kernel-matrix entries (y <= 0; 0 below -700).  Device arrays of n doubles.
 */
int vgp_debug_exp_neg(const vgp_map* m, const double* y_dev, double* out_dev, int64_t n, vgp_stream stream);

/*
 * Diagnostic: out_dev[i] = round(k 2^61), k = exp(-|a_i - b_i|^2 / (2 l^2)), as the emulated
 * factorisation (emulate_fp64 = 1) assembles its mixed-precision kernel matrix (Sec. III-A
 * kernel) from the FP32 world coordinates a_i = xa_dev[3i..3i+2], b_i = xb_dev[3i..3i+2]:
 * float-pair arithmetic on the FP32 pipe, error below 2^-45 k (1 + y) + 2 units of 2^-61
 * (y = |a - b|^2 / (2 l^2)); 0 where k < 2^-62.  Device arrays; n pairs; stream-ordered.
 */
int vgp_debug_kernel_fix(const vgp_map* m, const float* xa_dev, const float* xb_dev, int64_t n, int64_t* out_dev,
                         vgp_stream stream);

/* Number of CUDA kernels this library has launched in the process so far (diagnostic). */
int64_t vgp_launch_count(void);

/* Wait for all device work of the map. */
int vgp_sync(vgp_map* m);

/* Message of the last error on this thread ("" if none).  Never NULL. */
const char* vgp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* VGPDF_H */
