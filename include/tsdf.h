/*
 * tsdf.h - C ABI of the B300 sparse TSDF fusion library (libtsdf.so).
 *
 * The library implements the data-parallel hot path of Trifonov, "Real-time High
 * Resolution Fusion of Depth Maps on GPU" (arXiv 1311.7194):
 *   1. allocation of the 8^3-voxel blocks that a posed depth map's surface
 *      touches (section "Updating Sparse Structure"),
 *   2. per-voxel Kalman update of distance T and variance P (Alg. 3) from the
 *      projective measurement T_k (section "Integration of Measurements"),
 *   3. raycasting of the sparse TSDF into depth, normal and vertex maps
 *      (section "Scene Rendering": block-range maps, coarse march, refinement).
 *
 * Conventions used by every call
 *   - Lengths in metres. Camera: pinhole with OpenCV axes (x right, y down,
 *     z forward); pixel (u, v) has its centre at integer coordinates and
 *     u = fx * x / z + cx.
 *   - Poses are camera-to-world 4x4 matrices T_wc, row major, 16 doubles in
 *     HOST memory, last row (0 0 0 1).
 *   - Voxel index i (3 integers in [0, grid_dim)) sits at world position
 *     origin + i * voxel_size. Block b = floor(i / 8); the voxel's index inside
 *     its block is x + 8 y + 64 z of i mod 8.
 *   - Images (depth, variance, output maps) are DEVICE pointers owned by the
 *     caller, float32, row major, width * height elements (x3 interleaved for
 *     normal/vertex maps). Depth 0, negative, NaN, Inf or outside
 *     [depth_min, depth_max] means "no measurement" (the paper's chi).
 *   - Every compute call is asynchronous on the given stream (a cudaStream_t
 *     passed as void*, NULL = legacy default stream) and does not synchronise.
 *     Argument errors are returned at once; errors found on the device
 *     (pool exhausted; in a TSDF_DEBUG build also a failed index check) set a
 *     sticky flag that tsdf_get_status reports.
 *   - A volume is not thread safe: serialise calls on one volume.
 *   - No call aborts the process or traps the GPU.
 */
#ifndef TSDF_H
#define TSDF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tsdf_volume tsdf_volume; /* opaque; owned by the library */

typedef enum {
    TSDF_OK = 0,
    TSDF_ERR_INVALID_ARG = 1,   /* null pointer, bad size or non-finite parameter */
    TSDF_ERR_CAPACITY = 2,      /* pool full: some new blocks were not allocated */
    TSDF_ERR_HASH_FULL = 3,     /* reserved: the dense block table never fills */
    TSDF_ERR_CUDA = 4,          /* a CUDA runtime call or kernel launch failed */
    TSDF_ERR_NOT_READY = 5,     /* reserved */
    TSDF_ERR_OUT_OF_MEMORY = 6, /* device allocation failed (tsdf_create*, host-input staging) */
    TSDF_ERR_BOUNDS = 7         /* a device-side index check failed; only a library built with
                                   TSDF_DEBUG checks (see tsdf_debug_build) */
} tsdf_status;

/* How T is held in the pool (P is always float32 and all arithmetic float32;
 * the paper stores T in 8 bits and sizes memory at 2 bytes per voxel). */
typedef enum {
    TSDF_STORAGE_F32 = 0,       /* float32, chi = NaN: 8 bytes per voxel with P */
    TSDF_STORAGE_F16 = 1,       /* IEEE half (round to nearest even), chi = NaN: 6 bytes per voxel */
    TSDF_STORAGE_SNORM16 = 2    /* int16 q = rint(T * (32767/delta)) in [-32767, 32767],
                                   T = q * (delta/32767), chi = -32768: 6 bytes per voxel */
} tsdf_storage;

/* How a measurement T_k(x) enters the voxel (section "Integration of
 * Measurements"). Every rule starts a chi voxel at T_k and marks |T| > delta as
 * chi afterwards.
 *   KALMAN:   Alg. 3 (the default): P <- P + Q, K = P / (P + p_k),
 *             T <- T + K (T_k - T), P <- (1 - K) P; P is the pool's second array.
 *   AVERAGE:  Alg. 1: T <- (1 - w) T + w T_k with the fixed weight
 *             w = update_weight; the second array is neither read nor written.
 *   WEIGHTED: Alg. 2: T <- (W T + w T_k) / (W + w), W <- min(W + w, W_max), with
 *             W kept in the second array (first measurement: W = w). */
typedef enum {
    TSDF_UPDATE_KALMAN = 0,
    TSDF_UPDATE_AVERAGE = 1,
    TSDF_UPDATE_WEIGHTED = 2
} tsdf_update_rule;

/* Pinhole intrinsics of one depth map / output map. */
typedef struct {
    float fx, fy, cx, cy;
    int32_t width, height;
} tsdf_intrinsics;

/* Volume settings (tsdf_config_default fills the defaults named below). */
typedef struct {
    float voxel_size;           /* s > 0 (default 1.5e-3) */
    float truncation;           /* delta > 0, Eq. 1 (default 5 s) */
    double origin[3];           /* world position of voxel (0,0,0)
                                   (default -grid_dim*s/2 on every axis) */
    int32_t grid_dim;           /* G voxels per axis, multiple of 8, (G/8)^3 < 2^32
                                   (default 2048) */
    int64_t block_capacity;     /* pool size in blocks (default 2^20) */
    float process_variance;     /* Q >= 0 of Alg. 3 (default 0) */
    float depth_min, depth_max; /* valid measured depth range (default 0.1 .. 4) */
    float raycast_near, raycast_far; /* raycast depth range (default 0.1 .. 4) */
    float sigma_coeff;          /* a >= 0: sensor deviation a*D^2, used when no
                                   variance map is given (default 1.5e-3) */
    int32_t storage;            /* tsdf_storage (default TSDF_STORAGE_F32) */
    int32_t alloc_half_samples; /* J >= 0; 0 = ceil(2 delta / s) (default 0) */
    int32_t update_rule;        /* tsdf_update_rule (default TSDF_UPDATE_KALMAN) */
    float update_weight;        /* w_k of Alg. 1 (0 < w <= 1) and Alg. 2 (w > 0),
                                   the same for every measurement (default 0.1) */
    float weight_max;           /* W_max >= w of Alg. 2 (default 1) */
    int32_t refine_steps;       /* 0..8 Gauss-Newton steps refining T_k in the depth map
                                   (section "Integration of Measurements", last paragraph):
                                   T_k becomes the distance from the voxel to the bilinear
                                   back-projected depth surface, signed by its tangent plane,
                                   wherever the four pixels around each step are valid and
                                   within delta of each other (default 0 = the z-difference) */
} tsdf_config;

/* Counters of the last calls (tsdf_get_stats). */
typedef struct {
    int64_t n_blocks;           /* blocks in the pool */
    int64_t new_blocks;         /* blocks added by the last tsdf_allocate */
    int64_t visible_blocks;     /* blocks the last tsdf_integrate visited */
    int64_t voxel_updates;      /* voxels updated (T_k != chi) by the last tsdf_integrate */
    int64_t raycast_blocks;     /* blocks rasterised by the last tsdf_raycast */
    int64_t rays_hit;           /* pixels that found a surface in the last tsdf_raycast */
    int64_t frames;             /* tsdf_integrate calls since creation / reset */
    int64_t voxel_updates_total;   /* sums over all calls since creation / reset */
    int64_t visible_blocks_total;
    int64_t rays_hit_total;
    int64_t raycast_blocks_total;
    int64_t voxels_touched_total;  /* voxels whose T and P an integrate call read and wrote (updated by at
                                      least one of its frames), summed over calls: the unit of the
                                      integrate roofline; equals voxel_updates_total when every call
                                      fuses one frame */
} tsdf_stats;

/* Fill *cfg with the defaults listed in tsdf_config. Host only. */
void tsdf_config_default(tsdf_config* cfg);

/* Human-readable name of a status code (static string). */
const char* tsdf_status_string(tsdf_status s);

/* Create an empty volume with the given voxel size, truncation and pool
 * capacity, all other settings at their defaults (section "Volumetric Scene
 * Representation": two device buffers, a block table and a pool of M^3-voxel
 * blocks, here M = 8). Allocates device memory on the current CUDA device:
 * 4 (G/8)^3 bytes of block table plus 8*512 (float32 storage) or 6*512 bytes
 * per pool block plus small lists. *out receives the handle, to be freed with tsdf_destroy.
 * Errors: TSDF_ERR_INVALID_ARG (bad values, out == NULL),
 *         TSDF_ERR_OUT_OF_MEMORY, TSDF_ERR_CUDA. */
tsdf_status tsdf_create(float voxel_size, float truncation, int64_t block_capacity,
                        tsdf_volume** out);

/* Same with every setting given. Errors as tsdf_create. */
tsdf_status tsdf_create_ex(const tsdf_config* cfg, tsdf_volume** out);

/* Free a volume and its device memory (synchronises its last stream). NULL is
 * a no-op. */
void tsdf_destroy(tsdf_volume* vol);

/* Empty the volume (no blocks, frame counter 0, status cleared) without freeing
 * memory; asynchronous on stream. */
tsdf_status tsdf_reset(tsdf_volume* vol, void* stream);

/* Allocate the blocks one posed depth map's surface touches (section "Updating
 * Sparse Structure"; the paper samples the surface, writes block coordinates
 * and allocates them, missing a few blocks being tolerable). Every valid pixel
 * (i, j) is sampled at 2J+1 depths D + m delta/J, m = -J..J, along its ray; the
 * block of each sample inside the grid is allocated if it is not yet. New blocks
 * of one call join the pool in ascending key order (key = bx + N (by + N bz),
 * N = G/8), hold chi everywhere and remember the frame counter as their
 * allocation frame. The sample arithmetic is a fixed sequence of correctly
 * rounded float32 operations, so the block set is reproducible bit for bit:
 *   xn = (i - cx)/fx, yn = (j - cy)/fy; b = fma(M0, xn, fma(M1, yn, M2)) per row
 *   of M = R/s; z_m = fma(m, delta/J, D); q = fma(z_m, b, (t - origin)/s);
 *   inside iff 0 <= q < G; block = floor(q) / 8,
 * with M, delta/J and (t - origin)/s computed in double and rounded once.
 * depth: device, width*height float32. K: host. pose_wc: host, 16 doubles.
 * When the pool is full, the highest-key new blocks are dropped and the sticky
 * status TSDF_ERR_CAPACITY is set. Errors: TSDF_ERR_INVALID_ARG, TSDF_ERR_CUDA. */
tsdf_status tsdf_allocate(tsdf_volume* vol, const float* depth, const tsdf_intrinsics* K,
                          const double pose_wc[16], void* stream);

/* Fuse one posed depth map into the allocated blocks with Alg. 3. For every
 * voxel x of every allocated block: x_c = T_wc^-1 x; pixel = nearest
 * (floor(fx x_c/z_c + cx + 1/2), same for v); T_k = D(pixel) - z_c (the
 * projective distance, positive in front of the surface, Eq. 1), chi when
 * z_c <= 0, the pixel is outside the image, D is not valid, p_k is not a
 * positive finite number, or |T_k| > delta. For T_k != chi:
 *   T == chi:  T = T_k, P = p_k
 *   else:      P += Q; K = P/(P+p_k); T += K (T_k - T); P = (1-K) P
 *   then:      T = chi if |T| > delta.
 * p_k = variance[pixel] when variance != NULL (device, width*height float32),
 * else (sigma_coeff * D^2)^2. Only blocks whose box can reach the image, the
 * depth range and the truncation band of the depth under their footprint are
 * visited (a conservative cull: skipped voxels would all have T_k = chi); all
 * other voxels are unchanged. The first call with an image larger than any
 * before grows a small per-tile depth buffer (cudaMalloc, synchronising).
 * Increments the frame counter. Errors: TSDF_ERR_INVALID_ARG, TSDF_ERR_CUDA. */
tsdf_status tsdf_integrate(tsdf_volume* vol, const float* depth, const float* variance,
                           const tsdf_intrinsics* K, const double pose_wc[16], void* stream);

/* Fuse K posed depth maps (1 <= K <= 8) in one pass: the same result, bit for
 * bit, as K calls of tsdf_allocate followed by tsdf_integrate in order (frames
 * numbered from the current frame counter). Each frame is allocated in turn
 * (a block remembers the first frame that allocated it), then one kernel walks
 * the union of the K frames' visible blocks, loads each voxel's T and P once,
 * applies Alg. 3 for frames 0..K-1 in order - skipping frames before its
 * block's allocation - and stores them once. depth: host array of K device
 * pointers (width*height float32 each); variance: NULL (quadratic model for all
 * frames) or a host array of K device pointers; K: shared intrinsics;
 * poses_wc: host, K*16 doubles. The first call (and the first with a larger
 * image) allocates batch buffers of 256 bytes per pool block (cudaMalloc,
 * synchronising). Increments the frame counter by K. Errors:
 * TSDF_ERR_INVALID_ARG, TSDF_ERR_CUDA; pool exhaustion as tsdf_allocate. */
tsdf_status tsdf_integrate_batch(tsdf_volume* vol, int32_t K, const float* const* depth,
                                 const float* const* variance, const tsdf_intrinsics* Kin,
                                 const double* poses_wc, void* stream);

/* Raycast the fused surface into depth / normal / vertex maps of size
 * K->width x K->height (section "Scene Rendering"). Per pixel, a range map made
 * by rasterising the boxes of the allocated blocks (nearest front / farthest
 * back, clamped to [raycast_near, raycast_far]) bounds the march; the ray is
 * marched in camera z with step delta/2 over the trilinear interpolation of T
 * (undefined where any of the 8 voxels is chi or unallocated; unallocated
 * blocks are skipped whole) until the first + to - crossing; a - to + crossing
 * first ends the ray as a miss. The crossing is refined by secant steps.
 * depth_out: camera z (0 on a miss); vertex_out: world position (NaN on a miss);
 * normal_out: normalised central-difference gradient of T (+-1 voxel), in world
 * axes, facing the camera (NaN on a miss or undefined gradient). Any output may
 * be NULL. Outputs are device pointers (depth: W*H floats, normal/vertex:
 * W*H*3 floats, xyz interleaved). Errors: TSDF_ERR_INVALID_ARG, TSDF_ERR_CUDA. */
tsdf_status tsdf_raycast(tsdf_volume* vol, const tsdf_intrinsics* K, const double pose_wc[16],
                         float* depth_out, float* normal_out, float* vertex_out, void* stream);

/* The same raycast as tsdf_raycast, for callers that must not allocate device
 * memory during the call. The paper has no counterpart: this is a property of
 * the library's memory handling, not of the method.
 * tsdf_raycast grows its near / far range maps with cudaMalloc (and frees the
 * old ones, which synchronises the device) whenever it first sees a larger
 * image. Callers that cannot allow that - a real-time loop with a fixed memory
 * budget that must not stall, an application whose own allocator owns device
 * memory, code recording work for later replay - use this call instead: it
 * takes its scratch - the range maps (one near / far pair per 4x4-pixel tile)
 * and the ray-order lists (4 lists of 8x4-pixel tiles) - from a fixed 1.25 MiB
 * array inside the library (held by every GPU that loads the library until
 * the process exits) and allocates nothing. Limits and rules:
 *   - ceil(W/4) * ceil(H/4) <= 81920 and ceil(W/8) * ceil(H/4) <= 40960
 *     (every image up to 1280 x 1024 pixels), else TSDF_ERR_INVALID_ARG;
 *   - the current device must be the volume's device, else TSDF_ERR_INVALID_ARG;
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) and caches it; make that first call before any
 *     stream capture. The cached address does not survive cudaDeviceReset;
 *   - all calls on a device share the array, which keeps the last call's
 *     contents (each call clears the maps it uses first); calls whose GPU work
 *     overlaps race on it and must be serialised.
 * Arguments, outputs and the other errors are those of tsdf_raycast. */
tsdf_status tsdf_raycast_noalloc(tsdf_volume* vol, const tsdf_intrinsics* K, const double pose_wc[16],
                                 float* depth_out, float* normal_out, float* vertex_out, void* stream);

/* Traversal counts of one raycast, for measurement (no counterpart in the
 * paper). */
typedef struct {
    int64_t samples;        /* trilinear samples taken (march, re-scan, refinement, normal) */
    int64_t table_lookups;  /* block-table entries read by those samples */
    int64_t t_sectors;      /* distinct 32-byte sectors of the T pool read */
    int64_t table_sectors;  /* distinct 32-byte sectors of the block table read */
    int64_t rays;           /* W * H */
    int64_t rays_hit;
    /* by phase (samples = march_samples + rescan_samples + refine_samples
     * + normal_samples) */
    int64_t march_samples;  /* coarse march iterations (each takes one sample) */
    int64_t skips;          /* of those, samples in an unallocated block: an empty-space jump */
    int64_t rescans;        /* re-scans of a step that entered the field at or below zero */
    int64_t rescan_samples; /* samples those re-scans took */
    int64_t refine_samples; /* false-position samples of the crossing refinement */
    int64_t normal_samples; /* central-difference samples of the normals */
} tsdf_raycast_counts;

/* Run the raycast of tsdf_raycast at pose_wc with every sample traced and
 * return the counts in *out (host struct). Same rays, samples and crossings as
 * tsdf_raycast (the one-thread-per-pixel kernel with tracing compiled in); no
 * maps are written. It gives the unique bytes a raycast must read, the
 * algorithmic bytes of the raycast's roofline. Slow and synchronous: it
 * allocates and frees one flag byte per 32 bytes of the T pool and of the block
 * table (e.g. 64 + 8 MiB for 2^20 float32 blocks on a 2048^3 grid). Counts as a
 * raycast in tsdf_get_stats. Errors: TSDF_ERR_INVALID_ARG, TSDF_ERR_CUDA. */
tsdf_status tsdf_raycast_trace(tsdf_volume* vol, const tsdf_intrinsics* K, const double pose_wc[16],
                               tsdf_raycast_counts* out, void* stream);

/* Marching-cubes surface of the volume (section "Scene Rendering": the
 * paper's polygonising renderer). Every cell - the cube of lattice voxels
 * i + {0,1}^3 - whose 8 voxels are defined (allocated, not chi) is polygonised:
 * a corner is inside when T < 0, the surface crosses an edge at the linear
 * zero of T, and the cell's triangles come from a case table the library
 * builds from the published construction (per-face segments, a face with four
 * crossings pairing each inside corner's two edges, segments oriented so the
 * normal points from inside to outside, loops fan-split from their smallest
 * edge number), which keeps the surface closed across cells. Output:
 * triangles as 9 floats each (three world xyz vertices, counter-clockwise seen
 * from outside), ordered by pool slot and, within a block, by cell
 * (x fastest). Call with triangles = NULL to get the count in *n_triangles
 * (host), then with a device buffer of max_triangles >= that count; a smaller
 * buffer gets TSDF_ERR_CAPACITY and nothing written. Synchronous. Errors:
 * TSDF_ERR_INVALID_ARG, TSDF_ERR_CAPACITY, TSDF_ERR_CUDA. */
tsdf_status tsdf_mesh(tsdf_volume* vol, float* triangles, int64_t max_triangles, int64_t* n_triangles,
                      void* stream);

/* The case table entry for a corner pattern (bit c set = corner c inside,
 * corners c = x + 2y + 4z): *n_triangles and their edges, 3 per triangle, in
 * edges[24] (edges 0-3 run along x from corners 0, 2, 4, 6; 4-7 along y from
 * corners 0, 1, 4, 5; 8-11 along z from corners 0, 1, 2, 3). Host only.
 * Errors: TSDF_ERR_INVALID_ARG. */
tsdf_status tsdf_mesh_case(int32_t pattern, int32_t* n_triangles, int8_t edges[24]);

/* ---------------------------------------------------------------------------
 * Registration (section "Registration", Eqs. 2-8): point-to-plane ICP of a
 * depth frame against the model maps of tsdf_raycast.
 * ------------------------------------------------------------------------- */
typedef struct {
    float dist_max;         /* pairs farther apart than this are rejected, metres (default 0.05) */
    float normal_cos_min;   /* pairs whose normals' dot product is below this are rejected (default 0.8) */
    float eig_threshold;    /* theta of Eq. 8: eigen-directions with lambda / pairs <= theta are
                               dropped (default 0.005) */
    int32_t iterations;     /* ICP iterations per call, 1..100 (default 10) */
} tsdf_icp_params;

typedef struct {
    int64_t matches;        /* accepted pairs in the last iteration */
    double rms;             /* point-to-plane RMS of those pairs, before that iteration's motion (m) */
    int32_t rank;           /* eigen-directions kept in the last iteration (6 = fully constrained) */
    int32_t iterations;     /* iterations run */
} tsdf_icp_result;

/* Fill *p with the defaults above. Host only. */
void tsdf_icp_params_default(tsdf_icp_params* p);

/* Register a depth frame to the model: refine *pose_wc (host FP64 4x4 row-major
 * camera->world; in: initial estimate, out: refined pose) by prm->iterations
 * iterations of Chen-Medioni point-to-plane ICP. Each iteration back-projects
 * every frame pixel whose depth and 4-neighbours lie in the volume's
 * [depth_min, depth_max], takes its normal from the central differences of the
 * back-projected neighbours, moves both into the world with the current
 * estimate, matches the point to the model pixel nearest its projection into
 * the model camera (model_pose_wc), rejects the pair by dist_max and
 * normal_cos_min, and accumulates the Eq. 4 sums on the GPU (matching,
 * rejection and the first reduction level in one kernel, the rest in a second,
 * in double). The host then restates the 6x6 system in the box of the matched
 * points shrunk to the unit cube (Eqs. 5-7), drops eigen-directions with
 * lambda / pairs <= theta (Eq. 8), recovers the motion as r = S^-1 r^,
 * t = t^ - r x m (the scaled unknowns being r^ = S r, t^ = t + r x m), and
 * applies p -> exp([r]x) p + t to the pose.
 * depth: device W*H floats of the frame; model_vertex / model_normal: device
 * W*H*3 floats (world, NaN = no surface) as written by tsdf_raycast with the
 * same intrinsics K at model_pose_wc. Synchronises with the stream once per
 * iteration (the pose lives on the host); each iteration's sums and box reach
 * the host in one copy through a small pinned buffer that the volume
 * allocates on its first registration call (with the device buffer of the
 * partial sums) and frees in tsdf_destroy. *out (optional) receives the last
 * iteration's statistics. An iteration with fewer than 6 pairs leaves the pose
 * unchanged. Errors: TSDF_ERR_INVALID_ARG, TSDF_ERR_CUDA (also when either
 * buffer cannot be allocated). */
tsdf_status tsdf_icp(tsdf_volume* vol, const float* depth, const tsdf_intrinsics* K, const float* model_vertex,
                     const float* model_normal, const double model_pose_wc[16], const tsdf_icp_params* prm,
                     double pose_wc[16], tsdf_icp_result* out, void* stream);

/* One matching pass of tsdf_icp at pose_wc without solving: the 29 plain sums
 * of Eq. 4 to host sums[29] (the 21 entries of sum J J^T, upper triangle row
 * by row, J = (p x n, n); the 6 of sum J ((p - q).n); sum ((p - q).n)^2; the
 * number of pairs) and the box of the matched points to host box[6] (min x, y,
 * z, max x, y, z). Synchronous. Errors: as tsdf_icp. */
tsdf_status tsdf_icp_sums(tsdf_volume* vol, const float* depth, const tsdf_intrinsics* K, const float* model_vertex,
                          const float* model_normal, const double model_pose_wc[16], const tsdf_icp_params* prm,
                          const double pose_wc[16], double sums[29], float box[6], void* stream);

/* The host half of one iteration: the motion (r[3] rotation vector, t[3]) from
 * the sums and box of tsdf_icp_sums and theta (Eqs. 5-8); *rank (optional)
 * receives the number of eigen-directions kept. Host only, no GPU needed.
 * Errors: TSDF_ERR_INVALID_ARG (null pointers, theta < 0). */
tsdf_status tsdf_icp_solve(const double sums[29], const float box[6], float theta, double r[3], double t[3],
                           int32_t* rank);

/* CUDA-graph driver of the per-step pipeline (no counterpart in the paper; it
 * removes per-kernel launch gaps). A step fuses K frames (1 <= K <= 8) exactly
 * as tsdf_integrate (K = 1) or tsdf_integrate_batch (K > 1) would, then
 * raycasts the model at the last frame's pose exactly as tsdf_raycast. The step
 * is recorded by stream capture on a private stream and run as one graph
 * launch; later steps update the same executable graph in place.
 * tsdf_graph_create sizes every buffer the step needs for images of K->width x
 * K->height (it may allocate and synchronise); tsdf_graph_launch then
 * allocates nothing. One graph per volume at a time; calls on the graph and
 * its volume must be serialised. Errors: TSDF_ERR_INVALID_ARG, TSDF_ERR_CUDA,
 * TSDF_ERR_OUT_OF_MEMORY (create). */
typedef struct tsdf_graph tsdf_graph;
tsdf_status tsdf_graph_create(tsdf_volume* vol, int32_t K, const tsdf_intrinsics* Kin, tsdf_graph** out);
/* depth: host array of K device pointers; variance: NULL or K device pointers;
 * poses_wc: host, K*16 doubles; outputs as tsdf_raycast (each may be NULL). */
tsdf_status tsdf_graph_launch(tsdf_graph* g, const float* const* depth, const float* const* variance,
                              const double* poses_wc, float* depth_out, float* normal_out,
                              float* vertex_out, void* stream);
/* The same step from host depth maps. depth_host: host array of K host
 * pointers, each a width x height float32 map (page-locked memory lets the copy
 * overlap the previous step's kernels; pageable memory works but copies
 * synchronously). The maps are copied into one of two library-owned device
 * staging sets on a private stream, and the graph runs on `stream` once the
 * copy is done; the sets alternate per call, so a map may be reused by the
 * caller once this call's work on `stream` has completed. Variance: the
 * volume's own (quadratic, or the installed network). Outputs as
 * tsdf_graph_launch (device pointers). The first call allocates the staging
 * sets (2 K width x height floats) and may synchronise. Errors as
 * tsdf_graph_launch, and TSDF_ERR_OUT_OF_MEMORY for the staging sets. */
tsdf_status tsdf_graph_launch_host(tsdf_graph* g, const float* const* depth_host, const double* poses_wc,
                                   float* depth_out, float* normal_out, float* vertex_out, void* stream);
/* Number of graph instantiations so far (1 after the first step when every
 * update succeeded); -1 for NULL. */
int64_t tsdf_graph_instantiations(const tsdf_graph* g);
/* Events (cudaEvent_t as void*, created by the caller) recorded by the next
 * launches before allocation, before integration, before the raycast and at
 * the end of the step; NULL (or NULL entries) records none. */
tsdf_status tsdf_graph_set_events(tsdf_graph* g, void* const events[4]);
void tsdf_graph_destroy(tsdf_graph* g);

/* Launch shapes (no counterpart in the paper; none changes any result, only
 * speed): integrate voxels per thread (4 or 8) and persistent CTAs per SM
 * (1..32); raycast pixel tile per CTA (16x8, 8x8, 32x4, 8x16 or 16x16) or the
 * persistent raycast. Defaults: 4, 12, 16x8, not persistent. */
typedef struct {
    int32_t integrate_voxels_per_thread;
    int32_t integrate_ctas_per_sm;
    int32_t raycast_tile_w, raycast_tile_h;
    int32_t raycast_persistent;  /* 1: persistent raycast (lanes fetch rays and run
                                    march / refine / normal as a state machine),
                                    0: one thread per pixel in the tile above */
} tsdf_launch_config;
tsdf_status tsdf_get_launch_config(const tsdf_volume* vol, tsdf_launch_config* out);
/* TSDF_ERR_INVALID_ARG for a shape outside the lists above. */
tsdf_status tsdf_set_launch_config(tsdf_volume* vol, const tsdf_launch_config* cfg);

/* Autotuner: time every launch shape on the caller's frames (n device depth
 * maps, host poses n*16 doubles, shared intrinsics K) - integrate on the
 * frames fused from an empty volume, raycast at each frame's pose - keep the
 * fastest, and record it in the JSON-lines file cache_path (may be NULL) under
 * a key of GPU name, image size, grid size and storage. When the file already
 * holds the key, the cached shape is set without timing and *from_cache = 1.
 * Empties the volume (tsdf_reset) when done: tune before fusing. Allocates
 * and synchronises; not for use under stream capture. *out (may be NULL)
 * receives the chosen shape. Errors: TSDF_ERR_INVALID_ARG, TSDF_ERR_CUDA. */
tsdf_status tsdf_autotune(tsdf_volume* vol, int32_t n, const float* const* depth, const tsdf_intrinsics* K,
                          const double* poses_wc, const char* cache_path, tsdf_launch_config* out,
                          int32_t* from_cache);

/* Learned measurement variance (no counterpart in the paper, which motivates
 * per-measurement variances - deviation growing with depth, poorer data near
 * edges - but does not say how to estimate them). A 27-32-32-1 perceptron with
 * ReLU, bfloat16 weights and float32 arithmetic predicts out = log(p_k/p_quad)
 * at a pixel from
 *   f[0..24] = (D(u+d) - D(u)) / delta clamped to [-1, 1] over the 5x5
 *              neighbourhood (row-major), +1 where a neighbour is outside the
 *              image or not a valid measurement,
 *   f[25]    = D(u) / 4,
 *   f[26]    = |cos| between the viewing ray and the normal from the depth
 *              map's central differences (0 when a 4-neighbour is invalid);
 * p_k = p_quad exp(out), or p_quad when |out| > ln 4 or out is not finite
 * (p_quad = (sigma_coeff D^2)^2). Parameters (1985): W1[32][27], b1[32],
 * W2[32][32], b2[32], W3[32], b3. */
int32_t tsdf_mlp_param_count(void);
/* Install (host bfloat16 bits, n = 1985) or remove (NULL / n = 0) the network;
 * while installed, tsdf_integrate / tsdf_integrate_batch / graph steps given no
 * variance map compute p_k with it in the same stream. */
tsdf_status tsdf_set_variance_mlp(tsdf_volume* vol, const uint16_t* bf16_weights, int64_t n);
/* The variance map the network gives for one depth map (w: device bfloat16
 * weights; depth, var_out: device W*H float32; 0 where depth is invalid). The
 * volume supplies truncation, depth range and sigma_coeff. */
tsdf_status tsdf_mlp_variance(const tsdf_volume* vol, const uint16_t* w, const float* depth,
                              const tsdf_intrinsics* K, float* var_out, void* stream);
/* Features of n pixels (uv: device n x 2 int32) -> feats (device n x 27);
 * valid (device n bytes, may be NULL): whether the centre depth is valid. */
tsdf_status tsdf_mlp_features(const tsdf_volume* vol, const float* depth, const tsdf_intrinsics* K, int64_t n,
                              const int32_t* uv, float* feats, uint8_t* valid, void* stream);
/* Training pairs: for pixels where both the measured depth and the model's
 * raycast depth pred_depth (same pose; 0 = miss) are valid and the residual
 * r = depth - pred lies within 4 truncation distances, append the features and
 * s = r^2 / p_quad at *count (device counter, incremented; rows beyond max_n
 * are counted but not written). */
tsdf_status tsdf_mlp_harvest(const tsdf_volume* vol, const float* depth, const float* pred_depth,
                             const tsdf_intrinsics* K, int64_t max_n, float* feats, float* s, uint32_t* count,
                             void* stream);
/* Network outputs for n feature rows (device). */
tsdf_status tsdf_mlp_forward(const uint16_t* w, int64_t n, const float* feats, float* out, void* stream);
/* Adds to grad (device, 1985 float32) the gradient, and to loss (device
 * scalar) the value, of the summed Gaussian negative log-likelihood
 * (out + s exp(-out)) / 2 over rows idx[0..n) of (feats, s) (idx NULL: rows
 * 0..n). */
tsdf_status tsdf_mlp_loss_grad(const uint16_t* w, int64_t n, const int32_t* idx, const float* feats,
                               const float* s, float* grad, float* loss, void* stream);
/* One Adam step on float32 master weights w32 (moments m, v) with gradient
 * grad * grad_scale; writes the bfloat16 copy wbf16 and zeroes grad. step >= 1
 * is the step number used for bias correction. All pointers device, 1985 each. */
tsdf_status tsdf_mlp_adam(float* w32, uint16_t* wbf16, float* m, float* v, float* grad, float lr, float beta1,
                          float beta2, float eps, float grad_scale, int32_t step, void* stream);

/* Per-pixel measurement variance of a sensor whose deviation grows
 * quadratically with depth (Introduction; the text before Alg. 3):
 * var[i] = (sigma_coeff * depth[i]^2)^2 for valid depth > 0, else 0.
 * depth, var_out: device, n float32. Errors: TSDF_ERR_INVALID_ARG, TSDF_ERR_CUDA. */
tsdf_status tsdf_quadratic_variance(const float* depth, int64_t n, float sigma_coeff,
                                    float* var_out, void* stream);

/* Debug builds (no counterpart in the paper; the stand-in for a device memory
 * checker). A library built with TSDF_DEBUG checks, on the device, the block
 * table keys, the pool slots and the visible-list and range-map indices its
 * kernels use; a failed check skips the access and sets a sticky error that
 * tsdf_get_status reports as TSDF_ERR_BOUNDS (nothing traps). The in-tree
 * build writes it as libtsdf_debug.so next to libtsdf.so.
 * tsdf_debug_build: 1 in such a library, 0 in the release one.
 * tsdf_debug_check_slot: reads pool slot `slot` of the volume behind the same
 * check as the raycast's voxel loads, so that the host can make the check
 * fail (a slot outside [0, block_capacity)) and see TSDF_ERR_BOUNDS reported;
 * an in-range slot changes nothing. Synchronous. In a release build it
 * launches nothing and returns TSDF_ERR_NOT_READY. Errors:
 * TSDF_ERR_INVALID_ARG, TSDF_ERR_CUDA. */
int tsdf_debug_build(void);
tsdf_status tsdf_debug_check_slot(tsdf_volume* vol, int64_t slot, void* stream);

/* Synchronise the volume's last stream and return the first error seen:
 * a sticky device flag (TSDF_ERR_CAPACITY) or a CUDA error. */
tsdf_status tsdf_get_status(tsdf_volume* vol);

/* Synchronise and copy the counters into *out (host). */
tsdf_status tsdf_get_stats(tsdf_volume* vol, tsdf_stats* out);

/* The volume's configuration as it is now (tsdf_shift moves the origin).
 * Errors: TSDF_ERR_INVALID_ARG. */
tsdf_status tsdf_get_config(const tsdf_volume* vol, tsdf_config* out);

/* Block eviction (section "Discussion": the TSDF data of occupied blocks goes
 * to host storage so that scenes larger than device memory can be scanned).
 * Every allocated block whose block coordinates lie outside the box
 * [lo, hi) (per axis, block units) is removed from the volume and copied to
 * HOST buffers in pool order: coords_frame n x 4 int32 (bx, by, bz,
 * allocation frame), T n x 512 float32 decoded from the storage format
 * (chi = NaN), P n x 512 float32; any of the three may be NULL. *n_evicted
 * receives n. The kept blocks keep their data bit for bit; the pool is
 * compacted (the last kept blocks move into the freed slots) and the block
 * table and occupancy maps are updated. Synchronous; allocates and frees a
 * staging buffer of n x 4 KB on the device.
 * Errors: TSDF_ERR_INVALID_ARG (NULL vol / lo / hi / n_evicted, lo > hi on an
 * axis, max_blocks < 0); TSDF_ERR_CAPACITY when n > max_blocks, with
 * *n_evicted = n and nothing changed; TSDF_ERR_CUDA. */
tsdf_status tsdf_evict(tsdf_volume* vol, const int32_t lo[3], const int32_t hi[3], int64_t max_blocks,
                       int32_t* coords_frame, float* T, float* P, int64_t* n_evicted, void* stream);

/* Volume shift (section "Discussion": the shift evicts the TSDF data of the
 * blocks that leave the volume and rebuilds the offset array). The grid moves
 * by d whole blocks: origin += 8 * voxel_size * d, so a voxel keeps its world
 * position and its block coordinates become b - d. Blocks whose new
 * coordinates fall outside [0, grid_dim / 8) are evicted first, exactly as
 * tsdf_evict does (same outputs, coordinates before the shift); the block
 * table is then rebuilt from the kept blocks. The new origin is read back with
 * tsdf_get_config. Errors: those of tsdf_evict (nothing changes on an error),
 * TSDF_ERR_INVALID_ARG for |d| >= 2^24 on an axis. */
tsdf_status tsdf_shift(tsdf_volume* vol, const int32_t d[3], int64_t max_blocks, int32_t* coords_frame,
                       float* T, float* P, int64_t* n_evicted, void* stream);

/* Bring evicted blocks back: n blocks from HOST buffers laid out as
 * tsdf_evict writes them (the allocation-frame column is ignored: an imported
 * block counts as allocated at the current frame). T is encoded to the
 * storage format (a block evicted from a volume of the same format comes back
 * bit for bit). Synchronous.
 * Errors: TSDF_ERR_INVALID_ARG (NULL buffers with n > 0, n < 0, coordinates
 * outside the grid, a block given twice or already allocated - nothing is
 * changed then); TSDF_ERR_CAPACITY when the pool cannot hold n more blocks;
 * TSDF_ERR_CUDA. */
tsdf_status tsdf_import(tsdf_volume* vol, int64_t n, const int32_t* coords_frame, const float* T, const float* P,
                        void* stream);

/* Copy the volume to HOST buffers in pool order (synchronises). For n blocks:
 * coords_frame: n x 4 int32 (bx, by, bz, allocation frame); T: n x 512 float32
 * decoded from the storage format (chi = NaN); P: n x 512 float32 (unspecified
 * where T is chi). Any buffer may
 * be NULL; capacity is the number of blocks each buffer holds. *n_out receives
 * the pool size; if it exceeds capacity only the first capacity blocks are
 * copied. Errors: TSDF_ERR_INVALID_ARG, TSDF_ERR_CUDA. */
tsdf_status tsdf_export(tsdf_volume* vol, int32_t* coords_frame, float* T, float* P,
                        int64_t capacity, int64_t* n_out);

#ifdef __cplusplus
}
#endif

#endif /* TSDF_H */
