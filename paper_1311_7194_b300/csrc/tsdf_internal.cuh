// Internal declarations of libtsdf: device data layout, per-call constants and
// the launchers each stage file provides. Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tsdf.h"
#include "tsdf_storage.cuh"

namespace tsdf {

constexpr int kSide = 8;                 // M: voxels per block axis
constexpr int kBlockVoxels = 512;        // M^3
constexpr int kTileWords = 4096;         // new-block bitmap words per scan tile
constexpr int kTileThreads = 256;        // threads per scan tile (16 words each)
constexpr unsigned kErrCapacity = 1u;    // sticky device error bits: pool exhausted
constexpr unsigned kErrBounds = 2u;      // a device-side index check failed (TSDF_DEBUG builds)
constexpr int kDepthTile = 8;            // depth min / max tiles used by the integrate cull
constexpr int kMaxBatch = 8;             // frames per tsdf_integrate_batch call
constexpr int kMlpParams = 1985;         // learned-variance network: 27-32-32-1
constexpr int kOcc2 = 4;                 // occupancy level 2: cells of 4^3 blocks (32 voxels a side)
constexpr int kRangeTile = 4;            // raycast range maps hold one near / far pair per 4x4 pixels
constexpr unsigned kFarInit = 0u;        // range maps' initial values: float bits of +0 (far)
constexpr unsigned kNearInit = 0x7f800000u;   // and of +inf (near)

// Entries of one raycast range map (near or far) for a width x height image.
inline int64_t range_tiles(int width, int height) {
    return (int64_t)((width + kRangeTile - 1) / kRangeTile) * ((height + kRangeTile - 1) / kRangeTile);
}

// The persistent raycast hands out rays in 8x4-pixel tiles, the tiles with the
// longest ranges first: kRayBuckets lists of tile indices, each up to
// ray_tiles(W, H) entries.
constexpr int kRayBuckets = 4;
inline int64_t ray_tiles(int width, int height) { return (int64_t)((width + 7) / 8) * ((height + 3) / 4); }

// Device-resident counters; every data-dependent size lives here so that a
// sequence of calls needs no host round trip (and can be graph captured).
struct Counters {
    long long n_blocks;          // committed pool size
    long long n_blocks_prev;     // pool size before the last allocation
    unsigned int n_visible;      // entries in the integrate visible list
    unsigned int n_visible_rc;   // entries in the raycast visible list
    unsigned long long voxel_updates;
    unsigned long long rays_hit;
    unsigned int error;
    unsigned int pad;
    // totals over all calls before the current one (current = the fields above)
    unsigned long long updates_total;
    unsigned long long visible_total;
    unsigned long long rays_total;
    unsigned long long rc_blocks_total;
    unsigned int rc_next;        // next ray handed out by the persistent raycast
    unsigned int pad2;
    unsigned int rc_bucket[kRayBuckets];   // 8x4-pixel ray tiles per range-length bucket (ray order)
    unsigned long long voxels_touched;     // voxels updated by at least one frame of the current call
    unsigned long long touched_total;
};

// One visible block for the integrate kernel: pool slot, the camera-space
// position of its voxel (0,0,0) computed in double and rounded to float (o),
// the low part of its z (o[2] + oz_lo carries the double value, so that
// T_k = (D - o_z) - (oz_lo + dz) keeps full precision), and the camera-z range
// outside which no voxel of the block can lie within delta of a depth under its
// footprint.
struct __align__(16) VisibleBlock {
    int slot;
    float o[3];
    float oz_lo;
    float zlo, zhi;
    int pad;
};

// Constants of one allocation call (rounded once from double on the host).
struct AllocParams {
    float M[9];          // R / s, row major
    float a[3];          // (t - origin) / s
    float dz;            // delta / J
    float G;             // grid_dim as float
    float fx, fy, cx, cy;
    float depth_min, depth_max;
    int J;
    int nb;
    int width, height;
    unsigned int* err;   // the volume's sticky device error word
};

// Constants of one integrate / raycast call.
struct FrameParams {
    double R[9];         // camera -> world rotation, row major
    double t[3];         // camera centre in world
    double origin[3];
    double s;
    float cs[9];         // cs[3 r + a] = s * R[a][r]: camera axis r per voxel step along world axis a
    float Rs[9];         // R / s (world voxel units per camera unit)
    float q0[3];         // (t - origin) / s
    float oc0[3];        // camera position of voxel (0,0,0): R^T (origin - t)
    float oc0_lo[3];     // oc0 in double minus oc0: (oc0, oc0_lo) carry the double value as a float pair
    float cs_lo[9];      // likewise the low parts of cs
    float fx, fy, cx, cy, cxh, cyh;   // cxh = cx + 1/2
    float depth_min, depth_max;
    float delta, Q, sigma_coeff;
    float w, wmax;       // w_k and W_max of Alg. 1 / Alg. 2 (the rule itself is a kernel template argument)
    int refine_steps;    // Gauss-Newton steps refining T_k in the depth map (0 = off)
    float2 tsc;          // snorm16 scales: (delta / 32767, 32767 / delta)
    float zlo, zhi;      // camera z range a block must reach to matter
    float near_clip, far_clip;
    int width, height;
    int nb, G;
    int n2;              // occupancy cells per axis (cells of 4^3 blocks)
    int cap;             // pool capacity in blocks (index checks of TSDF_DEBUG builds)
    unsigned int* err;   // the volume's sticky device error word
};

// Constants of one batched integrate call: K frames fused in order.
struct BatchParams {
    FrameParams fp[kMaxBatch];
    const float* depth[kMaxBatch];
    const float* var[kMaxBatch];
    const float2* meas[kMaxBatch];   // per-pixel measurement maps written by depth_tiles
    int K;
    int f0;              // frame counter of the batch's first frame
};

// Launch shapes (chosen by tsdf_autotune; none changes any result).
struct LaunchConfig {
    int integrate_vpt;           // voxels per thread of the integrate kernel: 4 or 8
    int integrate_ctas_per_sm;   // persistent integrate CTAs per SM
    int raycast_tile_w, raycast_tile_h;   // raycast CTA tile in pixels
    int raycast_persistent;      // 1: persistent state-machine raycast, 0: one thread per pixel
};

}  // namespace tsdf

struct tsdf_volume {
    tsdf_config cfg;
    int device;
    int num_sms;
    int32_t nb;                    // blocks per axis
    uint64_t n_table;              // nb^3 entries of the block table
    uint32_t n_tiles;              // bitmap scan tiles
    int32_t* blk_slot;             // [n_table] pool slot or -1 (the paper's offset buffer)
    uint32_t* newbits;             // [n_tiles * kTileWords] new-block bitmap
    uint32_t* tile_sums;           // [n_tiles]
    int4* blocks;                  // [cap] bx, by, bz, allocation frame
    uint32_t* occ2;                // bit per 4^3-block cell: holds an allocated block
    int32_t n2;                    // cells per axis
    size_t occ2_words;
    void* T;                       // [cap * 512] in the storage format (tsdf_storage)
    float* P;                      // [cap * 512]
    tsdf::VisibleBlock* visible;   // [cap]
    int* visible_rc;               // [cap]
    tsdf::Counters* ctr;
    unsigned int* range;           // raycast near / far maps (one pair per 4x4 pixels), 2 * range_cap
    int64_t range_cap;             // entries of each map
    int* ray_order;                // [kRayBuckets * ray_order_cap] ray tiles by range-length bucket
    int64_t ray_order_cap;
    float2* dtiles;                // per 8x8-pixel tile (min, max) of the valid depth
    int64_t dtiles_cap;
    tsdf::VisibleBlock* visible_batch;   // [cap * kMaxBatch] per (block, frame) entries of a batch
    float2* dtiles_batch;          // [kMaxBatch * dtiles_batch_stride]
    int64_t dtiles_batch_stride;
    void* mlp_w;                   // learned-variance weights (bfloat16, device) or null
    float2* meas;                  // per pixel (depth, or NaN when it gives no measurement; p_k)
    int64_t var_cap;               // pixels of meas
    float2* meas_batch;            // [kMaxBatch * var_batch_stride] measurement maps of a batch
    int64_t var_batch_stride;
    double* icp_part;              // registration partial sums (lazily allocated)
    double* icp_host;              // pinned host copy of one pass's sums and box (lazily allocated)
    void* mesh_scratch;            // marching cubes: per-block counts and offsets (lazily allocated)
    int mesh_table_ready;          // the case table is in constant memory
    int64_t frame;                 // host copy of the frame counter
    cudaStream_t last_stream;
    tsdf_status host_error;        // sticky CUDA error seen on the host
    tsdf::LaunchConfig lc;
};

namespace tsdf {

// Launchers (tsdf_alloc.cu, tsdf_integrate.cu, tsdf_raycast.cu).
cudaError_t launch_allocate(tsdf_volume* v, const float* depth, const AllocParams& p,
                            int frame, cudaStream_t st);
// rc_cull_too: the integrate stage also starts the raycast of the same pose
// (counters, range maps cleared, visible list), and the raycast that follows
// is launched with rc_culled.
cudaError_t launch_integrate(tsdf_volume* v, const float* depth, const float* var,
                             const FrameParams& p, cudaStream_t st, bool rc_cull_too = false);
cudaError_t launch_integrate_batch(tsdf_volume* v, const BatchParams& bp, cudaStream_t st);
cudaError_t launch_variance_mlp(tsdf_volume* v, const float* depth, const FrameParams& p, float* var,
                                cudaStream_t st);
cudaError_t launch_raycast(tsdf_volume* v, const FrameParams& p, float* depth_out,
                           float* normal_out, float* vertex_out, cudaStream_t st, bool rc_culled = false);
// Raycast with caller-provided near / far range maps (each range_tiles(W, H)
// words) and ray-order lists (kRayBuckets * ray_tiles(W, H) words).
cudaError_t launch_icp_sums(tsdf_volume* v, const float* depth, const tsdf_intrinsics& K, const double pose[16],
                            const float* mv, const float* mn, const double model_pose[16], const tsdf_icp_params& prm,
                            double* host_sums, float* host_box, cudaStream_t st);
int icp_solve(const double* sums, const float* box, double theta, double r[3], double t[3]);
void icp_apply(const double r[3], const double t[3], double pose[16]);
cudaError_t launch_mesh(tsdf_volume* v, float* out, bool emit, long long* n, cudaStream_t st);
int mesh_case(int cs, signed char* edges);
cudaError_t launch_raycast_trace(tsdf_volume* v, const FrameParams& p, unsigned char* t_sector, long long n_t,
                                 unsigned char* table_sector, long long n_table, unsigned long long* counts,
                                 cudaStream_t st);
cudaError_t launch_raycast_ranges(tsdf_volume* v, const FrameParams& p, unsigned int* near_, unsigned int* far_,
                                  int* order, float* depth_out, float* normal_out, float* vertex_out, cudaStream_t st);
cudaError_t launch_quadratic_variance(const float* depth, int64_t n, float a, float* out,
                                      cudaStream_t st);
// One checked read of a pool slot (tsdf_debug_check_slot); sink: one device float.
cudaError_t launch_debug_slot(tsdf_volume* v, long long slot, float* sink, cudaStream_t st);
constexpr double kIdentityPose[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};

// Lazily grown per-image buffers and argument checks (tsdf_volume.cu).
cudaError_t ensure_dtiles(tsdf_volume* v, const tsdf_intrinsics& K, cudaStream_t st);
cudaError_t ensure_batch(tsdf_volume* v, const tsdf_intrinsics& K, cudaStream_t st);
cudaError_t ensure_range(tsdf_volume* v, const tsdf_intrinsics& K, cudaStream_t st);
bool pose_valid(const double* pose);
bool intrinsics_valid(const tsdf_intrinsics* K);

// Host-side constant preparation (tsdf_volume.cu).
AllocParams make_alloc_params(const tsdf_volume* v, const tsdf_intrinsics& K, const double* pose);
FrameParams make_frame_params(const tsdf_volume* v, const tsdf_intrinsics& K, const double* pose);

// Index checks of TSDF_DEBUG builds (the stand-in for a memory checker): a
// check that fails sets kErrBounds in the volume's error word, which
// tsdf_get_status reports as TSDF_ERR_BOUNDS, and the caller skips the access.
// Nothing traps. In release builds every check is true and compiles away.
__device__ __forceinline__ bool in_bounds(unsigned int* err, bool ok) {
#ifdef TSDF_DEBUG
    if (!ok) atomicOr(err, kErrBounds);
    return ok;
#else
    (void)err;
    (void)ok;
    return true;
#endif
}

__device__ __forceinline__ bool depth_ok(float d, float dmin, float dmax) {
    return (fabsf(d) < __int_as_float(0x7f800000)) & (d > 0.0f) & (d >= dmin) & (d <= dmax);
}

// Camera-space bounds of the box spanning voxels [8b - 1, 8b + 8] of a block
// (its samples and the trilinear cells shared with its neighbours), for the
// raycast's range cull and raster: camera z range, projected bounding
// rectangle, and whether the box reaches behind the camera plane. In float from
// the camera position of voxel (0,0,0) (oc0) and the per-voxel steps (cs): a
// few units of rounding at 3 m are far below the pixel of dilation the raster
// adds. Written with explicitly rounded operations so that every file that
// includes it (built with or without contraction) takes the same decisions.
__device__ __forceinline__ void rc_block_box(const FrameParams& p, int4 bc, float zr[2], float rect[4], bool* behind) {
    const float bx = (float)(kSide * bc.x - 1), by = (float)(kSide * bc.y - 1), bz = (float)(kSide * bc.z - 1);
    float oc[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
        oc[r] = __fadd_rn(__fadd_rn(__fadd_rn(p.oc0[r], __fmul_rn(bx, p.cs[3 * r])), __fmul_rn(by, p.cs[3 * r + 1])),
                          __fmul_rn(bz, p.cs[3 * r + 2]));
    const float ext = (float)(kSide + 1);
    float zmin = 3.0e38f, zmax = -3.0e38f, umin = 3.0e38f, umax = -3.0e38f, vmin = 3.0e38f, vmax = -3.0e38f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float ax = (c & 1) ? ext : 0.0f, ay = (c & 2) ? ext : 0.0f, az = (c & 4) ? ext : 0.0f;
        float q[3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
            q[r] = __fadd_rn(__fadd_rn(__fadd_rn(oc[r], __fmul_rn(ax, p.cs[3 * r])), __fmul_rn(ay, p.cs[3 * r + 1])),
                             __fmul_rn(az, p.cs[3 * r + 2]));
        zmin = fminf(zmin, q[2]);
        zmax = fmaxf(zmax, q[2]);
        const float rz = __fdiv_rn(1.0f, fmaxf(q[2], 1e-20f));
        const float u = __fadd_rn(__fmul_rn(__fmul_rn(p.fx, q[0]), rz), p.cx);
        const float v = __fadd_rn(__fmul_rn(__fmul_rn(p.fy, q[1]), rz), p.cy);
        umin = fminf(umin, u); umax = fmaxf(umax, u);
        vmin = fminf(vmin, v); vmax = fmaxf(vmax, v);
    }
    zr[0] = zmin;
    zr[1] = zmax;
    *behind = zmin <= 1e-4f;
    rect[0] = umin; rect[1] = umax; rect[2] = vmin; rect[3] = vmax;
}

// Whether the raycast rasterises block bc: its box reaches [near, far] and,
// when entirely in front of the camera, projects into the image dilated by a
// pixel and a half.
__device__ __forceinline__ bool rc_block_visible(const FrameParams& p, int4 bc) {
    float zr[2], rect[4];
    bool behind;
    rc_block_box(p, bc, zr, rect, &behind);
    bool keep = zr[1] >= p.near_clip && zr[0] <= p.far_clip;
    if (keep && !behind)
        keep = rect[1] >= -1.5f && rect[0] <= (float)p.width + 0.5f && rect[3] >= -1.5f &&
               rect[2] <= (float)p.height + 0.5f;
    return keep;
}

// The raycast call's counters: the last call's counts go to the totals and the
// per-call ones restart. Run by one thread of the first kernel of the call
// (the range clear, or in a graph step the integrate stage's first kernel,
// whose cull also makes the raycast's visible list).
__device__ __forceinline__ void reset_raycast_counters(Counters* ctr) {
    ctr->rc_next = 0;
    for (int b = 0; b < kRayBuckets; ++b) ctr->rc_bucket[b] = 0;
    ctr->rays_total += ctr->rays_hit;
    ctr->rays_hit = 0;
    ctr->rc_blocks_total += ctr->n_visible_rc;
    ctr->n_visible_rc = 0;
}

__device__ __forceinline__ unsigned int warp_sum(unsigned int x) {
    return __reduce_add_sync(0xffffffffu, x);
}

// Programmatic dependent launch. A kernel started by launch_pdl may be
// scheduled while the kernel before it in the stream (or graph) is still
// running; pdl_prologue(), the first statement of every such kernel, waits
// until that kernel has completed and its writes are visible (so nothing is
// read early), then allows the kernel after this one to be scheduled in turn.
// The launch latency of each kernel thus overlaps its predecessor's tail, one
// kernel ahead. Both instructions do nothing when the kernel was launched
// without the attribute.
__device__ __forceinline__ void pdl_prologue() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // a failed launch leaves its error for the caller's cudaGetLastError()
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace tsdf
