// Volume lifecycle and the C ABI entry points of libtsdf (declared in tsdf.h).
//
// Device layout (section "Volumetric Scene Representation", Figs. 4-5: an N^3
// offset buffer, -1 for empty blocks, and a pool of M^3-voxel blocks):
//   blk_slot   int32 [(G/8)^3]        pool slot of each block, -1 = empty. At
//                                     the largest grids used (4096^3 voxels) this
//                                     is 512 MB: cheap on a 270 GB device, and a
//                                     lookup is one load with no probing.
//   blocks     int4  [capacity]       bx, by, bz, allocation frame per slot
//   occ2       bitmap of 4^3-block cells holding any allocated block
//                                     (empty-space skipping in the raycast)
//   T, P       float [capacity * 512] distance and variance, structure of arrays
//                                     so that raycasting streams T alone
//   newbits    uint32 bitmap of blocks allocated by the current call
//   visible    per-call visible block lists; Counters holds every
//              data-dependent size on the device.
// All per-call constants (inverse pose, scaled rotations) are prepared here on
// the host in double precision and passed by value to the kernels.
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "tsdf_internal.cuh"

using tsdf::AllocParams;
using tsdf::Counters;
using tsdf::FrameParams;

namespace {

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

bool pose_ok(const double* pose) {
    if (!pose) return false;
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(pose[i])) return false;
    return true;
}

bool intr_ok(const tsdf_intrinsics* K) {
    if (!K) return false;
    if (!(std::isfinite(K->fx) && std::isfinite(K->fy) && std::isfinite(K->cx) && std::isfinite(K->cy)))
        return false;
    if (K->fx == 0.0f || K->fy == 0.0f) return false;
    if (K->width <= 0 || K->height <= 0) return false;
    return (int64_t)K->width * (int64_t)K->height < (int64_t)1 << 31;
}

// IEEE half -> float for exports of TSDF_STORAGE_F16 volumes.
float half_to_float(uint16_t h) {
    const uint32_t sign = (uint32_t)(h & 0x8000u) << 16;
    const uint32_t ex = (h >> 10) & 0x1fu, man = h & 0x3ffu;
    uint32_t bits;
    if (ex == 0x1fu) {
        bits = sign | 0x7f800000u | (man << 13);          // inf / NaN
    } else if (ex != 0) {
        bits = sign | ((ex + 112u) << 23) | (man << 13);   // normal
    } else if (man == 0) {
        bits = sign;                                         // zero
    } else {                                                 // subnormal: renormalise
        int e = -1;
        uint32_t m = man;
        do {
            m <<= 1;
            ++e;
        } while (!(m & 0x400u));
        bits = sign | ((uint32_t)(112 - e) << 23) | ((m & 0x3ffu) << 13);
    }
    float f;
    std::memcpy(&f, &bits, sizeof(f));
    return f;
}

tsdf_status fail_cuda(tsdf_volume* v, cudaError_t e) {
    if (e == cudaSuccess) return TSDF_OK;
    if (v && v->host_error == TSDF_OK) v->host_error = TSDF_ERR_CUDA;
    return TSDF_ERR_CUDA;
}

void free_all(tsdf_volume* v) {
    cudaFree(v->blk_slot);
    cudaFree(v->newbits);
    cudaFree(v->occ2);
    cudaFree(v->tile_sums);
    cudaFree(v->blocks);
    cudaFree(v->T);
    cudaFree(v->P);
    cudaFree(v->visible);
    cudaFree(v->visible_rc);
    cudaFree(v->ctr);
    cudaFree(v->range);
    cudaFree(v->ray_order);
    cudaFree(v->dtiles);
    cudaFree(v->visible_batch);
    cudaFree(v->dtiles_batch);
    cudaFree(v->mlp_w);
    cudaFree(v->meas);
    cudaFree(v->meas_batch);
    cudaFree(v->icp_part);
    cudaFreeHost(v->icp_host);
    cudaFree(v->mesh_scratch);
}

}  // namespace

namespace tsdf {

AllocParams make_alloc_params(const tsdf_volume* v, const tsdf_intrinsics& K, const double* pose) {
    AllocParams p;
    const double s = (double)v->cfg.voxel_size;
    const double delta = (double)v->cfg.truncation;
    p.J = v->cfg.alloc_half_samples > 0 ? v->cfg.alloc_half_samples : (int)std::ceil(2.0 * delta / s - 1e-6);
    p.dz = (float)(delta / (double)p.J);
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) p.M[3 * r + k] = (float)(pose[4 * r + k] / s);
        p.a[r] = (float)((pose[4 * r + 3] - v->cfg.origin[r]) / s);
    }
    p.G = (float)v->cfg.grid_dim;
    p.fx = K.fx; p.fy = K.fy; p.cx = K.cx; p.cy = K.cy;
    p.depth_min = v->cfg.depth_min;
    p.depth_max = v->cfg.depth_max;
    p.nb = v->nb;
    p.width = K.width;
    p.height = K.height;
    p.err = &v->ctr->error;
    return p;
}

FrameParams make_frame_params(const tsdf_volume* v, const tsdf_intrinsics& K, const double* pose) {
    FrameParams p;
    const double s = (double)v->cfg.voxel_size;
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) p.R[3 * r + k] = pose[4 * r + k];
        p.t[r] = pose[4 * r + 3];
        p.origin[r] = v->cfg.origin[r];
    }
    p.s = s;
    for (int r = 0; r < 3; ++r)
        for (int a = 0; a < 3; ++a) {
            const double c = s * p.R[3 * a + r];
            p.cs[3 * r + a] = (float)c;
            p.cs_lo[3 * r + a] = (float)(c - (double)p.cs[3 * r + a]);
            p.Rs[3 * r + a] = (float)(p.R[3 * r + a] / s);
        }
    for (int r = 0; r < 3; ++r) p.q0[r] = (float)((p.t[r] - p.origin[r]) / s);
    for (int r = 0; r < 3; ++r) {
        const double o = p.R[r] * (p.origin[0] - p.t[0]) + p.R[3 + r] * (p.origin[1] - p.t[1]) +
                         p.R[6 + r] * (p.origin[2] - p.t[2]);
        p.oc0[r] = (float)o;
        p.oc0_lo[r] = (float)(o - (double)p.oc0[r]);
    }
    p.fx = K.fx; p.fy = K.fy; p.cx = K.cx; p.cy = K.cy;
    p.cxh = (float)((double)K.cx + 0.5);
    p.cyh = (float)((double)K.cy + 0.5);
    p.depth_min = v->cfg.depth_min;
    p.depth_max = v->cfg.depth_max;
    p.delta = v->cfg.truncation;
    p.Q = v->cfg.process_variance;
    p.sigma_coeff = v->cfg.sigma_coeff;
    p.w = v->cfg.update_weight;
    p.wmax = v->cfg.weight_max;
    p.refine_steps = v->cfg.refine_steps;
    p.tsc = make_float2((float)((double)v->cfg.truncation / 32767.0), (float)(32767.0 / (double)v->cfg.truncation));
    const double dl = 1.01 * (double)v->cfg.truncation;
    p.zlo = (float)((double)v->cfg.depth_min - dl);
    p.zhi = (float)((double)v->cfg.depth_max + dl);
    p.near_clip = v->cfg.raycast_near;
    p.far_clip = v->cfg.raycast_far;
    p.width = K.width;
    p.height = K.height;
    p.nb = v->nb;
    p.G = v->cfg.grid_dim;
    p.n2 = v->n2;
    p.cap = (int)v->cfg.block_capacity;
    p.err = &v->ctr->error;
    return p;
}

// Lazily grown per-image buffers. Each growth synchronises the stream (and
// frees the old buffer), so it happens only on the first call with a larger
// image; tsdf_graph_create calls them up front so that nothing allocates
// during stream capture.
cudaError_t ensure_dtiles(tsdf_volume* v, const tsdf_intrinsics& K, cudaStream_t st) {
    const int64_t ntiles = (int64_t)((K.width + kDepthTile - 1) / kDepthTile) * ((K.height + kDepthTile - 1) / kDepthTile);
    const int64_t npix = (int64_t)K.width * K.height;
    if (ntiles <= v->dtiles_cap && npix <= v->var_cap) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && ntiles > v->dtiles_cap) {
        e = cudaFree(v->dtiles);
        v->dtiles = nullptr;
        v->dtiles_cap = 0;
        if (e == cudaSuccess) e = cudaMalloc(&v->dtiles, (size_t)ntiles * sizeof(float2));
        if (e == cudaSuccess) v->dtiles_cap = ntiles;
    }
    if (e == cudaSuccess && npix > v->var_cap) {   // measurement map
        e = cudaFree(v->meas);
        v->meas = nullptr;
        v->var_cap = 0;
        if (e == cudaSuccess) e = cudaMalloc(&v->meas, (size_t)npix * sizeof(float2));
        if (e == cudaSuccess) v->var_cap = npix;
    }
    return e;
}

cudaError_t ensure_batch(tsdf_volume* v, const tsdf_intrinsics& K, cudaStream_t st) {
    const int64_t ntiles = (int64_t)((K.width + kDepthTile - 1) / kDepthTile) * ((K.height + kDepthTile - 1) / kDepthTile);
    const int64_t npix = (int64_t)K.width * K.height;
    if (v->visible_batch && ntiles <= v->dtiles_batch_stride && npix <= v->var_batch_stride) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && !v->visible_batch)
        e = cudaMalloc(&v->visible_batch, (size_t)v->cfg.block_capacity * kMaxBatch * sizeof(VisibleBlock));
    if (e == cudaSuccess && ntiles > v->dtiles_batch_stride) {
        e = cudaFree(v->dtiles_batch);
        v->dtiles_batch = nullptr;
        v->dtiles_batch_stride = 0;
        if (e == cudaSuccess) e = cudaMalloc(&v->dtiles_batch, (size_t)ntiles * kMaxBatch * sizeof(float2));
        if (e == cudaSuccess) v->dtiles_batch_stride = ntiles;
    }
    if (e == cudaSuccess && npix > v->var_batch_stride) {
        e = cudaFree(v->meas_batch);
        v->meas_batch = nullptr;
        v->var_batch_stride = 0;
        if (e == cudaSuccess) e = cudaMalloc(&v->meas_batch, (size_t)npix * kMaxBatch * sizeof(float2));
        if (e == cudaSuccess) v->var_batch_stride = npix;
    }
    return e;
}

cudaError_t ensure_range(tsdf_volume* v, const tsdf_intrinsics& K, cudaStream_t st) {
    const int64_t n = range_tiles(K.width, K.height), m = ray_tiles(K.width, K.height);
    if (n <= v->range_cap && m <= v->ray_order_cap) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && n > v->range_cap) {
        e = cudaFree(v->range);
        v->range = nullptr;
        v->range_cap = 0;
        if (e == cudaSuccess) e = cudaMalloc(&v->range, 2 * (size_t)n * sizeof(unsigned int));
        if (e == cudaSuccess) v->range_cap = n;
    }
    if (e == cudaSuccess && m > v->ray_order_cap) {
        e = cudaFree(v->ray_order);
        v->ray_order = nullptr;
        v->ray_order_cap = 0;
        if (e == cudaSuccess) e = cudaMalloc(&v->ray_order, (size_t)kRayBuckets * m * sizeof(int));
        if (e == cudaSuccess) v->ray_order_cap = m;
    }
    return e;
}

bool pose_valid(const double* pose) { return pose_ok(pose); }
bool intrinsics_valid(const tsdf_intrinsics* K) { return intr_ok(K); }

}  // namespace tsdf

extern "C" {

void tsdf_config_default(tsdf_config* c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->voxel_size = 1.5e-3f;
    c->truncation = 7.5e-3f;
    c->grid_dim = 2048;
    for (int r = 0; r < 3; ++r) c->origin[r] = -0.5 * c->grid_dim * (double)c->voxel_size;
    c->block_capacity = (int64_t)1 << 20;
    c->process_variance = 0.0f;
    c->depth_min = 0.1f;
    c->depth_max = 4.0f;
    c->raycast_near = 0.1f;
    c->raycast_far = 4.0f;
    c->sigma_coeff = 1.5e-3f;
    c->storage = TSDF_STORAGE_F32;
    c->alloc_half_samples = 0;
    c->update_rule = TSDF_UPDATE_KALMAN;
    c->update_weight = 0.1f;
    c->weight_max = 1.0f;
    c->refine_steps = 0;
}

const char* tsdf_status_string(tsdf_status s) {
    switch (s) {
        case TSDF_OK: return "ok";
        case TSDF_ERR_INVALID_ARG: return "invalid argument";
        case TSDF_ERR_CAPACITY: return "block pool full: new blocks were dropped";
        case TSDF_ERR_HASH_FULL: return "block table full";
        case TSDF_ERR_CUDA: return "CUDA error";
        case TSDF_ERR_NOT_READY: return "not ready";
        case TSDF_ERR_OUT_OF_MEMORY: return "out of device memory";
        case TSDF_ERR_BOUNDS: return "device index check failed (debug build)";
    }
    return "unknown status";
}

tsdf_status tsdf_create_ex(const tsdf_config* cfg, tsdf_volume** out) {
    if (!cfg || !out) return TSDF_ERR_INVALID_ARG;
    *out = nullptr;
    const tsdf_config& c = *cfg;
    if (!finite_pos(c.voxel_size) || !finite_pos(c.truncation)) return TSDF_ERR_INVALID_ARG;
    if (c.grid_dim <= 0 || c.grid_dim % tsdf::kSide != 0) return TSDF_ERR_INVALID_ARG;
    const uint64_t nb = (uint64_t)(c.grid_dim / tsdf::kSide);
    if (nb * nb * nb >= ((uint64_t)1 << 32)) return TSDF_ERR_INVALID_ARG;
    if (c.block_capacity <= 0 || c.block_capacity > (int64_t)0x7fffffff) return TSDF_ERR_INVALID_ARG;
    if (!(std::isfinite(c.process_variance) && c.process_variance >= 0.0f)) return TSDF_ERR_INVALID_ARG;
    if (!(std::isfinite(c.sigma_coeff) && c.sigma_coeff >= 0.0f)) return TSDF_ERR_INVALID_ARG;
    if (!(c.depth_min >= 0.0f && c.depth_max > c.depth_min && !std::isnan(c.depth_max)))
        return TSDF_ERR_INVALID_ARG;
    if (!(finite_pos(c.raycast_near) && c.raycast_far > c.raycast_near && std::isfinite(c.raycast_far)))
        return TSDF_ERR_INVALID_ARG;
    if (c.storage != TSDF_STORAGE_F32 && c.storage != TSDF_STORAGE_F16 && c.storage != TSDF_STORAGE_SNORM16)
        return TSDF_ERR_INVALID_ARG;
    if (c.alloc_half_samples < 0 || c.alloc_half_samples > 4096) return TSDF_ERR_INVALID_ARG;
    if (c.update_rule < TSDF_UPDATE_KALMAN || c.update_rule > TSDF_UPDATE_WEIGHTED) return TSDF_ERR_INVALID_ARG;
    if (c.refine_steps < 0 || c.refine_steps > 8) return TSDF_ERR_INVALID_ARG;
    if (c.update_rule != TSDF_UPDATE_KALMAN) {
        if (!(std::isfinite(c.update_weight) && c.update_weight > 0.0f)) return TSDF_ERR_INVALID_ARG;
        if (c.update_rule == TSDF_UPDATE_AVERAGE && !(c.update_weight <= 1.0f)) return TSDF_ERR_INVALID_ARG;
        if (c.update_rule == TSDF_UPDATE_WEIGHTED &&
            !(std::isfinite(c.weight_max) && c.weight_max >= c.update_weight))
            return TSDF_ERR_INVALID_ARG;
    }
    for (int r = 0; r < 3; ++r)
        if (!std::isfinite(c.origin[r])) return TSDF_ERR_INVALID_ARG;
    if (c.alloc_half_samples == 0 && std::ceil(2.0 * c.truncation / c.voxel_size - 1e-6) > 4096.0)
        return TSDF_ERR_INVALID_ARG;

    tsdf_volume* v = (tsdf_volume*)std::calloc(1, sizeof(tsdf_volume));
    if (!v) return TSDF_ERR_OUT_OF_MEMORY;
    v->cfg = c;
    v->nb = (int32_t)nb;
    v->n_table = nb * nb * nb;
    const uint64_t words = (v->n_table + 31) / 32;
    v->n_tiles = (uint32_t)((words + tsdf::kTileWords - 1) / tsdf::kTileWords);
    v->n2 = (int32_t)((nb + tsdf::kOcc2 - 1) / tsdf::kOcc2);
    v->occ2_words = ((size_t)v->n2 * v->n2 * v->n2 + 31) / 32;
    v->host_error = TSDF_OK;
    v->lc = tsdf::LaunchConfig{4, 12, 16, 8, 0};
    cudaError_t e = cudaGetDevice(&v->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&v->num_sms, cudaDevAttrMultiProcessorCount, v->device);
    if (e != cudaSuccess) {
        std::free(v);
        return TSDF_ERR_CUDA;
    }
    const size_t cap = (size_t)c.block_capacity;
    bool ok = true;
    ok = ok && cudaMalloc(&v->blk_slot, v->n_table * sizeof(int32_t)) == cudaSuccess;
    ok = ok && cudaMalloc(&v->newbits, (size_t)v->n_tiles * tsdf::kTileWords * sizeof(uint32_t)) == cudaSuccess;
    ok = ok && cudaMalloc(&v->tile_sums, (size_t)v->n_tiles * sizeof(uint32_t)) == cudaSuccess;
    ok = ok && cudaMalloc(&v->blocks, cap * sizeof(int4)) == cudaSuccess;
    ok = ok && cudaMalloc(&v->occ2, v->occ2_words * sizeof(uint32_t)) == cudaSuccess;
    ok = ok && cudaMalloc(&v->T, cap * tsdf::kBlockVoxels * tsdf::storage_bytes(c.storage)) == cudaSuccess;
    ok = ok && cudaMalloc(&v->P, cap * tsdf::kBlockVoxels * sizeof(float)) == cudaSuccess;
    ok = ok && cudaMalloc(&v->visible, cap * sizeof(tsdf::VisibleBlock)) == cudaSuccess;
    ok = ok && cudaMalloc(&v->visible_rc, cap * sizeof(int)) == cudaSuccess;
    ok = ok && cudaMalloc(&v->ctr, sizeof(Counters)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_all(v);
        std::free(v);
        return TSDF_ERR_OUT_OF_MEMORY;
    }
    e = cudaMemset(v->blk_slot, 0xff, v->n_table * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(v->newbits, 0, (size_t)v->n_tiles * tsdf::kTileWords * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(v->ctr, 0, sizeof(Counters));
    if (e == cudaSuccess) e = cudaMemset(v->occ2, 0, v->occ2_words * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_all(v);
        std::free(v);
        return TSDF_ERR_CUDA;
    }
    *out = v;
    return TSDF_OK;
}

tsdf_status tsdf_create(float voxel_size, float truncation, int64_t block_capacity, tsdf_volume** out) {
    tsdf_config c;
    tsdf_config_default(&c);
    c.voxel_size = voxel_size;
    c.truncation = truncation;
    c.block_capacity = block_capacity;
    if (finite_pos(voxel_size))
        for (int r = 0; r < 3; ++r) c.origin[r] = -0.5 * c.grid_dim * (double)voxel_size;
    return tsdf_create_ex(&c, out);
}

void tsdf_destroy(tsdf_volume* v) {
    if (!v) return;
    if (v->last_stream) cudaStreamSynchronize(v->last_stream);
    cudaDeviceSynchronize();
    free_all(v);
    std::free(v);
}

tsdf_status tsdf_reset(tsdf_volume* v, void* stream) {
    if (!v) return TSDF_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(v->blk_slot, 0xff, v->n_table * sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->ctr, 0, sizeof(Counters), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->occ2, 0, v->occ2_words * sizeof(uint32_t), st);
    if (e != cudaSuccess) return fail_cuda(v, e);
    v->frame = 0;
    v->host_error = TSDF_OK;
    v->last_stream = st;
    return TSDF_OK;
}

tsdf_status tsdf_allocate(tsdf_volume* v, const float* depth, const tsdf_intrinsics* K, const double pose_wc[16],
                          void* stream) {
    if (!v || !depth || !intr_ok(K) || !pose_ok(pose_wc)) return TSDF_ERR_INVALID_ARG;
    const AllocParams p = tsdf::make_alloc_params(v, *K, pose_wc);
    cudaStream_t st = (cudaStream_t)stream;
    v->last_stream = st;
    return fail_cuda(v, tsdf::launch_allocate(v, depth, p, (int)v->frame, st));
}

tsdf_status tsdf_integrate(tsdf_volume* v, const float* depth, const float* variance, const tsdf_intrinsics* K,
                           const double pose_wc[16], void* stream) {
    if (!v || !depth || !intr_ok(K) || !pose_ok(pose_wc)) return TSDF_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const cudaError_t eb = tsdf::ensure_dtiles(v, *K, st);
    if (eb != cudaSuccess) return fail_cuda(v, eb);
    const FrameParams p = tsdf::make_frame_params(v, *K, pose_wc);
    v->last_stream = st;
    const tsdf_status s = fail_cuda(v, tsdf::launch_integrate(v, depth, variance, p, st));
    if (s == TSDF_OK) ++v->frame;
    return s;
}

tsdf_status tsdf_integrate_batch(tsdf_volume* v, int32_t K, const float* const* depth,
                                 const float* const* variance, const tsdf_intrinsics* Kin, const double* poses_wc,
                                 void* stream) {
    if (!v || K < 1 || K > tsdf::kMaxBatch || !depth || !intr_ok(Kin) || !poses_wc) return TSDF_ERR_INVALID_ARG;
    for (int k = 0; k < K; ++k) {
        if (!depth[k] || !pose_ok(poses_wc + 16 * k)) return TSDF_ERR_INVALID_ARG;
        if (variance && !variance[k]) return TSDF_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const cudaError_t eb = tsdf::ensure_batch(v, *Kin, st);
    if (eb != cudaSuccess) return fail_cuda(v, eb);
    v->last_stream = st;
    tsdf::BatchParams bp;
    std::memset(&bp, 0, sizeof(bp));
    bp.K = K;
    bp.f0 = (int)v->frame;
    for (int k = 0; k < K; ++k) {
        const AllocParams ap = tsdf::make_alloc_params(v, *Kin, poses_wc + 16 * k);
        const cudaError_t e = tsdf::launch_allocate(v, depth[k], ap, (int)v->frame + k, st);
        if (e != cudaSuccess) return fail_cuda(v, e);
        bp.fp[k] = tsdf::make_frame_params(v, *Kin, poses_wc + 16 * k);
        bp.depth[k] = depth[k];
        bp.var[k] = variance ? variance[k] : nullptr;
    }
    const tsdf_status s = fail_cuda(v, tsdf::launch_integrate_batch(v, bp, st));
    if (s == TSDF_OK) v->frame += K;
    return s;
}

tsdf_status tsdf_raycast(tsdf_volume* v, const tsdf_intrinsics* K, const double pose_wc[16], float* depth_out,
                         float* normal_out, float* vertex_out, void* stream) {
    if (!v || !intr_ok(K) || !pose_ok(pose_wc)) return TSDF_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const cudaError_t eb = tsdf::ensure_range(v, *K, st);
    if (eb != cudaSuccess) return fail_cuda(v, eb);
    const FrameParams p = tsdf::make_frame_params(v, *K, pose_wc);
    v->last_stream = st;
    return fail_cuda(v, tsdf::launch_raycast(v, p, depth_out, normal_out, vertex_out, st));
}

tsdf_status tsdf_raycast_trace(tsdf_volume* v, const tsdf_intrinsics* K, const double pose_wc[16],
                               tsdf_raycast_counts* out, void* stream) {
    if (!v || !out || !intr_ok(K) || !pose_ok(pose_wc)) return TSDF_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const cudaError_t eb = tsdf::ensure_range(v, *K, st);
    if (eb != cudaSuccess) return fail_cuda(v, eb);
    const FrameParams p = tsdf::make_frame_params(v, *K, pose_wc);
    v->last_stream = st;
    const long long n_t = (long long)((v->cfg.block_capacity * tsdf::kBlockVoxels *
                                       (int64_t)tsdf::storage_bytes(v->cfg.storage) + 31) / 32);
    const long long n_table = (long long)((v->n_table + 7) / 8);
    unsigned char *t_sector = nullptr, *table_sector = nullptr;
    unsigned long long* counts = nullptr;
    cudaError_t e = cudaMalloc(&t_sector, (size_t)n_t);
    if (e == cudaSuccess) e = cudaMalloc(&table_sector, (size_t)n_table);
    if (e == cudaSuccess) e = cudaMalloc(&counts, 10 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(t_sector, 0, (size_t)n_t, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(table_sector, 0, (size_t)n_table, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, 10 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = tsdf::launch_raycast_trace(v, p, t_sector, n_t, table_sector, n_table, counts, st);
    unsigned long long c[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    unsigned long long hits = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(c, counts, sizeof(c), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hits, &v->ctr->rays_hit, sizeof(hits), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(t_sector);
    cudaFree(table_sector);
    cudaFree(counts);
    if (e != cudaSuccess) return fail_cuda(v, e);
    out->samples = (int64_t)c[0];
    out->table_lookups = (int64_t)c[1];
    out->t_sectors = (int64_t)c[2];
    out->table_sectors = (int64_t)c[3];
    out->rays = (int64_t)K->width * K->height;
    out->rays_hit = (int64_t)hits;
    out->march_samples = (int64_t)c[4];
    out->skips = (int64_t)c[5];
    out->rescans = (int64_t)c[6];
    out->rescan_samples = (int64_t)c[7];
    out->refine_samples = (int64_t)c[8];
    out->normal_samples = (int64_t)c[9];
    return TSDF_OK;
}

tsdf_status tsdf_mesh(tsdf_volume* v, float* triangles, int64_t max_triangles, int64_t* n_triangles,
                      void* stream) {
    if (!v || !n_triangles || max_triangles < 0 || (triangles && max_triangles == 0)) return TSDF_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    v->last_stream = st;
    long long n = 0;
    cudaError_t e = tsdf::launch_mesh(v, nullptr, false, &n, st);
    if (e != cudaSuccess) return fail_cuda(v, e);
    *n_triangles = (int64_t)n;
    if (!triangles) return TSDF_OK;
    if (n > max_triangles) return TSDF_ERR_CAPACITY;
    e = tsdf::launch_mesh(v, triangles, true, &n, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? TSDF_OK : fail_cuda(v, e);
}

tsdf_status tsdf_mesh_case(int32_t pattern, int32_t* n_triangles, int8_t edges[24]) {
    if (pattern < 0 || pattern > 255 || !n_triangles || !edges) return TSDF_ERR_INVALID_ARG;
    signed char e[24];
    *n_triangles = tsdf::mesh_case(pattern, e);
    for (int k = 0; k < 24; ++k) edges[k] = (int8_t)e[k];
    return TSDF_OK;
}

void tsdf_icp_params_default(tsdf_icp_params* p) {
    if (!p) return;
    p->dist_max = 0.05f;
    p->normal_cos_min = 0.8f;
    p->eig_threshold = 0.005f;
    p->iterations = 10;
}

static bool icp_args_ok(tsdf_volume* v, const float* depth, const tsdf_intrinsics* K, const float* mv,
                        const float* mn, const double* model_pose, const tsdf_icp_params* prm, const double* pose) {
    if (!v || !depth || !mv || !mn || !prm || !intr_ok(K) || !pose_ok(model_pose) || !pose_ok(pose)) return false;
    if (!(std::isfinite(prm->dist_max) && prm->dist_max > 0.0f)) return false;
    if (!(std::isfinite(prm->normal_cos_min) && prm->normal_cos_min >= -1.0f && prm->normal_cos_min <= 1.0f))
        return false;
    if (!(std::isfinite(prm->eig_threshold) && prm->eig_threshold >= 0.0f)) return false;
    return prm->iterations >= 1 && prm->iterations <= 100;
}

tsdf_status tsdf_icp_sums(tsdf_volume* v, const float* depth, const tsdf_intrinsics* K, const float* mv,
                          const float* mn, const double model_pose_wc[16], const tsdf_icp_params* prm,
                          const double pose_wc[16], double sums[29], float box[6], void* stream) {
    if (!icp_args_ok(v, depth, K, mv, mn, model_pose_wc, prm, pose_wc) || !sums || !box) return TSDF_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    v->last_stream = st;
    return fail_cuda(v, tsdf::launch_icp_sums(v, depth, *K, pose_wc, mv, mn, model_pose_wc, *prm, sums, box, st));
}

tsdf_status tsdf_icp_solve(const double sums[29], const float box[6], float theta, double r[3], double t[3],
                           int32_t* rank) {
    if (!sums || !box || !r || !t || !(std::isfinite(theta) && theta >= 0.0f)) return TSDF_ERR_INVALID_ARG;
    const int k = tsdf::icp_solve(sums, box, (double)theta, r, t);
    if (rank) *rank = k;
    return TSDF_OK;
}

tsdf_status tsdf_icp(tsdf_volume* v, const float* depth, const tsdf_intrinsics* K, const float* mv, const float* mn,
                     const double model_pose_wc[16], const tsdf_icp_params* prm, double pose_wc[16],
                     tsdf_icp_result* out, void* stream) {
    if (!icp_args_ok(v, depth, K, mv, mn, model_pose_wc, prm, pose_wc)) return TSDF_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    v->last_stream = st;
    tsdf_icp_result res{0, 0.0, 0, 0};
    for (int it = 0; it < prm->iterations; ++it) {
        double sums[29];
        float box[6];
        const cudaError_t e = tsdf::launch_icp_sums(v, depth, *K, pose_wc, mv, mn, model_pose_wc, *prm, sums, box, st);
        if (e != cudaSuccess) return fail_cuda(v, e);
        res.iterations = it + 1;
        res.matches = (int64_t)sums[28];
        res.rms = sums[28] > 0.0 ? std::sqrt(sums[27] / sums[28]) : 0.0;
        res.rank = 0;
        if (sums[28] < 6.0) continue;
        double r[3], t[3];
        res.rank = tsdf::icp_solve(sums, box, (double)prm->eig_threshold, r, t);
        tsdf::icp_apply(r, t, pose_wc);
    }
    if (out) *out = res;
    return TSDF_OK;
}

tsdf_status tsdf_quadratic_variance(const float* depth, int64_t n, float sigma_coeff, float* var_out,
                                    void* stream) {
    if (n < 0 || (n > 0 && (!depth || !var_out)) || !(std::isfinite(sigma_coeff) && sigma_coeff >= 0.0f))
        return TSDF_ERR_INVALID_ARG;
    return tsdf::launch_quadratic_variance(depth, n, sigma_coeff, var_out, (cudaStream_t)stream) == cudaSuccess
               ? TSDF_OK
               : TSDF_ERR_CUDA;
}

int tsdf_debug_build(void) {
#ifdef TSDF_DEBUG
    return 1;
#else
    return 0;
#endif
}

tsdf_status tsdf_debug_check_slot(tsdf_volume* v, int64_t slot, void* stream) {
    if (!v) return TSDF_ERR_INVALID_ARG;
#ifdef TSDF_DEBUG
    cudaStream_t st = (cudaStream_t)stream;
    float* sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(float));
    if (e == cudaSuccess) e = tsdf::launch_debug_slot(v, (long long)slot, sink, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(sink);
    v->last_stream = st;
    return e == cudaSuccess ? TSDF_OK : fail_cuda(v, e);
#else
    (void)slot;
    (void)stream;
    return TSDF_ERR_NOT_READY;
#endif
}

tsdf_status tsdf_get_status(tsdf_volume* v) {
    if (!v) return TSDF_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(v->last_stream);
    if (e != cudaSuccess) return fail_cuda(v, e);
    if (v->host_error != TSDF_OK) return v->host_error;
    unsigned int err = 0;
    e = cudaMemcpy(&err, &v->ctr->error, sizeof(err), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_cuda(v, e);
    if (err & tsdf::kErrBounds) return TSDF_ERR_BOUNDS;
    if (err & tsdf::kErrCapacity) return TSDF_ERR_CAPACITY;
    return TSDF_OK;
}

tsdf_status tsdf_get_stats(tsdf_volume* v, tsdf_stats* out) {
    if (!v || !out) return TSDF_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(v->last_stream);
    Counters c;
    if (e == cudaSuccess) e = cudaMemcpy(&c, v->ctr, sizeof(c), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_cuda(v, e);
    out->n_blocks = c.n_blocks;
    out->new_blocks = c.n_blocks - c.n_blocks_prev;
    out->visible_blocks = c.n_visible;
    out->voxel_updates = (int64_t)c.voxel_updates;
    out->raycast_blocks = c.n_visible_rc;
    out->rays_hit = (int64_t)c.rays_hit;
    out->frames = v->frame;
    out->voxel_updates_total = (int64_t)(c.updates_total + c.voxel_updates);
    out->visible_blocks_total = (int64_t)(c.visible_total + c.n_visible);
    out->rays_hit_total = (int64_t)(c.rays_total + c.rays_hit);
    out->raycast_blocks_total = (int64_t)(c.rc_blocks_total + c.n_visible_rc);
    out->voxels_touched_total = (int64_t)(c.touched_total + c.voxels_touched);
    return TSDF_OK;
}

tsdf_status tsdf_export(tsdf_volume* v, int32_t* coords_frame, float* T, float* P, int64_t capacity,
                        int64_t* n_out) {
    if (!v || !n_out || capacity < 0) return TSDF_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(v->last_stream);
    long long n = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&n, &v->ctr->n_blocks, sizeof(n), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_cuda(v, e);
    *n_out = n;
    const size_t m = (size_t)(n < capacity ? n : capacity);
    if (m == 0) return TSDF_OK;
    if (coords_frame) e = cudaMemcpy(coords_frame, v->blocks, m * sizeof(int4), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && T) {
        const size_t nv = m * tsdf::kBlockVoxels;
        if (v->cfg.storage == TSDF_STORAGE_F32) {
            e = cudaMemcpy(T, v->T, nv * sizeof(float), cudaMemcpyDeviceToHost);
        } else {
            // 16-bit formats: copy the raw halves / snorm codes, decode on the host
            uint16_t* raw = (uint16_t*)std::malloc(nv * sizeof(uint16_t));
            if (!raw) return TSDF_ERR_OUT_OF_MEMORY;
            e = cudaMemcpy(raw, v->T, nv * sizeof(uint16_t), cudaMemcpyDeviceToHost);
            const float scale = (float)((double)v->cfg.truncation / 32767.0);
            for (size_t i = 0; e == cudaSuccess && i < nv; ++i)
                T[i] = v->cfg.storage == TSDF_STORAGE_F16 ? half_to_float(raw[i])
                       : raw[i] == 0x8000u ? std::nanf("") : (float)(int16_t)raw[i] * scale;
            std::free(raw);
        }
    }
    if (e == cudaSuccess && P) e = cudaMemcpy(P, v->P, m * tsdf::kBlockVoxels * sizeof(float), cudaMemcpyDeviceToHost);
    return fail_cuda(v, e);
}

}  // extern "C"
