// Raycasting of the sparse TSDF (section "Scene Rendering", Fig. 7).
//
// The paper draws the occupied blocks with the graphics pipeline into two range
// textures (nearest front face, farthest back face, clamped to the near and far
// planes) and then raycasts only between them, coarse intersection first, fine
// intersection and normal second. Here, without a graphics API:
//   rc_cull_kernel:   allocated blocks whose box (widened by one voxel, the reach
//                     of trilinear cells shared with neighbours) can project into
//                     the image within [raycast_near, raycast_far].
//   raster_kernel:    one warp per visible block: the block box's projected
//                     bounding rectangle (dilated by a pixel) gets atomicMin of
//                     the box's nearest camera z and atomicMax of its farthest,
//                     on floats ordered as unsigned integers.
//   raycast_kernel:   one thread per pixel marches from near to far in camera z
//                     with step delta/2 over the trilinear field of T; a sample
//                     whose lower corner lies in an unallocated block jumps to
//                     that block's exit. Where the field becomes defined already at
//                     or below zero, the last step is re-scanned in delta/32
//                     substeps for a short positive run. At the first + to - pair
//                     the crossing is
//                     refined by Illinois false position (a secant method that keeps
//                     a bracket) to 0.005 voxel, then
//                     the normal is the central difference of the field.
// The coarse and fine stages run in one kernel: on sm_103a the register budget
// that made the paper split them is not the limit, and fusing them avoids a
// round trip of the per-pixel crossing through memory.
#include "tsdf_internal.cuh"

namespace tsdf {
namespace {

constexpr int kMaxMarch = 8192;     // bound on march iterations per ray
constexpr int kRefine = 10;         // refinement samples per hit (Illinois false position)
constexpr int kFine = 16;           // substeps of the re-scan on entering the field below zero
constexpr unsigned kFarInit = 0u;   // float bits of +0
constexpr unsigned kNearInit = 0x7f800000u;   // float bits of +inf

__device__ __forceinline__ void cam_point(const FrameParams& p, double X, double Y, double Z, float o[3]) {
    const double x = X - p.t[0], y = Y - p.t[1], z = Z - p.t[2];
    o[0] = (float)(p.R[0] * x + p.R[3] * y + p.R[6] * z);
    o[1] = (float)(p.R[1] * x + p.R[4] * y + p.R[7] * z);
    o[2] = (float)(p.R[2] * x + p.R[5] * y + p.R[8] * z);
}

// camera-space corners of the box spanning voxels [8b - 1, 8b + 8] of a block
__device__ __forceinline__ void block_box(const FrameParams& p, int4 bc, float zr[2], float rect[4], bool* behind) {
    float oc[3];
    cam_point(p, p.origin[0] + (double)(kSide * bc.x - 1) * p.s, p.origin[1] + (double)(kSide * bc.y - 1) * p.s,
              p.origin[2] + (double)(kSide * bc.z - 1) * p.s, oc);
    const float ext = (float)(kSide + 1);
    float zmin = 3.0e38f, zmax = -3.0e38f, umin = 3.0e38f, umax = -3.0e38f, vmin = 3.0e38f, vmax = -3.0e38f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float ax = (c & 1) ? ext : 0.0f, ay = (c & 2) ? ext : 0.0f, az = (c & 4) ? ext : 0.0f;
        const float x = oc[0] + ax * p.cs[0] + ay * p.cs[1] + az * p.cs[2];
        const float y = oc[1] + ax * p.cs[3] + ay * p.cs[4] + az * p.cs[5];
        const float z = oc[2] + ax * p.cs[6] + ay * p.cs[7] + az * p.cs[8];
        zmin = fminf(zmin, z);
        zmax = fmaxf(zmax, z);
        const float rz = 1.0f / fmaxf(z, 1e-20f);
        const float u = p.fx * x * rz + p.cx, v = p.fy * y * rz + p.cy;
        umin = fminf(umin, u); umax = fmaxf(umax, u);
        vmin = fminf(vmin, v); vmax = fmaxf(vmax, v);
    }
    zr[0] = zmin;
    zr[1] = zmax;
    *behind = zmin <= 1e-4f;
    rect[0] = umin; rect[1] = umax; rect[2] = vmin; rect[3] = vmax;
}

__global__ void __launch_bounds__(256) rc_cull_kernel(Counters* __restrict__ ctr, const int4* __restrict__ blocks,
                                                      FrameParams p, int* __restrict__ vis) {
    const long long n = ctr->n_blocks;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); b0 < n; b0 += stride) {
        const long long b = b0 + lane;
        bool keep = false;
        if (b < n) {
            float zr[2], rect[4];
            bool behind;
            block_box(p, blocks[b], zr, rect, &behind);
            keep = zr[1] >= p.near_clip && zr[0] <= p.far_clip;
            if (keep && !behind)
                keep = rect[1] >= -1.5f && rect[0] <= (float)p.width + 0.5f && rect[3] >= -1.5f &&
                       rect[2] <= (float)p.height + 0.5f;
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (!m) continue;
        unsigned base = 0;
        if (lane == __ffs(m) - 1) base = atomicAdd(&ctr->n_visible_rc, (unsigned)__popc(m));
        base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
        if (keep) vis[base + __popc(m & ((1u << lane) - 1u))] = (int)b;
    }
}

__global__ void range_clear_kernel(unsigned int* __restrict__ near_, unsigned int* __restrict__ far_, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        near_[i] = kNearInit;
        far_[i] = kFarInit;
    }
}

__global__ void __launch_bounds__(256) raster_kernel(const Counters* __restrict__ ctr, const int* __restrict__ vis,
                                                     const int4* __restrict__ blocks, FrameParams p,
                                                     unsigned int* __restrict__ near_, unsigned int* __restrict__ far_) {
    const unsigned n = ctr->n_visible_rc;
    const int lane = threadIdx.x & 31;
    const unsigned warps = (gridDim.x * blockDim.x) >> 5;
    for (unsigned w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n; w += warps) {
        float zr[2], rect[4];
        bool behind;
        block_box(p, blocks[vis[w]], zr, rect, &behind);
        const float zn = fmaxf(zr[0], p.near_clip), zf = fminf(zr[1], p.far_clip);
        if (!(zn <= zf)) continue;
        int u0 = 0, u1 = p.width - 1, v0 = 0, v1 = p.height - 1;
        if (!behind) {
            u0 = max(u0, (int)floorf(fmaxf(rect[0], -2.0f)) - 1);
            u1 = min(u1, (int)ceilf(fminf(rect[1], (float)p.width + 1.0f)) + 1);
            v0 = max(v0, (int)floorf(fmaxf(rect[2], -2.0f)) - 1);
            v1 = min(v1, (int)ceilf(fminf(rect[3], (float)p.height + 1.0f)) + 1);
        }
        if (u0 > u1 || v0 > v1) continue;
        const int cols = u1 - u0 + 1;
        const int count = cols * (v1 - v0 + 1);
        const unsigned zn_bits = __float_as_uint(zn), zf_bits = __float_as_uint(zf);
        for (int k = lane; k < count; k += 32) {
            const int pix = (v0 + k / cols) * p.width + u0 + k % cols;
            atomicMin(near_ + pix, zn_bits);
            atomicMax(far_ + pix, zf_bits);
        }
    }
}

// Trilinear T at voxel-space point q. Returns 0 = defined (value in *f),
// 1 = undefined (a corner is chi, unallocated or outside the grid),
// 2 = the lower corner's block is unallocated or outside the grid (the caller
// may skip the whole block).
__device__ __forceinline__ int trilinear(const FrameParams& p, const int* __restrict__ table,
                                         const float* __restrict__ T, float qx, float qy, float qz, float* f,
                                         int* blk) {
    const float fx0 = floorf(qx), fy0 = floorf(qy), fz0 = floorf(qz);
    const int ix = (int)fmaxf(fminf(fx0, 1e9f), -1e9f);
    const int iy = (int)fmaxf(fminf(fy0, 1e9f), -1e9f);
    const int iz = (int)fmaxf(fminf(fz0, 1e9f), -1e9f);
    const int bx = ix >> 3, by = iy >> 3, bz = iz >> 3;
    blk[0] = bx; blk[1] = by; blk[2] = bz;
    if (bx < 0 || by < 0 || bz < 0 || bx >= p.nb || by >= p.nb || bz >= p.nb) return 2;
    const int s0 = __ldg(table + (unsigned)bx + (unsigned)p.nb * ((unsigned)by + (unsigned)p.nb * (unsigned)bz));
    if (s0 < 0) return 2;
    if (ix + 1 >= p.G || iy + 1 >= p.G || iz + 1 >= p.G) return 1;
    const float tx = qx - fx0, ty = qy - fy0, tz = qz - fz0;
    float c[8];
    const int lx = ix & 7, ly = iy & 7, lz = iz & 7;
    if (lx < 7 && ly < 7 && lz < 7) {
        const float* b = T + (size_t)s0 * kBlockVoxels + lx + 8 * ly + 64 * lz;
        c[0] = __ldg(b); c[1] = __ldg(b + 1); c[2] = __ldg(b + 8); c[3] = __ldg(b + 9);
        c[4] = __ldg(b + 64); c[5] = __ldg(b + 65); c[6] = __ldg(b + 72); c[7] = __ldg(b + 73);
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int jx = ix + (k & 1), jy = iy + ((k >> 1) & 1), jz = iz + (k >> 2);
            const int s = __ldg(table + (unsigned)(jx >> 3) +
                                (unsigned)p.nb * ((unsigned)(jy >> 3) + (unsigned)p.nb * (unsigned)(jz >> 3)));
            c[k] = s < 0 ? __int_as_float(0x7fc00000)
                         : __ldg(T + (size_t)s * kBlockVoxels + (jx & 7) + 8 * (jy & 7) + 64 * (jz & 7));
        }
    }
    const float c00 = __fmaf_rn(tx, c[1] - c[0], c[0]);
    const float c10 = __fmaf_rn(tx, c[3] - c[2], c[2]);
    const float c01 = __fmaf_rn(tx, c[5] - c[4], c[4]);
    const float c11 = __fmaf_rn(tx, c[7] - c[6], c[6]);
    const float c0 = __fmaf_rn(ty, c10 - c00, c00);
    const float c1 = __fmaf_rn(ty, c11 - c01, c01);
    const float v = __fmaf_rn(tz, c1 - c0, c0);
    *f = v;
    return isnan(v) ? 1 : 0;   // chi (NaN) in any corner makes the sum NaN
}

__global__ void __launch_bounds__(128) raycast_kernel(const FrameParams p, const unsigned int* __restrict__ near_,
                                                      const unsigned int* __restrict__ far_,
                                                      const int* __restrict__ table, const float* __restrict__ T,
                                                      float* __restrict__ depth_out, float* __restrict__ normal_out,
                                                      float* __restrict__ vertex_out, Counters* __restrict__ ctr) {
    const int u = blockIdx.x * 16 + (threadIdx.x & 15);
    const int v = blockIdx.y * 8 + (threadIdx.x >> 4);
    const bool in = u < p.width && v < p.height;
    bool hit = false;
    if (in) {
        const int pix = v * p.width + u;
        const float nanf_ = __int_as_float(0x7fc00000);
        float zs = 0.0f, n[3] = {nanf_, nanf_, nanf_}, vert[3] = {nanf_, nanf_, nanf_};
        const float zn = __uint_as_float(near_[pix]), zf = __uint_as_float(far_[pix]);
        if (zn <= zf) {
            // ray in camera z: world point t + z R dc, in voxel units q0 + z dq
            const float dcx = ((float)u - p.cx) / p.fx, dcy = ((float)v - p.cy) / p.fy;
            const float dqx = p.Rs[0] * dcx + p.Rs[1] * dcy + p.Rs[2];
            const float dqy = p.Rs[3] * dcx + p.Rs[4] * dcy + p.Rs[5];
            const float dqz = p.Rs[6] * dcx + p.Rs[7] * dcy + p.Rs[8];
            const float h = 0.5f * p.delta;
            float z = fmaxf(zn, p.near_clip);
            const float zend = fminf(zf, p.far_clip);
            bool prev_def = false, found = false;
            float fprev = 0.0f, zprev = 0.0f, f = 0.0f;
            int blk[3];
            for (int it = 0; it < kMaxMarch && z <= zend; ++it) {
                const int st = trilinear(p, table, T, __fmaf_rn(z, dqx, p.q0[0]), __fmaf_rn(z, dqy, p.q0[1]),
                                         __fmaf_rn(z, dqz, p.q0[2]), &f, blk);
                if (st == 2) {
                    // leave the lower corner's block: first z where q crosses its box
                    float ze = 3.0e38f;
                    if (dqx > 0.0f) ze = fminf(ze, ((float)(8 * blk[0] + 8) - p.q0[0]) / dqx);
                    if (dqx < 0.0f) ze = fminf(ze, ((float)(8 * blk[0]) - p.q0[0]) / dqx);
                    if (dqy > 0.0f) ze = fminf(ze, ((float)(8 * blk[1] + 8) - p.q0[1]) / dqy);
                    if (dqy < 0.0f) ze = fminf(ze, ((float)(8 * blk[1]) - p.q0[1]) / dqy);
                    if (dqz > 0.0f) ze = fminf(ze, ((float)(8 * blk[2] + 8) - p.q0[2]) / dqz);
                    if (dqz < 0.0f) ze = fminf(ze, ((float)(8 * blk[2]) - p.q0[2]) / dqz);
                    z = fmaxf(ze, z) + 1e-3f * h;
                    prev_def = false;
                    continue;
                }
                const bool def = st == 0;
                if (def && !prev_def && f <= 0.0f && it > 0) {
                    // The field starts here already at or below zero: its positive
                    // side may be a run shorter than one coarse step (the samples
                    // before were undefined). Re-scan the last step finely.
                    bool ldef = false, stop = false;
                    float fl = 0.0f, zl = 0.0f;
                    for (int j = 0; j <= kFine; ++j) {
                        const float zq = j == kFine ? z : z - h + (float)j * (h / (float)kFine);
                        float fq = f;
                        const int sq = j == kFine ? 0
                                                  : trilinear(p, table, T, __fmaf_rn(zq, dqx, p.q0[0]),
                                                              __fmaf_rn(zq, dqy, p.q0[1]), __fmaf_rn(zq, dqz, p.q0[2]),
                                                              &fq, blk);
                        if (sq != 0) {
                            ldef = false;
                            continue;
                        }
                        if (ldef && fl > 0.0f && fq <= 0.0f) {
                            zprev = zl; fprev = fl; z = zq; f = fq;
                            found = true;
                            break;
                        }
                        if (ldef && fl < 0.0f && fq > 0.0f) {
                            stop = true;
                            break;
                        }
                        ldef = true; fl = fq; zl = zq;
                    }
                    if (found || stop) break;
                }
                if (def && prev_def) {
                    if (fprev > 0.0f && f <= 0.0f) {
                        found = true;
                        break;
                    }
                    if (fprev < 0.0f && f > 0.0f) break;   // back face first: miss
                }
                prev_def = def;
                fprev = f;
                zprev = z;
                z += h;
            }
            if (found) {
                // Illinois-modified regula falsi on the bracket [zprev, z]: the
                // retained end's value is halved when the same side is kept twice,
                // which avoids the one-sided stagnation of plain false position on
                // the piecewise-cubic trilinear field.
                float z1 = zprev, f1 = fprev, z2 = z, f2 = f;
                const float eps = 0.005f * (float)p.s;
                int side = 0;
                zs = z1 + (z2 - z1) * (f1 / (f1 - f2));
                for (int r = 0; r < kRefine && z2 - z1 > eps; ++r) {
                    float fs;
                    if (trilinear(p, table, T, __fmaf_rn(zs, dqx, p.q0[0]), __fmaf_rn(zs, dqy, p.q0[1]),
                                  __fmaf_rn(zs, dqz, p.q0[2]), &fs, blk) != 0)
                        break;
                    if (fs > 0.0f) {
                        z1 = zs; f1 = fs;
                        if (side == 1) f2 *= 0.5f;
                        side = 1;
                    } else {
                        z2 = zs; f2 = fs;
                        if (side == -1) f1 *= 0.5f;
                        side = -1;
                    }
                    if (f1 == f2) break;
                    zs = z1 + (z2 - z1) * (f1 / (f1 - f2));
                }
                const float qx = __fmaf_rn(zs, dqx, p.q0[0]), qy = __fmaf_rn(zs, dqy, p.q0[1]),
                            qz = __fmaf_rn(zs, dqz, p.q0[2]);
                float fp[3], fm[3];
                bool ok = true;
                ok = ok && trilinear(p, table, T, qx + 1.0f, qy, qz, &fp[0], blk) == 0;
                ok = ok && trilinear(p, table, T, qx - 1.0f, qy, qz, &fm[0], blk) == 0;
                ok = ok && trilinear(p, table, T, qx, qy + 1.0f, qz, &fp[1], blk) == 0;
                ok = ok && trilinear(p, table, T, qx, qy - 1.0f, qz, &fm[1], blk) == 0;
                ok = ok && trilinear(p, table, T, qx, qy, qz + 1.0f, &fp[2], blk) == 0;
                ok = ok && trilinear(p, table, T, qx, qy, qz - 1.0f, &fm[2], blk) == 0;
                if (ok) {
                    float g[3] = {fp[0] - fm[0], fp[1] - fm[1], fp[2] - fm[2]};
                    const float gn = sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
                    if (gn > 0.0f) {
                        const float sg = (g[0] * dqx + g[1] * dqy + g[2] * dqz) > 0.0f ? -1.0f : 1.0f;
                        const float inv = sg / gn;
                        n[0] = g[0] * inv; n[1] = g[1] * inv; n[2] = g[2] * inv;
                    }
                }
                // world vertex: origin + q s, with q in voxel units
                vert[0] = (float)(p.origin[0] + (double)qx * p.s);
                vert[1] = (float)(p.origin[1] + (double)qy * p.s);
                vert[2] = (float)(p.origin[2] + (double)qz * p.s);
                hit = true;
            }
        }
        if (depth_out) depth_out[pix] = hit ? zs : 0.0f;
        if (normal_out) {
            normal_out[3 * pix] = n[0]; normal_out[3 * pix + 1] = n[1]; normal_out[3 * pix + 2] = n[2];
        }
        if (vertex_out) {
            vertex_out[3 * pix] = vert[0]; vertex_out[3 * pix + 1] = vert[1]; vertex_out[3 * pix + 2] = vert[2];
        }
    }
    const unsigned hits = warp_sum(hit ? 1u : 0u);
    if ((threadIdx.x & 31) == 0 && hits) atomicAdd(&ctr->rays_hit, (unsigned long long)hits);
}

__global__ void reset_rc_counters(Counters* ctr) {
    ctr->rays_total += ctr->rays_hit;
    ctr->rc_blocks_total += ctr->n_visible_rc;
    ctr->n_visible_rc = 0;
    ctr->rays_hit = 0;
}

}  // namespace

cudaError_t launch_raycast(tsdf_volume* v, const FrameParams& p, float* depth_out, float* normal_out,
                           float* vertex_out, cudaStream_t st) {
    const long long npix = (long long)p.width * p.height;
    unsigned int* near_ = v->range;
    unsigned int* far_ = v->range + v->range_pixels;
    reset_rc_counters<<<1, 1, 0, st>>>(v->ctr);
    range_clear_kernel<<<v->num_sms * 4, 256, 0, st>>>(near_, far_, npix);
    rc_cull_kernel<<<v->num_sms * 8, 256, 0, st>>>(v->ctr, v->blocks, p, v->visible_rc);
    raster_kernel<<<v->num_sms * 8, 256, 0, st>>>(v->ctr, v->visible_rc, v->blocks, p, near_, far_);
    const dim3 grid((unsigned)((p.width + 15) / 16), (unsigned)((p.height + 7) / 8));
    raycast_kernel<<<grid, 128, 0, st>>>(p, near_, far_, v->blk_slot, v->T, depth_out, normal_out, vertex_out, v->ctr);
    return cudaGetLastError();
}

cudaError_t launch_raycast_ranges(tsdf_volume* v, const FrameParams& p, unsigned int* near_, unsigned int* far_,
                                  float* depth_out, float* normal_out, float* vertex_out, cudaStream_t st) {
    const long long npix = (long long)p.width * p.height;
    reset_rc_counters<<<1, 1, 0, st>>>(v->ctr);
    range_clear_kernel<<<v->num_sms * 4, 256, 0, st>>>(near_, far_, npix);
    rc_cull_kernel<<<v->num_sms * 8, 256, 0, st>>>(v->ctr, v->blocks, p, v->visible_rc);
    raster_kernel<<<v->num_sms * 8, 256, 0, st>>>(v->ctr, v->visible_rc, v->blocks, p, near_, far_);
    const dim3 grid((unsigned)((p.width + 15) / 16), (unsigned)((p.height + 7) / 8));
    raycast_kernel<<<grid, 128, 0, st>>>(p, near_, far_, v->blk_slot, v->T, depth_out, normal_out, vertex_out, v->ctr);
    return cudaGetLastError();
}

}  // namespace tsdf
