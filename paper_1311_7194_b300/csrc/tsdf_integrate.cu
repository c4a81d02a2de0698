// Measurement integration (section "Integration of Measurements", Alg. 3).
//
//   depth_tiles:      per 8x8-pixel tile, the min and max valid measured depth;
//                     per pixel, the measurement map (D, p_k): D is NaN where
//                     the pixel gives no measurement (invalid depth or variance),
//                     so a single band test |D - z| <= delta rejects it too.
//   cull_kernel:      one thread per allocated block; keeps blocks whose box can
//                     project into the image within the depth range where a
//                     voxel can have |T_k| <= delta, and whose projected footprint
//                     holds some depth within delta of the box's depth range (a
//                     conservative superset of the blocks with T_k != chi,
//                     dom(T_k) of section "Updating Sparse Structure"), and stores
//                     the camera-space position of the block's first voxel,
//                     computed in double and split into a float hi/lo pair.
//   integrate_kernel: persistent CTAs of 128 threads walk the visible list; a
//                     thread owns 4 consecutive voxels of an x row, so a warp
//                     covers 128 voxels = 512 contiguous bytes of T and of P.
//                     Each voxel is projected into the depth map first; only
//                     voxels with T_k != chi load, update and store T and P
//                     (float4 per thread), so a warp whose voxels are all out of
//                     the band touches no pool memory. No atomics inside a block.
//
// Precision: at 3 m a float's spacing (2.4e-7 m) exceeds 1e-5 of a 7.5 mm
// truncation, so z is never formed as one float. T_k = (D - z_hi) - (z_lo + dz):
// D - z_hi is exact (Sterbenz: both within a factor 2 whenever |T_k| <= delta),
// z_lo + dz is small, and the result keeps full precision. x and y only choose
// the pixel and need no such care.
//
// In the batched kernel a voxel whose camera z lies outside the block's reach of
// the band (the depth range under the block's footprint widened by delta, from
// the cull) is rejected by its flag: it cannot have |T_k| <= delta. An empty
// range marks a frame of the batch the block cannot reach, and the kernel skips
// that frame for the whole block. For a single frame the range rejects few
// voxels and is not tested.
#include "tsdf_internal.cuh"
#include "tsdf_mlp.cuh"

namespace tsdf {
namespace {

constexpr int kIntegrateThreads = 128;

// Error-free transformations of float arithmetic (Knuth's two-sum, and the
// product by a fused multiply-add): a + b = s + e and a b = p + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// Camera position of the block's voxel (0,0,0), R^T (origin + 8 b s - t) =
// oc0 + sum_a (8 b_a) cs[., a], in float-float arithmetic: oc0 and cs are
// carried as float pairs rounded once from double on the host, each product
// 8 b_a cs is exact (two_prod), and the sums keep their rounding errors
// (two_sum), so the pair (o, lo) holds the double value to about 2^-48 of its
// size (4e-14 m at room scale, far below the 1e-12 m the hi/lo split of z
// needs). o is that value's nearest float. On sm_103a this replaces double
// arithmetic, whose throughput is a small fraction of float's.
__device__ __forceinline__ void cam_block_origin(const FrameParams& p, int4 bc, float o[3], float* z_lo) {
    const float m[3] = {(float)(kSide * bc.x), (float)(kSide * bc.y), (float)(kSide * bc.z)};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float sh = p.oc0[r], sl = p.oc0_lo[r];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float ph, pl, s, e;
            two_prod(m[a], p.cs[3 * r + a], ph, pl);
            pl = __fmaf_rn(m[a], p.cs_lo[3 * r + a], pl);
            two_sum(sh, ph, s, e);
            e = __fadd_rn(e, __fadd_rn(sl, pl));
            two_sum(s, e, sh, sl);
        }
        o[r] = sh;
        if (r == 2) *z_lo = sl;
    }
}

// Conservative visibility of the box spanning voxel offsets [lo, hi] of a block
// whose voxel (0,0,0) sits at camera position oc: the box must reach the camera
// depth range [zlo, zhi] and, when entirely in front of the camera, its
// projection must overlap the image dilated by `pad` pixels.
__device__ __forceinline__ bool box_visible(const FrameParams& p, const float oc[3], float lo, float hi,
                                            float zlo, float zhi, float pad, float* zmin_out,
                                            float* zmax_out, float rect[4]) {
    float zmin = 3.0e38f, zmax = -3.0e38f;
    float umin = 3.0e38f, umax = -3.0e38f, vmin = 3.0e38f, vmax = -3.0e38f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float ax = (c & 1) ? hi : lo, ay = (c & 2) ? hi : lo, az = (c & 4) ? hi : lo;
        const float x = oc[0] + ax * p.cs[0] + ay * p.cs[1] + az * p.cs[2];
        const float y = oc[1] + ax * p.cs[3] + ay * p.cs[4] + az * p.cs[5];
        const float z = oc[2] + ax * p.cs[6] + ay * p.cs[7] + az * p.cs[8];
        zmin = fminf(zmin, z);
        zmax = fmaxf(zmax, z);
        float rz;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rz) : "f"(fmaxf(z, 1e-20f)));   // the rect is padded by a pixel
        const float u = p.fx * x * rz + p.cx, v = p.fy * y * rz + p.cy;
        umin = fminf(umin, u); umax = fmaxf(umax, u);
        vmin = fminf(vmin, v); vmax = fmaxf(vmax, v);
    }
    *zmin_out = zmin;
    *zmax_out = zmax;
    if (zmax < zlo || zmin > zhi) return false;
    if (zmin <= 1e-6f) {
        rect[0] = -1e30f; rect[1] = 1e30f; rect[2] = -1e30f; rect[3] = 1e30f;
        return true;     // the box reaches behind the camera plane: keep it
    }
    rect[0] = umin; rect[1] = umax; rect[2] = vmin; rect[3] = vmax;
    return umax >= -0.5f - pad && umin <= (float)p.width - 0.5f + pad && vmax >= -0.5f - pad &&
           vmin <= (float)p.height - 0.5f + pad;
}

// The integrate call's counters: the last call's counts go to the totals and
// the per-call ones restart. Runs in the first kernel of the call, ahead of
// every kernel that reads them (stream order).
__device__ __forceinline__ void reset_frame_counters(Counters* ctr, bool rc_too) {
    if (rc_too) reset_raycast_counters(ctr);   // this stage also starts the step's raycast
    ctr->updates_total += ctr->voxel_updates;
    ctr->visible_total += ctr->n_visible;
    ctr->touched_total += ctr->voxels_touched;
    ctr->n_visible = 0;
    ctr->voxel_updates = 0;
    ctr->voxels_touched = 0;
}

// Per 8x8-pixel tile: (min, max) of the valid measured depth, (+inf, -inf) when
// the tile has none. Per pixel: meas = (D, p_k), p_k from the variance map when
// one is given, else the quadratic model (a D^2)^2; D becomes NaN when it is
// not a valid depth or p_k is not a positive finite variance. One warp per
// tile, two pixels per lane. Thread 0 also resets the call's counters when
// `reset` is given.
__global__ void __launch_bounds__(256) depth_tiles_kernel(const float* __restrict__ depth,
                                                          const float* __restrict__ var, FrameParams p,
                                                          float2* __restrict__ tiles, float2* __restrict__ meas,
                                                          Counters* __restrict__ reset, int reset_rc) {
    pdl_prologue();
    if (reset && blockIdx.x == 0 && threadIdx.x == 0) reset_frame_counters(reset, reset_rc != 0);
    const int tiles_x = (p.width + kDepthTile - 1) / kDepthTile;
    const int tiles_y = (p.height + kDepthTile - 1) / kDepthTile;
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < tiles_x * tiles_y; t += warps) {
        const int u = (t % tiles_x) * kDepthTile + (lane & 3) * 2;
        const int v = (t / tiles_x) * kDepthTile + (lane >> 2);
        float lo = __int_as_float(0x7f800000), hi = -__int_as_float(0x7f800000);
        if (v < p.height) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (u + k < p.width) {
                    const size_t pix = (size_t)v * p.width + u + k;
                    const float d = __ldg(depth + pix);
                    const bool valid = depth_ok(d, p.depth_min, p.depth_max);
                    if (valid) {
                        lo = fminf(lo, d);
                        hi = fmaxf(hi, d);
                    }
                    float pv;
                    if (var) {
                        pv = __ldg(var + pix);
                    } else {
                        const float sg = __fmul_rn(__fmul_rn(p.sigma_coeff, d), d);
                        pv = __fmul_rn(sg, sg);
                    }
                    const bool use = valid && pv > 0.0f && pv <= 3.0e38f;
                    meas[pix] = make_float2(use ? d : __int_as_float(0x7fc00000), pv);
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) tiles[t] = make_float2(lo, hi);
    }
}

// depth_tiles with the learned-variance network giving each pixel's p_k. A
// CTA of kMlpThreads threads takes kMlpTiles 8x8 tiles per pass, one pixel per
// thread: it stages the pixels' features in shared memory (transposed, input
// by pixel), evaluates both layers for all its pixels as register tiles of 4
// pixels x 8 neurons per thread (a warp shares one group of 8 neurons, so each
// weight is a broadcast load that serves 4 pixels, and each feature load serves
// 8 neurons), and sums each pixel's output over the neurons in order. Every
// neuron's sum runs over its inputs in order, one fused multiply-add each, so
// the outputs are those of mlp_eval bit for bit. The features read a 5x5
// window around each pixel: each pass first copies its tiles' depths with a
// 2-pixel halo (12x12 per tile, NaN outside the image, which no validity test
// accepts, as none accepts a pixel outside it) into shared memory, rows
// kPatchPitch floats apart so that a warp's 4x8 pixels fall on 32 banks.
constexpr int kMlpThreads = 128;
constexpr int kMlpTiles = kMlpThreads / (kDepthTile * kDepthTile);   // 2
static_assert(kMlpThreads == 4 * 32 && kHid == 32, "4 pixel groups of 32 threads, 4 neuron groups of 8");
constexpr int kHalo = 2, kPatch = kDepthTile + 2 * kHalo, kPatchPitch = 24, kPatchFloats = kPatch * kPatchPitch;
static_assert(kPatch <= kPatchPitch && kMlpTiles * kPatchFloats <= kHid * kMlpThreads, "the patches fit in sH");

__global__ void __launch_bounds__(kMlpThreads) depth_tiles_mlp_kernel(const float* __restrict__ depth, FrameParams p,
                                                                      float2* __restrict__ tiles,
                                                                      float2* __restrict__ meas,
                                                                      Counters* __restrict__ reset, int reset_rc,
                                                                      const __nv_bfloat16* __restrict__ mlp_w) {
    pdl_prologue();
    __shared__ __align__(16) float smem[kInferFloats];
    __shared__ __align__(16) float sA[kHid][kMlpThreads];   // features [input][pixel], then layer-2 outputs
    __shared__ __align__(16) float sH[kHid][kMlpThreads];   // layer-1 outputs [neuron][pixel]
    __shared__ float2 sTile[kMlpThreads / 32];
    const MlpInfer m = load_infer(mlp_w, smem);
    if (reset && blockIdx.x == 0 && threadIdx.x == 0) reset_frame_counters(reset, reset_rc != 0);
    const int tiles_x = (p.width + kDepthTile - 1) / kDepthTile;
    const int n_tiles = tiles_x * ((p.height + kDepthTile - 1) / kDepthTile);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int px = threadIdx.x;                        // this thread's pixel in the pass
    const int pg = lane, ng = warp;                    // register tile: pixels 4 pg.., neurons 8 ng..
    for (int base = blockIdx.x * kMlpTiles; base < n_tiles; base += gridDim.x * kMlpTiles) {
        // the pixel: tile base + px / 64, row (px / 8) % 8, column px % 8
        const int t = base + px / (kDepthTile * kDepthTile);
        const int q = px % (kDepthTile * kDepthTile);
        const int u = (t % tiles_x) * kDepthTile + q % kDepthTile;
        const int v = (t / tiles_x) * kDepthTile + q / kDepthTile;
        const bool in = t < n_tiles && u < p.width && v < p.height;
        // the depth patches (sH is free here: the previous pass read it before its last two barriers)
        float* patch = &sH[0][0];
        for (int e = threadIdx.x; e < kMlpTiles * kPatch * kPatch; e += kMlpThreads) {
            const int i = e / (kPatch * kPatch), r = (e / kPatch) % kPatch, c = e % kPatch;
            const int ti = base + i;
            const int x = (ti % tiles_x) * kDepthTile - kHalo + c, y = (ti / tiles_x) * kDepthTile - kHalo + r;
            float dv = __int_as_float(0x7fc00000);
            if (ti < n_tiles && x >= 0 && y >= 0 && x < p.width && y < p.height)
                dv = __ldg(depth + (size_t)y * p.width + x);
            patch[i * kPatchFloats + r * kPatchPitch + c] = dv;
        }
        __syncthreads();
        // this pixel's patch and the image coordinates of its first entry
        const float* pt = patch + (px / (kDepthTile * kDepthTile)) * kPatchFloats;
        const int ox = u - q % kDepthTile - kHalo, oy = v - q / kDepthTile - kHalo;
        auto D = [&](int x, int y, float* dd) {
            *dd = pt[(y - oy) * kPatchPitch + (x - ox)];
            return depth_ok(*dd, p.depth_min, p.depth_max);
        };
        float d = 0.0f, pq = 0.0f;
        bool valid = false, fok = false;
        float f[kIn];
        if (in) {
            valid = D(u, v, &d);
            const float sg = __fmul_rn(__fmul_rn(p.sigma_coeff, d), d);
            pq = __fmul_rn(sg, sg);
            fok = features_from(D, p, u, v, f);
        }
#pragma unroll
        for (int i = 0; i < kIn; ++i) sA[i][px] = fok ? f[i] : 0.0f;
        // tile depth range: each warp holds half a tile
        float lo = valid ? d : __int_as_float(0x7f800000), hi = valid ? d : -__int_as_float(0x7f800000);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) sTile[warp] = make_float2(lo, hi);
        __syncthreads();
        if (threadIdx.x < kMlpTiles && base + threadIdx.x < n_tiles) {
            const float2 a = sTile[2 * threadIdx.x], b = sTile[2 * threadIdx.x + 1];
            tiles[base + threadIdx.x] = make_float2(fminf(a.x, b.x), fmaxf(a.y, b.y));
        }
        // layer 1: sH[j][pixel] = relu(b1[j] + sum_i W1[j][i] f[pixel][i])
        {
            float2 acc[4][4];   // [pixel][neuron pair]
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(m.b1[8 * ng + 2 * c], m.b1[8 * ng + 2 * c + 1]);
            asm volatile("" ::: "memory");
#pragma unroll
            for (int i = 0; i < kIn; ++i) {
                const float4 x = *reinterpret_cast<const float4*>(&sA[i][4 * pg]);
                const float4 w0 = *reinterpret_cast<const float4*>(m.W1t + i * kHid + 8 * ng);
                const float4 w1 = *reinterpret_cast<const float4*>(m.W1t + i * kHid + 8 * ng + 4);
                const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float2 xr = make_float2(xs[r], xs[r]);
                    acc[r][0] = __ffma2_rn(make_float2(w0.x, w0.y), xr, acc[r][0]);
                    acc[r][1] = __ffma2_rn(make_float2(w0.z, w0.w), xr, acc[r][1]);
                    acc[r][2] = __ffma2_rn(make_float2(w1.x, w1.y), xr, acc[r][2]);
                    acc[r][3] = __ffma2_rn(make_float2(w1.z, w1.w), xr, acc[r][3]);
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                *reinterpret_cast<float4*>(&sH[8 * ng + 2 * c][4 * pg]) =
                    make_float4(fmaxf(acc[0][c].x, 0.0f), fmaxf(acc[1][c].x, 0.0f), fmaxf(acc[2][c].x, 0.0f),
                                fmaxf(acc[3][c].x, 0.0f));
                *reinterpret_cast<float4*>(&sH[8 * ng + 2 * c + 1][4 * pg]) =
                    make_float4(fmaxf(acc[0][c].y, 0.0f), fmaxf(acc[1][c].y, 0.0f), fmaxf(acc[2][c].y, 0.0f),
                                fmaxf(acc[3][c].y, 0.0f));
            }
        }
        __syncthreads();
        // layer 2: sA[j][pixel] = relu(b2[j] + sum_i W2[j][i] sH[i][pixel])
        {
            float2 acc[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(m.b2[8 * ng + 2 * c], m.b2[8 * ng + 2 * c + 1]);
            asm volatile("" ::: "memory");
#pragma unroll
            for (int i = 0; i < kHid; ++i) {
                const float4 x = *reinterpret_cast<const float4*>(&sH[i][4 * pg]);
                const float4 w0 = *reinterpret_cast<const float4*>(m.W2t + i * kHid + 8 * ng);
                const float4 w1 = *reinterpret_cast<const float4*>(m.W2t + i * kHid + 8 * ng + 4);
                const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float2 xr = make_float2(xs[r], xs[r]);
                    acc[r][0] = __ffma2_rn(make_float2(w0.x, w0.y), xr, acc[r][0]);
                    acc[r][1] = __ffma2_rn(make_float2(w0.z, w0.w), xr, acc[r][1]);
                    acc[r][2] = __ffma2_rn(make_float2(w1.x, w1.y), xr, acc[r][2]);
                    acc[r][3] = __ffma2_rn(make_float2(w1.z, w1.w), xr, acc[r][3]);
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                *reinterpret_cast<float4*>(&sA[8 * ng + 2 * c][4 * pg]) =
                    make_float4(fmaxf(acc[0][c].x, 0.0f), fmaxf(acc[1][c].x, 0.0f), fmaxf(acc[2][c].x, 0.0f),
                                fmaxf(acc[3][c].x, 0.0f));
                *reinterpret_cast<float4*>(&sA[8 * ng + 2 * c + 1][4 * pg]) =
                    make_float4(fmaxf(acc[0][c].y, 0.0f), fmaxf(acc[1][c].y, 0.0f), fmaxf(acc[2][c].y, 0.0f),
                                fmaxf(acc[3][c].y, 0.0f));
            }
        }
        __syncthreads();
        if (in) {
            float out = m.b3;
#pragma unroll
            for (int j = 0; j < kHid; ++j) out = fmaf(m.W3[j], sA[j][px], out);
            // learned_variance's decision: 0 without features, p_quad outside [-ln 4, ln 64]
            const float pv = !fok ? 0.0f
                             : (out >= -1.3862943611198906f && out <= 4.1588830833596715f) ? pq * expf(out) : pq;
            const bool use = valid && pv > 0.0f && pv <= 3.0e38f;
            meas[(size_t)v * p.width + u] = make_float2(use ? d : __int_as_float(0x7fc00000), pv);
        }
        __syncthreads();   // sA, sTile and sH are rewritten by the next pass
    }
}

// Whether any pixel a voxel of the block can project to holds a depth within
// delta of the block's camera-depth range: when none does, every voxel of the
// block has T_k = chi and the block is skipped. rect: projected corners.
__device__ __forceinline__ bool band_reachable(const FrameParams& p, const float2* __restrict__ tiles,
                                               const float rect[4], float zmin, float zmax, float* dlo,
                                               float* dhi) {
    const float W = (float)p.width, H = (float)p.height;
    // nearest-pixel indices the voxels can round to, widened by one pixel
    const int u0 = max(0, (int)floorf(fminf(fmaxf(rect[0], -4.0f), W + 4.0f) + 0.5f) - 1);
    const int u1 = min(p.width - 1, (int)floorf(fminf(fmaxf(rect[1], -4.0f), W + 4.0f) + 0.5f) + 1);
    const int v0 = max(0, (int)floorf(fminf(fmaxf(rect[2], -4.0f), H + 4.0f) + 0.5f) - 1);
    const int v1 = min(p.height - 1, (int)floorf(fminf(fmaxf(rect[3], -4.0f), H + 4.0f) + 0.5f) + 1);
    if (u0 > u1 || v0 > v1) return false;
    const int tx0 = u0 / kDepthTile, tx1 = u1 / kDepthTile, ty0 = v0 / kDepthTile, ty1 = v1 / kDepthTile;
    if ((tx1 - tx0 + 1) * (ty1 - ty0 + 1) > 256) return true;   // very near blocks: no test
    const int tiles_x = (p.width + kDepthTile - 1) / kDepthTile;
    float lo = __int_as_float(0x7f800000), hi = -__int_as_float(0x7f800000);
    for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) {
            const float2 m = tiles[ty * tiles_x + tx];
            lo = fminf(lo, m.x);
            hi = fmaxf(hi, m.y);
        }
    const float slack = 1.01f * p.delta + 2e-6f * fabsf(zmax);
    *dlo = lo - slack;
    *dhi = hi + slack;
    return lo <= zmax + slack && hi >= zmin - slack;
}

// The visible-list entry of block b for one frame; false when no voxel of the
// block can have T_k != chi in that frame.
__device__ __forceinline__ bool make_entry(const FrameParams& p, const float2* __restrict__ tiles, int4 bc, int slot,
                                           VisibleBlock* e) {
    // visibility from a float32 camera position of the block's first voxel
    // (a few ulps from the exact one: far inside the pixel of padding and the
    // band slack); the float-float position only for blocks that pass
    float of[3];
    const float bx = (float)(kSide * bc.x), by = (float)(kSide * bc.y), bz = (float)(kSide * bc.z);
#pragma unroll
    for (int r = 0; r < 3; ++r)
        of[r] = __fmaf_rn(bz, p.cs[3 * r + 2], __fmaf_rn(by, p.cs[3 * r + 1], __fmaf_rn(bx, p.cs[3 * r], p.oc0[r])));
    float zmin, zmax, rect[4];
    float zlo = -3.0e38f, zhi = 3.0e38f;
    bool keep = box_visible(p, of, 0.0f, (float)(kSide - 1), p.zlo, p.zhi, 1.0f, &zmin, &zmax, rect);
    if (keep && rect[0] > -1e29f) keep = band_reachable(p, tiles, rect, zmin, zmax, &zlo, &zhi);
    e->slot = slot;
    float oz_lo = 0.0f;
    if (keep) cam_block_origin(p, bc, of, &oz_lo);
    for (int r = 0; r < 3; ++r) e->o[r] = of[r];
    e->oz_lo = oz_lo;
    e->zlo = keep ? zlo : 3.0e38f;     // an empty range makes every voxel chi
    e->zhi = keep ? zhi : -3.0e38f;
    e->pad = 0;
    return keep;
}

// kRc: the same pass also starts the raycast of the same pose (a fusion step
// raycasts at the pose it has just fused): it clears the range maps and makes
// the raycast's visible list (rc_block_visible), so the raycast needs no pass
// of its own over the blocks.
template <bool kRc>
__global__ void __launch_bounds__(256) cull_kernel(Counters* __restrict__ ctr, const int4* __restrict__ blocks,
                                                   FrameParams p, const float2* __restrict__ tiles,
                                                   VisibleBlock* __restrict__ vis, int* __restrict__ vis_rc,
                                                   unsigned int* __restrict__ near_, unsigned int* __restrict__ far_,
                                                   long long n_range) {
    pdl_prologue();
    if (kRc)
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_range;
             i += (long long)gridDim.x * blockDim.x) {
            near_[i] = kNearInit;
            far_[i] = kFarInit;
        }
    const long long n = ctr->n_blocks;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); b0 < n; b0 += stride) {
        const long long b = b0 + lane;
        VisibleBlock e;
        const int4 bc = b < n ? blocks[b] : make_int4(0, 0, 0, 0);
        const bool keep = b < n && make_entry(p, tiles, bc, (int)b, &e);
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (m) {
            unsigned base = 0;
            if (lane == __ffs(m) - 1) base = atomicAdd(&ctr->n_visible, (unsigned)__popc(m));
            base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
            const unsigned at = base + __popc(m & lt);
            if (keep && in_bounds(p.err, at < (unsigned)p.cap)) vis[at] = e;
        }
        if (kRc) {
            const bool keep_rc = b < n && rc_block_visible(p, bc);
            const unsigned mr = __ballot_sync(0xffffffffu, keep_rc);
            if (!mr) continue;
            unsigned base = 0;
            if (lane == __ffs(mr) - 1) base = atomicAdd(&ctr->n_visible_rc, (unsigned)__popc(mr));
            base = __shfl_sync(0xffffffffu, base, __ffs(mr) - 1);
            const unsigned at = base + __popc(mr & lt);
            if (keep_rc && in_bounds(p.err, at < (unsigned)p.cap)) vis_rc[at] = (int)b;
        }
    }
}

// Batched cull: a block joins the list when it is visible in any of the K
// frames; its K entries (one per frame, empty for frames it cannot reach) are
// stored together.
__global__ void __launch_bounds__(256) cull_batch_kernel(Counters* __restrict__ ctr, const int4* __restrict__ blocks,
                                                         BatchParams bp, const float2* __restrict__ tiles,
                                                         long long tiles_stride, VisibleBlock* __restrict__ vis) {
    pdl_prologue();
    const long long n = ctr->n_blocks;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); b0 < n; b0 += stride) {
        const long long b = b0 + lane;
        bool keep = false;
        int4 bc = make_int4(0, 0, 0, 0);
        if (b < n) {
            bc = blocks[b];
            for (int k = 0; k < bp.K; ++k) {
                VisibleBlock e;
                keep |= bp.f0 + k >= bc.w && make_entry(bp.fp[k], tiles + k * tiles_stride, bc, (int)b, &e);
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (!m) continue;
        unsigned base = 0;
        if (lane == __ffs(m) - 1) base = atomicAdd(&ctr->n_visible, (unsigned)__popc(m));
        base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
        if (keep && in_bounds(bp.fp[0].err, base + __popc(m & ((1u << lane) - 1u)) < (unsigned)bp.fp[0].cap)) {
            const size_t i = (size_t)(base + __popc(m & ((1u << lane) - 1u)));
            for (int k = 0; k < bp.K; ++k) {
                VisibleBlock e;
                make_entry(bp.fp[k], tiles + k * tiles_stride, bc, (int)b, &e);
                vis[i * kMaxBatch + k] = e;
            }
        }
    }
}

// 1/x by the hardware approximation (at most 1 ulp off, PTX rcp.approx): in the
// Kalman gain that perturbs T by under 1e-6 delta.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 1/x refined by one Newton-Raphson step r + r (1 - x r), which roughly squares
// the approximation's relative error: the projection's pixel choice then
// tracks a correctly rounded 1/z (a voxel within 5e-4 px of a half-pixel line
// may go either way; nearly all others agree with FP64).
__device__ __forceinline__ float rcp_newton(float x) {
    const float r = rcp_approx(x);
    return __fmaf_rn(r, __fmaf_rn(-x, r, 1.0f), r);
}

// T_k refined by Gauss-Newton steps in the depth map (section "Integration of
// Measurements", last paragraph): the measured surface is the depth map
// back-projected with bilinear depth, S(u, v) = D~(u, v) ((u - cx)/fx,
// (v - cy)/fy, 1); steps on |S - X|^2 start at the voxel's projection (u, v);
// an evaluation needs the four pixels valid and within delta of each other.
// T_k is |S - X| at the last valid evaluation, signed by the side of S's
// tangent plane X lies on (camera side positive), or t0 (the z-difference)
// when no evaluation is valid. X = (x, y, zh + zl): the z part is kept as a
// hi/lo pair so that S_z - X_z = (D~ - zh) - zl keeps full precision.
__device__ __forceinline__ float refine_tk(const FrameParams& p, const float* __restrict__ depth, float x, float y,
                                           float zh, float zl, float u, float v, float t0) {
    float dist = -1.0f, side = 1.0f;
    for (int k = 0; k <= p.refine_steps; ++k) {
        const float fi = floorf(u), fj = floorf(v);
        if (!(fi >= 0.0f && fj >= 0.0f && fi + 1.0f < (float)p.width && fj + 1.0f < (float)p.height)) break;
        const int i = (int)fi, j = (int)fj;
        const float* row = depth + (size_t)j * p.width + i;
        const float d00 = __ldg(row), d10 = __ldg(row + 1), d01 = __ldg(row + p.width), d11 = __ldg(row + p.width + 1);
        if (!(depth_ok(d00, p.depth_min, p.depth_max) && depth_ok(d10, p.depth_min, p.depth_max) &&
              depth_ok(d01, p.depth_min, p.depth_max) && depth_ok(d11, p.depth_min, p.depth_max)))
            break;
        if (fmaxf(fmaxf(d00, d10), fmaxf(d01, d11)) - fminf(fminf(d00, d10), fminf(d01, d11)) > p.delta) break;
        const float a = u - fi, b = v - fj;
        const float D = (1.0f - a) * (1.0f - b) * d00 + a * (1.0f - b) * d10 + (1.0f - a) * b * d01 + a * b * d11;
        const float Du = (1.0f - b) * (d10 - d00) + b * (d11 - d01);
        const float Dv = (1.0f - a) * (d01 - d00) + a * (d11 - d10);
        const float rx_ = (u - p.cx) / p.fx, ry_ = (v - p.cy) / p.fy;
        const float S[3] = {D * rx_, D * ry_, D};
        const float Ju[3] = {Du * rx_ + D / p.fx, Du * ry_, Du};
        const float Jv[3] = {Dv * rx_, Dv * ry_ + D / p.fy, Dv};
        const float r[3] = {S[0] - x, S[1] - y, (D - zh) - zl};
        dist = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        float n[3] = {Ju[1] * Jv[2] - Ju[2] * Jv[1], Ju[2] * Jv[0] - Ju[0] * Jv[2], Ju[0] * Jv[1] - Ju[1] * Jv[0]};
        if (n[0] * S[0] + n[1] * S[1] + n[2] * S[2] > 0.0f) {
            n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2];
        }
        side = (-r[0] * n[0] - r[1] * n[1] - r[2] * n[2]) >= 0.0f ? 1.0f : -1.0f;
        if (k == p.refine_steps) break;
        const float a11 = Ju[0] * Ju[0] + Ju[1] * Ju[1] + Ju[2] * Ju[2];
        const float a12 = Ju[0] * Jv[0] + Ju[1] * Jv[1] + Ju[2] * Jv[2];
        const float a22 = Jv[0] * Jv[0] + Jv[1] * Jv[1] + Jv[2] * Jv[2];
        const float g1 = Ju[0] * r[0] + Ju[1] * r[1] + Ju[2] * r[2];
        const float g2 = Jv[0] * r[0] + Jv[1] * r[1] + Jv[2] * r[2];
        const float det = a11 * a22 - a12 * a12;
        if (!(det > 0.0f)) break;
        u -= (a22 * g1 - a12 * g2) / det;
        v -= (a11 * g2 - a12 * g1) / det;
    }
    return dist < 0.0f ? t0 : side * dist;
}

// The projective measurement T_k of two neighbouring voxels of a row (Fusion:
// project x onto the depth map, distance to the measured point; chi when there
// is no measurement), at x offsets lx and lx + 1 from a row start whose camera
// position is (xr, yr, o_z + zr); zr carries the low part of o_z. kZRange:
// voxels outside the entry's camera-z range [zlo, zhi] also fail the flag
// (batched kernel); in the single-frame kernel that range rejects few voxels,
// and the band test alone decides. The nearest pixel is floor(u + 1/2) in
// [0, W), found without a branch: a voxel that fails a test still loads pixel
// 0 and is rejected by the flag (for z <= 1e-30, u and v may be infinite or
// NaN; the flag drops them). Computed with sm_100's paired float
// instructions, each of which rounds both elements exactly as its scalar
// counterpart, so half the floating-point instructions are issued.
template <bool kRefine, bool kZRange = true>
__device__ __forceinline__ void measure2(const FrameParams& p, const VisibleBlock& vb, float lx, float xr, float yr,
                                         float zr, const float2* __restrict__ meas, const float* __restrict__ depth,
                                         float* Tk, float* pk, bool* ok) {
    const float2 L = make_float2(lx, lx + 1.0f);
    const float2 zs = __ffma2_rn(L, make_float2(p.cs[6], p.cs[6]), make_float2(zr, zr));
    const float2 z = __fadd2_rn(make_float2(vb.o[2], vb.o[2]), zs);
    const float2 x = __ffma2_rn(L, make_float2(p.cs[0], p.cs[0]), make_float2(xr, xr));
    const float2 y = __ffma2_rn(L, make_float2(p.cs[3], p.cs[3]), make_float2(yr, yr));
    // 1/z: hardware approximation refined by one Newton-Raphson step, as rcp_newton
    float2 rz = make_float2(rcp_approx(z.x), rcp_approx(z.y));
    const float2 err = __ffma2_rn(make_float2(-z.x, -z.y), rz, make_float2(1.0f, 1.0f));
    rz = __ffma2_rn(rz, err, rz);
    const float2 uf = __ffma2_rn(make_float2(p.fx, p.fx), __fmul2_rn(x, rz), make_float2(p.cxh, p.cxh));
    const float2 vf = __ffma2_rn(make_float2(p.fy, p.fy), __fmul2_rn(y, rz), make_float2(p.cyh, p.cyh));
    const float zv[2] = {z.x, z.y}, uv[2] = {uf.x, uf.y}, vv[2] = {vf.x, vf.y};
    float2 m[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int ui = __float2int_rd(uv[e]), vi = __float2int_rd(vv[e]);
        ok[e] = (zv[e] > 1e-30f) & ((unsigned)ui < (unsigned)p.width) & ((unsigned)vi < (unsigned)p.height);
        if (kZRange) ok[e] &= (zv[e] >= vb.zlo) & (zv[e] <= vb.zhi);
        m[e] = __ldg(meas + (ok[e] ? vi * p.width + ui : 0));   // (D or NaN, p_k)
    }
    const float2 t = __fadd2_rn(__fadd2_rn(make_float2(m[0].x, m[1].x), make_float2(-vb.o[2], -vb.o[2])),
                                make_float2(-zs.x, -zs.y));
    const float tv[2] = {t.x, t.y}, xv[2] = {x.x, x.y}, yv[2] = {y.x, y.y}, zsv[2] = {zs.x, zs.y};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        ok[e] &= fabsf(tv[e]) <= p.delta;                 // false for a NaN D
        Tk[e] = tv[e];
        if (kRefine && ok[e])
            Tk[e] = refine_tk(p, depth, xv[e], yv[e], vb.o[2], zsv[e], uv[e] - 0.5f, vv[e] - 0.5f, tv[e]);
        pk[e] = m[e].y;
    }
}

// One measurement into one voxel, chi is NaN; kRule is a tsdf_update_rule.
//   Alg. 3 (Kalman): (1 - K) P is formed as P p_k / (P + p_k), the same quantity
//     without the cancellation of 1 - K when K is near 1.
//   Alg. 1 (running average): T <- (1 - w) T + w T_k; P untouched.
//   Alg. 2 (weighted average): T <- (W T + w T_k) / (W + w), W <- min(W + w, W_max),
//     with W in P.
template <int kRule>
__device__ __forceinline__ void update(const FrameParams& p, float& T, float& P, float Tk, float pk) {
    if (isnan(T)) {
        T = Tk;
        if (kRule == TSDF_UPDATE_KALMAN) P = pk;
        if (kRule == TSDF_UPDATE_WEIGHTED) P = p.w;
    } else if (kRule == TSDF_UPDATE_KALMAN) {
        P = __fadd_rn(P, p.Q);                            // predict
        const float r = rcp_approx(__fadd_rn(P, pk));
        const float K = __fmul_rn(P, r);                  // gain P / (P + p_k)
        T = __fmaf_rn(K, __fsub_rn(Tk, T), T);            // correct
        P = __fmul_rn(P, __fmul_rn(pk, r));               // (1 - K) P, as P p_k / (P + p_k)
    } else if (kRule == TSDF_UPDATE_AVERAGE) {
        T = __fmaf_rn(p.w, __fsub_rn(Tk, T), T);          // (1 - w) T + w T_k
    } else {
        const float Wn = __fadd_rn(P, p.w);
        T = __fdiv_rn(__fmaf_rn(P, T, __fmul_rn(p.w, Tk)), Wn);
        P = fminf(Wn, p.wmax);
    }
    if (fabsf(T) > p.delta) T = __int_as_float(0x7fc00000);
}

// First voxel (x + 8 y + 64 z) of thread t's run of kVPT voxels along x. The
// threads of a warp cover a box 4 voxels high in y (8 x 4 x 4 for 4 voxels a
// thread, 8 x 4 x 8 for 8), so the measurement-map loads of one instruction
// fall on about 4 image rows rather than 8.
template <int kVPT>
__device__ __forceinline__ int row_start(int t) {
    if (kVPT == 4) {
        const int xg = t & 1, y = ((t >> 1) & 3) | (((t >> 5) & 1) << 2), z = ((t >> 3) & 3) | (((t >> 6) & 1) << 2);
        return 4 * xg + 8 * y + 64 * z;
    }
    const int y = (t & 3) | (((t >> 5) & 1) << 2), z = (t >> 2) & 7;
    return 8 * y + 64 * z;
}

template <int kS, int kVPT, int kRule, bool kRefine>
__global__ void __launch_bounds__(kBlockVoxels / kVPT, 16) integrate_kernel(Counters* __restrict__ ctr,
                                                                        const VisibleBlock* __restrict__ vis,
                                                                        typename Codec<kS>::E* __restrict__ T,
                                                                        float* __restrict__ P,
                                                                        const float2* __restrict__ meas,
                                                                        const float* __restrict__ depth, FrameParams p) {
    pdl_prologue();
    static_assert(kVPT == 4 || kVPT == 8, "a thread owns 4 or 8 consecutive voxels of an x row");
    const unsigned nvis = ctr->n_visible;
    const int v0 = row_start<kVPT>(threadIdx.x);          // first of this thread's voxels
    const float lx0 = (float)(v0 & 7), ly = (float)((v0 >> 3) & 7), lz = (float)(v0 >> 6);
    unsigned updates = 0;
    for (unsigned i = blockIdx.x; i < nvis; i += gridDim.x) {
        const VisibleBlock vb = vis[i];
        if (!in_bounds(p.err, vb.slot >= 0 && vb.slot < p.cap)) continue;   // uniform over the CTA
        // camera position of this thread's row start (lx = 0)
        const float xr = __fmaf_rn(ly, p.cs[1], __fmaf_rn(lz, p.cs[2], vb.o[0]));
        const float yr = __fmaf_rn(ly, p.cs[4], __fmaf_rn(lz, p.cs[5], vb.o[1]));
        const float zr = __fmaf_rn(ly, p.cs[7], __fmaf_rn(lz, p.cs[8], vb.oz_lo));
        float tk[kVPT], pk[kVPT];
        bool ok[kVPT];
        bool any = false;
#pragma unroll
        for (int e = 0; e < kVPT; e += 2)
            measure2<kRefine, false>(p, vb, lx0 + (float)e, xr, yr, zr, meas, depth, &tk[e], &pk[e], &ok[e]);
#pragma unroll
        for (int e = 0; e < kVPT; ++e) any |= ok[e];
        if (!any) continue;
        const size_t off = (size_t)vb.slot * kBlockVoxels + (size_t)v0;
        float tv[kVPT], pv[kVPT];
#pragma unroll
        for (int g = 0; g < kVPT; g += 4) {
            Codec<kS>::load4(T + off + g, tv + g, p.tsc);
            float4 p4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (kRule != TSDF_UPDATE_AVERAGE) p4 = *reinterpret_cast<const float4*>(P + off + g);
            pv[g] = p4.x; pv[g + 1] = p4.y; pv[g + 2] = p4.z; pv[g + 3] = p4.w;
        }
#pragma unroll
        for (int e = 0; e < kVPT; ++e) {
            if (ok[e]) {
                update<kRule>(p, tv[e], pv[e], tk[e], pk[e]);
                ++updates;
            }
        }
#pragma unroll
        for (int g = 0; g < kVPT; g += 4) {
            Codec<kS>::store4(T + off + g, tv + g, p.tsc);
            if (kRule != TSDF_UPDATE_AVERAGE)
                *reinterpret_cast<float4*>(P + off + g) = make_float4(pv[g], pv[g + 1], pv[g + 2], pv[g + 3]);
        }
    }
    updates = warp_sum(updates);
    if ((threadIdx.x & 31) == 0 && updates) {
        atomicAdd(&ctr->voxel_updates, (unsigned long long)updates);
        atomicAdd(&ctr->voxels_touched, (unsigned long long)updates);   // one frame: each update touches a voxel once
    }
}

// K frames in one pass: T and P of a voxel are loaded once (at its first valid
// measurement), updated by Alg. 3 for frames 0..K-1 in order - skipping frames
// before the block's allocation - and stored once. Same measurement and update
// functions as integrate_kernel, so the result equals K sequential calls bit
// for bit.
// The grid is kBatchCtasPerSm CTAs per SM, all resident at once (the launch
// bounds cap the registers accordingly).
constexpr int kBatchCtasPerSm = 12;

template <int kS, int kRule, bool kRefine>
__global__ void __launch_bounds__(kIntegrateThreads, kBatchCtasPerSm) integrate_batch_kernel(Counters* __restrict__ ctr,
                                                                            const VisibleBlock* __restrict__ vis,
                                                                            const int4* __restrict__ blocks,
                                                                            typename Codec<kS>::E* __restrict__ T,
                                                                            float* __restrict__ P, BatchParams bp) {
    pdl_prologue();
    const unsigned nvis = ctr->n_visible;
    const int v0 = threadIdx.x * 4;
    const float lx0 = (float)(v0 & 7), ly = (float)((v0 >> 3) & 7), lz = (float)(v0 >> 6);
    unsigned updates = 0, touched = 0;
    for (unsigned i = blockIdx.x; i < nvis; i += gridDim.x) {
        const VisibleBlock* ve = vis + (size_t)i * kMaxBatch;
        const int slot = ve[0].slot;
        if (!in_bounds(bp.fp[0].err, slot >= 0 && slot < bp.fp[0].cap)) continue;   // uniform over the CTA
        const int first = blocks[slot].w - bp.f0;     // first batch frame that sees the block
        const size_t off = (size_t)slot * kBlockVoxels + (size_t)v0;
        float tv[4], pv[4];
        bool loaded = false;
        unsigned hit = 0;    // bit e: voxel e updated by some frame of the batch
        for (int k = max(first, 0); k < bp.K; ++k) {
            const FrameParams& p = bp.fp[k];
            const VisibleBlock vb = ve[k];
            if (!(vb.zlo <= vb.zhi)) continue;             // a frame the block cannot reach
            const float xr = __fmaf_rn(ly, p.cs[1], __fmaf_rn(lz, p.cs[2], vb.o[0]));
            const float yr = __fmaf_rn(ly, p.cs[4], __fmaf_rn(lz, p.cs[5], vb.o[1]));
            const float zr = __fmaf_rn(ly, p.cs[7], __fmaf_rn(lz, p.cs[8], vb.oz_lo));
            float tk[4], pk[4];
            bool ok[4];
            bool any = false;
#pragma unroll
            for (int e = 0; e < 4; e += 2)
                measure2<kRefine>(p, vb, lx0 + (float)e, xr, yr, zr, bp.meas[k], bp.depth[k], &tk[e], &pk[e], &ok[e]);
#pragma unroll
            for (int e = 0; e < 4; ++e) any |= ok[e];
            if (!any) continue;
            if (!loaded) {
                Codec<kS>::load4(T + off, tv, bp.fp[0].tsc);
                float4 p4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (kRule != TSDF_UPDATE_AVERAGE) p4 = *reinterpret_cast<const float4*>(P + off);
                pv[0] = p4.x; pv[1] = p4.y; pv[2] = p4.z; pv[3] = p4.w;
                loaded = true;
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (ok[e]) {
                    update<kRule>(p, tv[e], pv[e], tk[e], pk[e]);
                    ++updates;
                    hit |= 1u << e;
                }
            }
        }
        touched += (unsigned)__popc(hit);
        if (loaded) {
            Codec<kS>::store4(T + off, tv, bp.fp[0].tsc);
            if (kRule != TSDF_UPDATE_AVERAGE)
                *reinterpret_cast<float4*>(P + off) = make_float4(pv[0], pv[1], pv[2], pv[3]);
        }
    }
    updates = warp_sum(updates);
    touched = warp_sum(touched);
    if ((threadIdx.x & 31) == 0 && updates) {
        atomicAdd(&ctr->voxel_updates, (unsigned long long)updates);
        atomicAdd(&ctr->voxels_touched, (unsigned long long)touched);
    }
}


template <int kS, int kVPT, int kRule, bool kRefine>
void launch_integrate_f(tsdf_volume* v, const float* depth, const FrameParams& p, unsigned grid, cudaStream_t st) {
    auto* T = static_cast<typename Codec<kS>::E*>(v->T);
    constexpr int threads = kBlockVoxels / kVPT;
    launch_pdl(integrate_kernel<kS, kVPT, kRule, kRefine>, dim3(grid), dim3(threads), st, v->ctr, v->visible, T,
               v->P, static_cast<const float2*>(v->meas), depth, p);
}

// The refined measurement is instantiated for 4 voxels per thread only.
template <int kS, int kVPT, int kRule>
void launch_integrate_r(tsdf_volume* v, const float* depth, const FrameParams& p, unsigned grid, cudaStream_t st) {
    if (p.refine_steps > 0)
        launch_integrate_f<kS, 4, kRule, true>(v, depth, p, grid, st);
    else
        launch_integrate_f<kS, kVPT, kRule, false>(v, depth, p, grid, st);
}

template <int kS, int kVPT>
void launch_integrate_v(tsdf_volume* v, const float* depth, const FrameParams& p, unsigned grid, cudaStream_t st) {
    switch (v->cfg.update_rule) {
        case TSDF_UPDATE_AVERAGE: launch_integrate_r<kS, kVPT, TSDF_UPDATE_AVERAGE>(v, depth, p, grid, st); break;
        case TSDF_UPDATE_WEIGHTED: launch_integrate_r<kS, kVPT, TSDF_UPDATE_WEIGHTED>(v, depth, p, grid, st); break;
        default: launch_integrate_r<kS, kVPT, TSDF_UPDATE_KALMAN>(v, depth, p, grid, st); break;
    }
}

template <int kS>
void launch_integrate_s(tsdf_volume* v, const float* depth, const FrameParams& p, unsigned grid, cudaStream_t st) {
    if (v->lc.integrate_vpt == 8)
        launch_integrate_v<kS, 8>(v, depth, p, grid, st);
    else
        launch_integrate_v<kS, 4>(v, depth, p, grid, st);
}

template <int kS, int kRule, bool kRefine>
void launch_integrate_batch_f(tsdf_volume* v, const BatchParams& bp, unsigned grid, cudaStream_t st) {
    auto* T = static_cast<typename Codec<kS>::E*>(v->T);
    launch_pdl(integrate_batch_kernel<kS, kRule, kRefine>, dim3(grid), dim3(kIntegrateThreads), st, v->ctr,
               v->visible_batch, v->blocks, T, v->P, bp);
}

template <int kS, int kRule>
void launch_integrate_batch_r(tsdf_volume* v, const BatchParams& bp, unsigned grid, cudaStream_t st) {
    if (bp.fp[0].refine_steps > 0)
        launch_integrate_batch_f<kS, kRule, true>(v, bp, grid, st);
    else
        launch_integrate_batch_f<kS, kRule, false>(v, bp, grid, st);
}

template <int kS>
void launch_integrate_batch_s(tsdf_volume* v, const BatchParams& bp, unsigned grid, cudaStream_t st) {
    switch (v->cfg.update_rule) {
        case TSDF_UPDATE_AVERAGE: launch_integrate_batch_r<kS, TSDF_UPDATE_AVERAGE>(v, bp, grid, st); break;
        case TSDF_UPDATE_WEIGHTED: launch_integrate_batch_r<kS, TSDF_UPDATE_WEIGHTED>(v, bp, grid, st); break;
        default: launch_integrate_batch_r<kS, TSDF_UPDATE_KALMAN>(v, bp, grid, st); break;
    }
}

}  // namespace

// The measurement map and depth tiles of one frame; with a network set and no
// variance map, the network gives each pixel's p_k inside the same kernel.
void launch_depth_tiles(tsdf_volume* v, const float* depth, const float* var, const FrameParams& p, float2* tiles,
                        float2* meas, Counters* reset, bool reset_rc, cudaStream_t st) {
    const auto* w = static_cast<const __nv_bfloat16*>(v->mlp_w);
    if (!var && w)
        launch_pdl(depth_tiles_mlp_kernel, dim3(v->num_sms * 8), dim3(kMlpThreads), st, depth, p, tiles, meas, reset,
                   (int)reset_rc, w);
    else
        launch_pdl(depth_tiles_kernel, dim3(v->num_sms * 4), dim3(256), st, depth, var, p, tiles, meas, reset,
                   (int)reset_rc);
}

cudaError_t launch_integrate(tsdf_volume* v, const float* depth, const float* var, const FrameParams& p,
                             cudaStream_t st, bool rc_cull_too) {
    launch_depth_tiles(v, depth, var, p, v->dtiles, v->meas, v->ctr, rc_cull_too, st);
    if (rc_cull_too)
        launch_pdl(cull_kernel<true>, dim3(v->num_sms * 8), dim3(256), st, v->ctr, v->blocks, p, v->dtiles, v->visible,
                   v->visible_rc, v->range, v->range + v->range_cap, (long long)range_tiles(p.width, p.height));
    else
        launch_pdl(cull_kernel<false>, dim3(v->num_sms * 8), dim3(256), st, v->ctr, v->blocks, p, v->dtiles, v->visible,
                   (int*)nullptr, (unsigned int*)nullptr, (unsigned int*)nullptr, 0ll);
    const unsigned grid = (unsigned)(v->num_sms * v->lc.integrate_ctas_per_sm);
    switch (v->cfg.storage) {
        case TSDF_STORAGE_F16: launch_integrate_s<TSDF_STORAGE_F16>(v, depth, p, grid, st); break;
        case TSDF_STORAGE_SNORM16: launch_integrate_s<TSDF_STORAGE_SNORM16>(v, depth, p, grid, st); break;
        default: launch_integrate_s<TSDF_STORAGE_F32>(v, depth, p, grid, st); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_integrate_batch(tsdf_volume* v, const BatchParams& bp_in, cudaStream_t st) {
    BatchParams bp = bp_in;
    for (int k = 0; k < bp.K; ++k) {
        float2* mk = v->meas_batch + k * v->var_batch_stride;
        launch_depth_tiles(v, bp.depth[k], bp.var[k], bp.fp[k], v->dtiles_batch + k * v->dtiles_batch_stride, mk,
                           k == 0 ? v->ctr : nullptr, false, st);
        bp.meas[k] = mk;
    }
    launch_pdl(cull_batch_kernel, dim3(v->num_sms * 8), dim3(256), st, v->ctr, v->blocks, bp, v->dtiles_batch,
               v->dtiles_batch_stride, v->visible_batch);
    const unsigned grid = (unsigned)v->num_sms * kBatchCtasPerSm;
    switch (v->cfg.storage) {
        case TSDF_STORAGE_F16: launch_integrate_batch_s<TSDF_STORAGE_F16>(v, bp, grid, st); break;
        case TSDF_STORAGE_SNORM16: launch_integrate_batch_s<TSDF_STORAGE_SNORM16>(v, bp, grid, st); break;
        default: launch_integrate_batch_s<TSDF_STORAGE_F32>(v, bp, grid, st); break;
    }
    return cudaGetLastError();
}

__global__ void quadratic_variance_kernel(const float* __restrict__ depth, long long n, float a,
                                          float* __restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = depth[i];
        float r = 0.0f;
        if (isfinite(d) && d > 0.0f) {
            const float sg = __fmul_rn(__fmul_rn(a, d), d);
            r = __fmul_rn(sg, sg);
        }
        out[i] = r;
    }
}

cudaError_t launch_quadratic_variance(const float* depth, int64_t n, float a, float* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const long long blocks = (n + 255) / 256;
    quadratic_variance_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(depth, n, a, out);
    return cudaGetLastError();
}

}  // namespace tsdf
