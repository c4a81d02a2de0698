// Raycasting of the sparse TSDF (section "Scene Rendering", Fig. 7).
//
// The paper draws the occupied blocks with the graphics pipeline into two range
// textures (nearest front face, farthest back face, clamped to the near and far
// planes) and then raycasts only between them, coarse intersection first, fine
// intersection and normal second. Here, without a graphics API:
//   rc_cull_kernel:   allocated blocks whose box (widened by one voxel, the reach
//                     of trilinear cells shared with neighbours) can project into
//                     the image within [raycast_near, raycast_far].
//   raster_kernel:    one warp per visible block: every 4x4-pixel tile touched by
//                     the block box's projected bounding rectangle (dilated by a
//                     pixel) gets atomicMin of the box's nearest camera z and
//                     atomicMax of its farthest, on floats ordered as unsigned
//                     integers. Tiles rather than pixels cut the atomics 16-fold;
//                     the range only bounds the march, so a looser one changes
//                     which samples are taken, not which crossings exist.
//   raycast_kernel:   one thread per pixel marches from near to far in camera z
//                     with step delta/2 over the trilinear field of T; a sample
//                     whose lower corner lies in an unallocated block jumps to
//                     the exit of the largest empty cell around it (the block,
//                     or a 4^3-block cell empty in the occupancy map kept by
//                     the allocation). Where the field becomes defined already
//                     at or below zero, the last step is re-scanned in delta/32
//                     substeps for a short positive run. At the first + to -
//                     pair the crossing is refined by Illinois false position
//                     (a secant method that keeps a bracket) to 0.02 voxel,
//                     then the normal is the central difference of the field.
// The coarse and fine stages run in one kernel: on sm_103a the register budget
// that made the paper split them is not the limit, and fusing them avoids a
// round trip of the per-pixel crossing through memory.
#include "tsdf_internal.cuh"

namespace tsdf {
namespace {

constexpr int kMaxMarch = 8192;     // bound on march iterations per ray
constexpr int kRefine = 10;         // refinement samples per hit (Illinois false position)
constexpr int kFine = 16;           // substeps of the re-scan on entering the field below zero

__global__ void __launch_bounds__(256) rc_cull_kernel(Counters* __restrict__ ctr, const int4* __restrict__ blocks,
                                                      FrameParams p, int* __restrict__ vis) {
    pdl_prologue();
    const long long n = ctr->n_blocks;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); b0 < n; b0 += stride) {
        const long long b = b0 + lane;
        const bool keep = b < n && rc_block_visible(p, blocks[b]);
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (!m) continue;
        unsigned base = 0;
        if (lane == __ffs(m) - 1) base = atomicAdd(&ctr->n_visible_rc, (unsigned)__popc(m));
        base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
        const unsigned at = base + __popc(m & ((1u << lane) - 1u));
        if (keep && in_bounds(p.err, at < (unsigned)p.cap)) vis[at] = (int)b;
    }
}

__global__ void range_clear_kernel(unsigned int* __restrict__ near_, unsigned int* __restrict__ far_, long long n,
                                   Counters* __restrict__ ctr) {
    pdl_prologue();
    if (blockIdx.x == 0 && threadIdx.x == 0) reset_raycast_counters(ctr);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        near_[i] = kNearInit;
        far_[i] = kFarInit;
    }
}

__global__ void __launch_bounds__(256) raster_kernel(const Counters* __restrict__ ctr, const int* __restrict__ vis,
                                                     const int4* __restrict__ blocks, FrameParams p,
                                                     unsigned int* __restrict__ near_, unsigned int* __restrict__ far_) {
    pdl_prologue();
    const unsigned n = ctr->n_visible_rc;
    const int lane = threadIdx.x & 31;
    const int tiles_x = (p.width + kRangeTile - 1) / kRangeTile;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned w0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); w0 < n; w0 += stride) {
        // each lane bounds one block: tile rectangle and clipped depth range
        int tx0 = 1, tx1 = 0, ty0 = 1, ty1 = 0;
        unsigned zn_bits = 0, zf_bits = 0;
        if (w0 + lane < n) {
            float zr[2], rect[4];
            bool behind;
            rc_block_box(p, blocks[vis[w0 + lane]], zr, rect, &behind);
            const float zn = fmaxf(zr[0], p.near_clip), zf = fminf(zr[1], p.far_clip);
            if (zn <= zf) {
                int u0 = 0, u1 = p.width - 1, v0 = 0, v1 = p.height - 1;
                if (!behind) {
                    u0 = max(u0, (int)floorf(fmaxf(rect[0], -2.0f)) - 1);
                    u1 = min(u1, (int)ceilf(fminf(rect[1], (float)p.width + 1.0f)) + 1);
                    v0 = max(v0, (int)floorf(fmaxf(rect[2], -2.0f)) - 1);
                    v1 = min(v1, (int)ceilf(fminf(rect[3], (float)p.height + 1.0f)) + 1);
                }
                if (u0 <= u1 && v0 <= v1) {
                    tx0 = u0 / kRangeTile; tx1 = u1 / kRangeTile;
                    ty0 = v0 / kRangeTile; ty1 = v1 / kRangeTile;
                    zn_bits = __float_as_uint(zn);
                    zf_bits = __float_as_uint(zf);
                }
            }
        }
        // the warp writes the lanes' rectangles one after another
        for (int j = 0; j < 32; ++j) {
            const int a0 = __shfl_sync(0xffffffffu, tx0, j), a1 = __shfl_sync(0xffffffffu, tx1, j);
            const int b0 = __shfl_sync(0xffffffffu, ty0, j), b1 = __shfl_sync(0xffffffffu, ty1, j);
            const unsigned zn_j = __shfl_sync(0xffffffffu, zn_bits, j), zf_j = __shfl_sync(0xffffffffu, zf_bits, j);
            if (a0 > a1 || b0 > b1) continue;
            const int cols = a1 - a0 + 1;
            const int count = cols * (b1 - b0 + 1);
            for (int k = lane; k < count; k += 32) {
                const int tile = (b0 + k / cols) * tiles_x + a0 + k % cols;
                if (!in_bounds(p.err, tile >= 0 && tile < tiles_x * ((p.height + kRangeTile - 1) / kRangeTile))) continue;
                atomicMin(near_ + tile, zn_j);
                atomicMax(far_ + tile, zf_j);
            }
        }
    }
}

// Ray order of the persistent raycast: one thread per 8x4-pixel ray tile (the
// unit in which rays are handed out) takes the longest clipped range of its two
// 4x4 range tiles and appends the tile to one of kRayBuckets lists, by that
// length as a fraction of [raycast_near, raycast_far]: > 0.3, > 0.1, > 0.03,
// the rest (and tiles with no range). The raycast hands out the lists in that
// order, so the rays likely to march longest start first and the kernel's tail
// is left with short ones. The order changes no result.
__global__ void __launch_bounds__(256) ray_order_kernel(Counters* __restrict__ ctr, const unsigned int* __restrict__ near_,
                                                        const unsigned int* __restrict__ far_, FrameParams p,
                                                        int* __restrict__ order) {
    pdl_prologue();
    const int tiles_x = (p.width + 7) / 8, n = tiles_x * ((p.height + 3) / 4);
    const int rtiles_x = (p.width + kRangeTile - 1) / kRangeTile;
    const int lane = threadIdx.x & 31;
    const float span = p.far_clip - p.near_clip;
    for (int t0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); t0 < n; t0 += gridDim.x * blockDim.x) {
        const int t = t0 + lane;
        int b = kRayBuckets;
        if (t < n) {
            const int tx = t % tiles_x, ty = t / tiles_x;
            float len = -1.0f;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int rx = 2 * tx + k;
                if (rx < rtiles_x) {
                    const float zn = __uint_as_float(near_[ty * rtiles_x + rx]);
                    const float zf = __uint_as_float(far_[ty * rtiles_x + rx]);
                    if (zn <= zf) len = fmaxf(len, fminf(zf, p.far_clip) - fmaxf(zn, p.near_clip));
                }
            }
            const float f = len / span;
            b = f > 0.3f ? 0 : f > 0.1f ? 1 : f > 0.03f ? 2 : 3;
        }
#pragma unroll
        for (int k = 0; k < kRayBuckets; ++k) {
            const unsigned m = __ballot_sync(0xffffffffu, b == k);
            if (!m) continue;
            unsigned base = 0;
            if (lane == __ffs(m) - 1) base = atomicAdd(&ctr->rc_bucket[k], (unsigned)__popc(m));
            base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
            if (b == k) order[(size_t)k * n + base + __popc(m & ((1u << lane) - 1u))] = t;
        }
    }
}

__device__ __forceinline__ int slot_of(const FrameParams& p, const int* __restrict__ table, int bx, int by, int bz) {
    return __ldg(table + (unsigned)bx + (unsigned)p.nb * ((unsigned)by + (unsigned)p.nb * (unsigned)bz));
}

// kNarrow: the pool index slot * 512 + off fits 32 bits (capacity <= 2^23
// blocks), which saves the 64-bit multiply per corner
template <int kS, bool kNarrow>
__device__ __forceinline__ float voxel(const typename Codec<kS>::E* __restrict__ T, int slot, int off, float2 sc) {
    if (slot < 0) return __int_as_float(0x7fc00000);
    if (kNarrow) return Codec<kS>::load(T + ((unsigned)slot * (unsigned)kBlockVoxels + (unsigned)off), sc);
    return Codec<kS>::load(T + (size_t)slot * kBlockVoxels + off, sc);
}

// Traversal tracing (tsdf_raycast_trace only; compiled out of every other
// kernel): samples, block-table lookups, and flags for each 32-byte sector of
// T and of the block table that a sample reads.
struct TraceState {
    unsigned char* t_sector;       // one flag per 32 B of the T pool
    unsigned char* table_sector;   // one flag per 32 B of the block table
    unsigned long long* counts;    // [0] samples, [1] table lookups
    int t_bytes;                   // bytes per stored T value
};
__device__ TraceState g_trace;

template <int kS>
__device__ __forceinline__ void trace_corner(int slot, int off) {
    if (slot < 0) return;
    const unsigned long long byte = ((unsigned long long)slot * kBlockVoxels + (unsigned)off) * (unsigned)g_trace.t_bytes;
    g_trace.t_sector[byte >> 5] = 1;
}

// counts[4..9]: march samples, empty-space skips, re-scans, re-scan samples,
// refinement samples, normal samples
enum { kTraceMarch = 4, kTraceSkip, kTraceRescan, kTraceRescanSample, kTraceRefineSample, kTraceNormalSample };
template <bool kTrace>
__device__ __forceinline__ void trace_add(int i, unsigned long long n = 1) {
    if (kTrace) atomicAdd(&g_trace.counts[i], n);
}

__device__ __forceinline__ void trace_lookup(const FrameParams& p, int bx, int by, int bz) {
    const unsigned long long e = (unsigned)bx + (unsigned long long)p.nb * ((unsigned)by + (unsigned long long)p.nb * (unsigned)bz);
    g_trace.table_sector[e >> 3] = 1;
    atomicAdd(&g_trace.counts[1], 1ull);
}

// Trilinear T at voxel-space point q. Returns 0 = defined (value in *f),
// 1 = undefined (a corner is chi, unallocated or outside the grid),
// 2 = the lower corner's block is unallocated or outside the grid (the caller
// may skip empty space; blk receives that block's coordinates).
// The 8 corners are fetched by the same instructions whether or not the cell
// crosses a block face (only the extra block lookups are conditional), which
// keeps the lanes of a warp together.
template <int kS, bool kTrace = false, bool kNarrow = false>
__device__ __forceinline__ int trilinear(const FrameParams& p, const int* __restrict__ table,
                                         const typename Codec<kS>::E* __restrict__ T, float qx, float qy, float qz,
                                         float* f, int* blk) {
    if (kTrace) atomicAdd(&g_trace.counts[0], 1ull);
    const float fx0 = floorf(qx), fy0 = floorf(qy), fz0 = floorf(qz);
    const int ix = (int)fmaxf(fminf(fx0, 1e9f), -1e9f);
    const int iy = (int)fmaxf(fminf(fy0, 1e9f), -1e9f);
    const int iz = (int)fmaxf(fminf(fz0, 1e9f), -1e9f);
    const int bx = ix >> 3, by = iy >> 3, bz = iz >> 3;
    blk[0] = bx; blk[1] = by; blk[2] = bz;
    if (bx < 0 || by < 0 || bz < 0 || bx >= p.nb || by >= p.nb || bz >= p.nb) return 2;
    const int s000 = slot_of(p, table, bx, by, bz);
    if (kTrace) trace_lookup(p, bx, by, bz);
    if (s000 < 0) return 2;
    if (ix + 1 >= p.G || iy + 1 >= p.G || iz + 1 >= p.G) return 1;
    const int lx = ix & 7, ly = iy & 7, lz = iz & 7;
    const int ex = lx == 7, ey = ly == 7, ez = lz == 7;
    // Corner (dx, dy, dz) lies in block (bx + ex dx, by + ey dy, bz + ez dz):
    // each distinct block is looked up once (a cell crossing one face needs
    // one more block, two faces three more, three faces seven more).
    int s100 = s000, s010 = s000, s110 = s000, s001 = s000, s101 = s000, s011 = s000, s111 = s000;
    if (ex | ey | ez) {   // corners in up to 8 blocks
        if (ex) s100 = slot_of(p, table, bx + 1, by, bz);
        if (ey) s010 = slot_of(p, table, bx, by + 1, bz);
        if (ez) s001 = slot_of(p, table, bx, by, bz + 1);
        s110 = (ex & ey) ? slot_of(p, table, bx + 1, by + 1, bz) : (ex ? s100 : s010);
        s101 = (ex & ez) ? slot_of(p, table, bx + 1, by, bz + 1) : (ex ? s100 : s001);
        s011 = (ey & ez) ? slot_of(p, table, bx, by + 1, bz + 1) : (ey ? s010 : s001);
        s111 = (ex & ey & ez) ? slot_of(p, table, bx + 1, by + 1, bz + 1) : (ex & ey) ? s110 : (ex & ez) ? s101
               : (ey & ez) ? s011 : ex ? s100 : ey ? s010 : s001;
        if (kTrace) {
            if (ex) trace_lookup(p, bx + 1, by, bz);
            if (ey) trace_lookup(p, bx, by + 1, bz);
            if (ez) trace_lookup(p, bx, by, bz + 1);
            if (ex & ey) trace_lookup(p, bx + 1, by + 1, bz);
            if (ex & ez) trace_lookup(p, bx + 1, by, bz + 1);
            if (ey & ez) trace_lookup(p, bx, by + 1, bz + 1);
            if (ex & ey & ez) trace_lookup(p, bx + 1, by + 1, bz + 1);
        }
    }
    // every corner's block is a pool slot below the capacity or unallocated
    if (!in_bounds(p.err, max(max(max(s000, s100), max(s010, s110)), max(max(s001, s101), max(s011, s111))) < p.cap))
        return 1;
    const int x0 = lx, x1 = ex ? 0 : lx + 1;
    const int y0 = 8 * ly, y1 = ey ? 0 : 8 * (ly + 1);
    const int z0 = 64 * lz, z1 = ez ? 0 : 64 * (lz + 1);
    const float2 sc = p.tsc;
    if (kTrace) {
        trace_corner<kS>(s000, x0 + y0 + z0); trace_corner<kS>(s100, x1 + y0 + z0);
        trace_corner<kS>(s010, x0 + y1 + z0); trace_corner<kS>(s110, x1 + y1 + z0);
        trace_corner<kS>(s001, x0 + y0 + z1); trace_corner<kS>(s101, x1 + y0 + z1);
        trace_corner<kS>(s011, x0 + y1 + z1); trace_corner<kS>(s111, x1 + y1 + z1);
    }
    const float c000 = voxel<kS, kNarrow>(T, s000, x0 + y0 + z0, sc), c100 = voxel<kS, kNarrow>(T, s100, x1 + y0 + z0, sc);
    const float c010 = voxel<kS, kNarrow>(T, s010, x0 + y1 + z0, sc), c110 = voxel<kS, kNarrow>(T, s110, x1 + y1 + z0, sc);
    const float c001 = voxel<kS, kNarrow>(T, s001, x0 + y0 + z1, sc), c101 = voxel<kS, kNarrow>(T, s101, x1 + y0 + z1, sc);
    const float c011 = voxel<kS, kNarrow>(T, s011, x0 + y1 + z1, sc), c111 = voxel<kS, kNarrow>(T, s111, x1 + y1 + z1, sc);
    const float tx = qx - fx0, ty = qy - fy0, tz = qz - fz0;
    const float c00 = __fmaf_rn(tx, c100 - c000, c000);
    const float c10 = __fmaf_rn(tx, c110 - c010, c010);
    const float c01 = __fmaf_rn(tx, c101 - c001, c001);
    const float c11 = __fmaf_rn(tx, c111 - c011, c011);
    const float c0 = __fmaf_rn(ty, c10 - c00, c00);
    const float c1 = __fmaf_rn(ty, c11 - c01, c01);
    const float v = __fmaf_rn(tz, c1 - c0, c0);
    *f = v;
    return isnan(v) ? 1 : 0;   // chi (NaN) in any corner makes the sum NaN
}

__device__ __forceinline__ bool occupied(const unsigned int* __restrict__ occ, int n, int cx, int cy, int cz) {
    const unsigned c = (unsigned)cx + (unsigned)n * ((unsigned)cy + (unsigned)n * (unsigned)cz);
    return (__ldg(occ + (c >> 5)) >> (c & 31u)) & 1u;
}

// Camera z at which the ray leaves the empty cell around block blk: its
// (4 blocks)^3 cell when the occupancy map marks that cell empty, else the block
// itself; outside the grid, where nothing is allocated, its (16 blocks)^3 cell.
// (A 16^3-block occupancy level was measured to cost more than it saves: near
// surfaces its cells are occupied and its lookup only adds a dependent load.)
// inv: 1 / dq per axis (0 where the ray does not move along that axis).
__device__ __forceinline__ float empty_exit(const FrameParams& p, const unsigned int* __restrict__ occ2,
                                            const int blk[3], const float inv[3]) {
    const bool inside = blk[0] >= 0 && blk[1] >= 0 && blk[2] >= 0 && blk[0] < p.nb && blk[1] < p.nb && blk[2] < p.nb;
    int shift = 0;   // log2 of blocks per cell side
    if (!inside)
        shift = 4;   // outside the grid nothing is allocated: a 16^3-block cell
    else if (!occupied(occ2, p.n2, blk[0] >> 2, blk[1] >> 2, blk[2] >> 2))
        shift = 2;
    const float size = (float)(kSide << shift);
    float ze = 3.0e38f;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float lo = (float)((blk[r] >> shift) << shift) * (float)kSide;
        if (inv[r] > 0.0f) ze = fminf(ze, (lo + size - p.q0[r]) * inv[r]);
        if (inv[r] < 0.0f) ze = fminf(ze, (lo - p.q0[r]) * inv[r]);
    }
    return ze;
}

template <int kS, int kTW, int kTH, bool kTrace = false>
__global__ void __launch_bounds__(kTW * kTH) raycast_kernel(const FrameParams p, const unsigned int* __restrict__ near_,
                                                      const unsigned int* __restrict__ far_,
                                                      const int* __restrict__ table,
                                                      const typename Codec<kS>::E* __restrict__ T,
                                                      const unsigned int* __restrict__ occ2,
                                                      float* __restrict__ depth_out, float* __restrict__ normal_out,
                                                      float* __restrict__ vertex_out, Counters* __restrict__ ctr) {
    pdl_prologue();
    const int u = blockIdx.x * kTW + (threadIdx.x % kTW);
    const int v = blockIdx.y * kTH + (threadIdx.x / kTW);
    const bool in = u < p.width && v < p.height;
    bool hit = false;
    if (in) {
        const int pix = v * p.width + u;
        const float nanf_ = __int_as_float(0x7fc00000);
        float zs = 0.0f, n[3] = {nanf_, nanf_, nanf_}, vert[3] = {nanf_, nanf_, nanf_};
        const int tile = (v / kRangeTile) * ((p.width + kRangeTile - 1) / kRangeTile) + u / kRangeTile;
        const float zn = __uint_as_float(near_[tile]), zf = __uint_as_float(far_[tile]);
        if (zn <= zf) {
            // ray in camera z: world point t + z R dc, in voxel units q0 + z dq
            const float dcx = ((float)u - p.cx) / p.fx, dcy = ((float)v - p.cy) / p.fy;
            const float dqx = p.Rs[0] * dcx + p.Rs[1] * dcy + p.Rs[2];
            const float dqy = p.Rs[3] * dcx + p.Rs[4] * dcy + p.Rs[5];
            const float dqz = p.Rs[6] * dcx + p.Rs[7] * dcy + p.Rs[8];
            const float inv[3] = {dqx != 0.0f ? 1.0f / dqx : 0.0f, dqy != 0.0f ? 1.0f / dqy : 0.0f,
                                  dqz != 0.0f ? 1.0f / dqz : 0.0f};
            const float h = 0.5f * p.delta;
            float z = fmaxf(zn, p.near_clip);
            const float zend = fminf(zf, p.far_clip);
            bool prev_def = false, found = false;
            float fprev = 0.0f, zprev = 0.0f, f = 0.0f;
            float zprev_any = z, zstep = h;   // last sample taken and the step since
            int blk[3];
            for (int it = 0; it < kMaxMarch && z <= zend; ++it) {
                trace_add<kTrace>(kTraceMarch);
                const int st = trilinear<kS, kTrace>(p, table, T, __fmaf_rn(z, dqx, p.q0[0]), __fmaf_rn(z, dqy, p.q0[1]),
                                         __fmaf_rn(z, dqz, p.q0[2]), &f, blk);
                if (st == 2) {
                    trace_add<kTrace>(kTraceSkip);
                    // everything before the empty cell's exit is undefined
                    zprev_any = fmaxf(empty_exit(p, occ2, blk, inv), z);
                    z = zprev_any + 1e-3f * h;
                    zstep = z - zprev_any;
                    prev_def = false;
                    continue;
                }
                const bool def = st == 0;
                if (def && !prev_def && f <= 0.0f && it > 0) {
                    // The field starts here already at or below zero: its positive
                    // side may be a run shorter than the last step (the samples
                    // before were undefined). Re-scan the last step finely.
                    bool ldef = false, stop = false;
                    float fl = 0.0f, zl = 0.0f;
                    const float back = fminf(zstep, z - zprev_any);
                    trace_add<kTrace>(kTraceRescan);
                    for (int j = 0; j <= kFine; ++j) {
                        const float zq = j == kFine ? z : z - back + (float)j * (back / (float)kFine);
                        if (j < kFine) trace_add<kTrace>(kTraceRescanSample);
                        float fq = f;
                        const int sq = j == kFine ? 0
                                                  : trilinear<kS, kTrace>(p, table, T, __fmaf_rn(zq, dqx, p.q0[0]),
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
                zprev_any = z;
                // chi or partly unallocated cells: no crossing can be bracketed by
                // this sample, so the march takes a double step (a positive run
                // hidden in it is found by the re-scan above)
                zstep = def ? h : 2.0f * h;
                z += zstep;
            }
            if (found) {
                // Illinois-modified regula falsi on the bracket [zprev, z]: the
                // retained end's value is halved when the same side is kept twice,
                // which avoids the one-sided stagnation of plain false position on
                // the piecewise-cubic trilinear field.
                float z1 = zprev, f1 = fprev, z2 = z, f2 = f;
                const float eps = 0.02f * (float)p.s;
                int side = 0;
                zs = z1 + (z2 - z1) * (f1 / (f1 - f2));
                for (int r = 0; r < kRefine && z2 - z1 > eps; ++r) {
                    float fs;
                    trace_add<kTrace>(kTraceRefineSample);
                    if (trilinear<kS, kTrace>(p, table, T, __fmaf_rn(zs, dqx, p.q0[0]), __fmaf_rn(zs, dqy, p.q0[1]),
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
                trace_add<kTrace>(kTraceNormalSample);
                ok = ok && trilinear<kS, kTrace>(p, table, T, qx + 1.0f, qy, qz, &fp[0], blk) == 0;
                if (ok) trace_add<kTrace>(kTraceNormalSample);
                ok = ok && trilinear<kS, kTrace>(p, table, T, qx - 1.0f, qy, qz, &fm[0], blk) == 0;
                if (ok) trace_add<kTrace>(kTraceNormalSample);
                ok = ok && trilinear<kS, kTrace>(p, table, T, qx, qy + 1.0f, qz, &fp[1], blk) == 0;
                if (ok) trace_add<kTrace>(kTraceNormalSample);
                ok = ok && trilinear<kS, kTrace>(p, table, T, qx, qy - 1.0f, qz, &fm[1], blk) == 0;
                if (ok) trace_add<kTrace>(kTraceNormalSample);
                ok = ok && trilinear<kS, kTrace>(p, table, T, qx, qy, qz + 1.0f, &fp[2], blk) == 0;
                if (ok) trace_add<kTrace>(kTraceNormalSample);
                ok = ok && trilinear<kS, kTrace>(p, table, T, qx, qy, qz - 1.0f, &fm[2], blk) == 0;
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

// Persistent variant of raycast_kernel with the same per-ray operations, so the
// same results bit for bit. A warp draws one 8x4-pixel ray tile at a time from
// an atomic counter (in the ray order of ray_order_kernel) and draws the next
// only when none of its 32 rays is still marching: neighbouring rays cross the
// same blocks at about the same step, so the lanes stay on one path and share
// cache lines. (Refilling idle lanes with rays of other tiles while the rest
// march keeps more lanes busy but splits the warp between march phases: a
// refill at 12, 20 or 28 idle lanes was 4.4, 3.0 and 1.0 % slower.) Lanes only
// march (and, rarely, re-scan); a lane that brackets a crossing pushes the
// bracket to its warp's queue in shared memory. When 32 brackets are queued
// (or no rays are left) the whole warp refines them and takes their six normal
// samples together, one bracket per lane, so neither stage runs with idle
// lanes and the six independent normal samples are in flight at once.
constexpr int kRcWarps = 4;          // warps per CTA
constexpr int kQueue = 64;           // brackets per warp queue (< 32 queued + 32 pushed)

// j-th of the kFine re-scan points of the step (zt - back, zt]
__device__ __forceinline__ float zt_minus(float zt, float back, int j) {
    return zt - back + (float)j * (back / (float)kFine);
}

// One point of a re-scan (the step before a sample that found the field
// already at or below zero): sq the point's trilinear status, fq its value, zq
// its camera z; ldef / fa / za the last point (defined, value, z). A + to -
// pair of defined points brackets the crossing; a - to + pair ends the ray.
__device__ __forceinline__ void rescan_step(int sq, float fq, float zq, bool& ldef, float& fa, float& za, float* b1,
                                            float* c1, float* b2, float* c2, bool* push, bool* miss, bool* done) {
    if (sq != 0) {
        ldef = false;
    } else if (ldef && fa > 0.0f && fq <= 0.0f) {
        *b1 = za; *c1 = fa; *b2 = zq; *c2 = fq;
        *push = true;
        *done = true;
    } else if (ldef && fa < 0.0f && fq > 0.0f) {
        *miss = true;
        *done = true;
    } else {
        ldef = true; fa = fq; za = zq;
    }
}

template <int kS, bool kNarrow>
__device__ __forceinline__ void refine_and_shade(const FrameParams& p, const int* __restrict__ table,
                                                 const typename Codec<kS>::E* __restrict__ T, int pix, float z1,
                                                 float f1, float z2, float f2, float dqx, float dqy, float dqz,
                                                 float* __restrict__ depth_out, float* __restrict__ normal_out,
                                                 float* __restrict__ vertex_out) {
    const float nanf_ = __int_as_float(0x7fc00000);
    const float eps = 0.02f * (float)p.s;
    int blk[3];
    int side = 0;
    float zs = z1 + (z2 - z1) * (f1 / (f1 - f2));
    for (int r = 0; r < kRefine && z2 - z1 > eps; ++r) {
        float fs;
        if (trilinear<kS, false, kNarrow>(p, table, T, __fmaf_rn(zs, dqx, p.q0[0]), __fmaf_rn(zs, dqy, p.q0[1]),
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
    const float qx = __fmaf_rn(zs, dqx, p.q0[0]), qy = __fmaf_rn(zs, dqy, p.q0[1]), qz = __fmaf_rn(zs, dqz, p.q0[2]);
    float fp[3], fm[3];
    const int s0 = trilinear<kS, false, kNarrow>(p, table, T, qx + 1.0f, qy, qz, &fp[0], blk);
    const int s1 = trilinear<kS, false, kNarrow>(p, table, T, qx - 1.0f, qy, qz, &fm[0], blk);
    const int s2 = trilinear<kS, false, kNarrow>(p, table, T, qx, qy + 1.0f, qz, &fp[1], blk);
    const int s3 = trilinear<kS, false, kNarrow>(p, table, T, qx, qy - 1.0f, qz, &fm[1], blk);
    const int s4 = trilinear<kS, false, kNarrow>(p, table, T, qx, qy, qz + 1.0f, &fp[2], blk);
    const int s5 = trilinear<kS, false, kNarrow>(p, table, T, qx, qy, qz - 1.0f, &fm[2], blk);
    float n0 = nanf_, n1 = nanf_, n2 = nanf_;
    if ((s0 | s1 | s2 | s3 | s4 | s5) == 0) {
        const float g0 = fp[0] - fm[0], g1 = fp[1] - fm[1], g2 = fp[2] - fm[2];
        const float gn = sqrtf(g0 * g0 + g1 * g1 + g2 * g2);
        if (gn > 0.0f) {
            const float sg = (g0 * dqx + g1 * dqy + g2 * dqz) > 0.0f ? -1.0f : 1.0f;
            const float iv = sg / gn;
            n0 = g0 * iv; n1 = g1 * iv; n2 = g2 * iv;
        }
    }
    if (depth_out) depth_out[pix] = zs;
    if (normal_out) { normal_out[3 * pix] = n0; normal_out[3 * pix + 1] = n1; normal_out[3 * pix + 2] = n2; }
    if (vertex_out) {
        vertex_out[3 * pix] = (float)(p.origin[0] + (double)qx * p.s);
        vertex_out[3 * pix + 1] = (float)(p.origin[1] + (double)qy * p.s);
        vertex_out[3 * pix + 2] = (float)(p.origin[2] + (double)qz * p.s);
    }
}

template <int kS, bool kNarrow>
__global__ void __launch_bounds__(32 * kRcWarps, 8) raycast_persistent_kernel(
    const FrameParams p, const unsigned int* __restrict__ near_, const unsigned int* __restrict__ far_,
    const int* __restrict__ order, const int* __restrict__ table, const typename Codec<kS>::E* __restrict__ T,
    const unsigned int* __restrict__ occ2, float* __restrict__ depth_out, float* __restrict__ normal_out,
    float* __restrict__ vertex_out, Counters* __restrict__ ctr) {
    pdl_prologue();
    // ray tiles per bucket of the ray order (ray_order_kernel)
    const unsigned nb0 = ctr->rc_bucket[0], nb1 = ctr->rc_bucket[1], nb2 = ctr->rc_bucket[2];
    // bracket queue of each warp: pix, z1, f1, z2, f2, dq (x, y, z)
    __shared__ float sq[kRcWarps][8][kQueue];
    float(*q)[kQueue] = sq[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const float nanf_ = __int_as_float(0x7fc00000);
    const float h = 0.5f * p.delta;
    const int tiles_x = (p.width + 7) / 8;
    const unsigned n_rays = (unsigned)(tiles_x * ((p.height + 3) / 4)) * 32u;
    const int rtiles_x = (p.width + kRangeTile - 1) / kRangeTile;
    // t / tiles_x as __umulhi(t, tdiv), exact while t * tiles_x < 2^32 (every
    // image up to 8192 x 8192 pixels); plain division beyond
    const unsigned tdiv = 0xffffffffu / (unsigned)tiles_x + 1u;
    const bool fast_div = tiles_x > 1 && (unsigned long long)(n_rays >> 5) * (unsigned)tiles_x < (1ull << 32);
    unsigned hits = 0;
    int queued = 0;     // warp-uniform

    // The march state of a lane's ray, kept small (registers decide how many
    // warps an SM holds): zl is the camera z of the last sample taken (the
    // bracket's near end when that sample was defined), zstep the step since,
    // iv the inverse ray direction used by empty-space skips; the re-scan runs
    // inline.
    bool busy = false, prev_def = false, rays_left = true;
    int pix = 0, it = 0;
    int rj = -1;        // re-scan substep of the lane's ray, -1 while it marches
    float ft = 0.f;     // the field at the sample that started the re-scan
    float dqx = 0.f, dqy = 0.f, dqz = 0.f, ivx = 0.f, ivy = 0.f, ivz = 0.f;
    float z = 0.f, zend = 0.f, fprev = 0.f, zl = 0.f, zstep = 0.f;

    for (;;) {
        // the next ray tile once no lane marches; a tile whose 32 rays all
        // miss their range maps (nothing to march) is followed by the next
        while (rays_left && !__any_sync(0xffffffffu, busy)) {
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(&ctr->rc_next, 32u);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base >= n_rays) {
                rays_left = false;
                break;
            }
            const unsigned w = (unsigned)lane;
            // the base / 32-th ray tile in bucket order
            unsigned t = base >> 5;
            {
                const unsigned n_t = n_rays >> 5;
                unsigned b = 0;
                if (t >= nb0) { t -= nb0; ++b; if (t >= nb1) { t -= nb1; ++b; if (t >= nb2) { t -= nb2; ++b; } } }
                t = (unsigned)__ldg(order + (size_t)b * n_t + t);
            }
            const unsigned ty = fast_div ? __umulhi(t, tdiv) : t / (unsigned)tiles_x;
            const unsigned tx = t - ty * (unsigned)tiles_x;
            const int u = (int)(tx * 8u + (w & 7u)), v = (int)(ty * 4u + (w >> 3));
            if (u >= p.width || v >= p.height) continue;
            pix = v * p.width + u;
            const int tile = (int)((unsigned)v / kRangeTile) * rtiles_x + (int)((unsigned)u / kRangeTile);
            const float zn = __uint_as_float(near_[tile]), zf = __uint_as_float(far_[tile]);
            z = fmaxf(zn, p.near_clip);
            zend = fminf(zf, p.far_clip);
            if (!(zn <= zf) || !(z <= zend)) {
                if (depth_out) depth_out[pix] = 0.0f;
                if (normal_out) { normal_out[3 * pix] = nanf_; normal_out[3 * pix + 1] = nanf_; normal_out[3 * pix + 2] = nanf_; }
                if (vertex_out) { vertex_out[3 * pix] = nanf_; vertex_out[3 * pix + 1] = nanf_; vertex_out[3 * pix + 2] = nanf_; }
                continue;
            }
            const float dcx = ((float)u - p.cx) / p.fx, dcy = ((float)v - p.cy) / p.fy;
            dqx = p.Rs[0] * dcx + p.Rs[1] * dcy + p.Rs[2];
            dqy = p.Rs[3] * dcx + p.Rs[4] * dcy + p.Rs[5];
            dqz = p.Rs[6] * dcx + p.Rs[7] * dcy + p.Rs[8];
            ivx = dqx != 0.0f ? 1.0f / dqx : 0.0f;
            ivy = dqy != 0.0f ? 1.0f / dqy : 0.0f;
            ivz = dqz != 0.0f ? 1.0f / dqz : 0.0f;
            prev_def = false;
            fprev = 0.0f;
            zl = z;
            zstep = h;
            it = 0;
            rj = -1;
            busy = true;
        }
        const bool marching = __any_sync(0xffffffffu, busy);
        if (!marching && queued == 0) break;
        if (queued >= 32 || !marching) {
            // the warp refines and shades the newest min(queued, 32) brackets
            const int n = min(queued, 32);
            queued -= n;
            if (lane < n) {
                const int e = queued + lane;
                refine_and_shade<kS, kNarrow>(p, table, T, __float_as_int(q[0][e]), q[1][e], q[2][e], q[3][e], q[4][e],
                                     q[5][e], q[6][e], q[7][e], depth_out, normal_out, vertex_out);
                ++hits;
            }
            __syncwarp();
            continue;
        }

        // one march sample per busy lane (a re-scanning lane samples its next substep)
        float f = 0.0f;
        int blk[3] = {0, 0, 0};
        const float zs_ = rj >= 0 ? zt_minus(z, zstep, rj) : z;
        const int st = busy ? trilinear<kS, false, kNarrow>(p, table, T, __fmaf_rn(zs_, dqx, p.q0[0]),
                                                            __fmaf_rn(zs_, dqy, p.q0[1]), __fmaf_rn(zs_, dqz, p.q0[2]),
                                                            &f, blk)
                            : 0;
        bool miss = false, push = false;
        float b1 = 0.f, c1 = 0.f, b2 = 0.f, c2 = 0.f;   // bracket (z1, f1, z2, f2)
        if (busy) {
            bool done = false;
            bool advance = false;   // the march moves on from z (counts an iteration)
            if (rj >= 0) {
                // Re-scan substep rj at zs_ (the state holds its own data: prev_def
                // whether the last substep was defined, fprev / zl its value and
                // position, zstep the re-scanned length, ft the field at z).
                rescan_step(st, f, zs_, prev_def, fprev, zl, &b1, &c1, &b2, &c2, &push, &miss, &done);
                if (!done && ++rj == kFine) {
                    // the re-scan ends at the sample that started it
                    rescan_step(0, ft, z, prev_def, fprev, zl, &b1, &c1, &b2, &c2, &push, &miss, &done);
                    if (!done) {
                        rj = -1;
                        prev_def = true;
                        fprev = ft;
                        zl = z;
                        zstep = h;
                        z += h;
                        advance = true;
                    }
                }
            } else if (st == 2) {
                const float inv[3] = {ivx, ivy, ivz};
                zl = fmaxf(empty_exit(p, occ2, blk, inv), z);
                z = zl + 1e-3f * h;
                zstep = z - zl;
                prev_def = false;
                advance = true;
            } else {
                const bool def = st == 0;
                if (def && !prev_def && f <= 0.0f && it > 0) {
                    // The field starts here already at or below zero: re-scan the
                    // last step in kFine substeps for a short positive run, one
                    // substep per iteration, so that the other lanes of the warp
                    // keep marching meanwhile.
                    rj = 0;
                    ft = f;
                    zstep = fminf(zstep, z - zl);
                    prev_def = false;
                } else if (def && prev_def && fprev > 0.0f && f <= 0.0f) {
                    b1 = zl; c1 = fprev; b2 = z; c2 = f;
                    push = true;
                    done = true;
                } else if (def && prev_def && fprev < 0.0f && f > 0.0f) {
                    miss = true;                      // back face first
                    done = true;
                } else {
                    prev_def = def;
                    fprev = f;
                    zl = z;
                    zstep = def ? h : 2.0f * h;
                    z += zstep;
                    advance = true;
                }
            }
            if (advance) {
                ++it;
                if (!(it < kMaxMarch && z <= zend)) miss = true;
            }
            if (done || miss) rj = -1;
        }
        const unsigned pm = __ballot_sync(0xffffffffu, push);
        if (push) {
            const int e = queued + __popc(pm & lt_mask);
            q[0][e] = __int_as_float(pix);
            q[1][e] = b1; q[2][e] = c1; q[3][e] = b2; q[4][e] = c2;
            q[5][e] = dqx; q[6][e] = dqy; q[7][e] = dqz;
            busy = false;
        }
        queued += __popc(pm);
        __syncwarp();
        if (miss) {
            if (depth_out) depth_out[pix] = 0.0f;
            if (normal_out) { normal_out[3 * pix] = nanf_; normal_out[3 * pix + 1] = nanf_; normal_out[3 * pix + 2] = nanf_; }
            if (vertex_out) { vertex_out[3 * pix] = nanf_; vertex_out[3 * pix + 1] = nanf_; vertex_out[3 * pix + 2] = nanf_; }
            busy = false;
        }
    }
    hits = warp_sum(hits);
    if (lane == 0 && hits) atomicAdd(&ctr->rays_hit, (unsigned long long)hits);
}


template <int kS, int kTW, int kTH>
void launch_march_t(tsdf_volume* v, const FrameParams& p, const unsigned int* near_, const unsigned int* far_,
                    float* depth_out, float* normal_out, float* vertex_out, cudaStream_t st) {
    const dim3 grid((unsigned)((p.width + kTW - 1) / kTW), (unsigned)((p.height + kTH - 1) / kTH));
    launch_pdl(raycast_kernel<kS, kTW, kTH>, grid, dim3(kTW * kTH), st, p, near_, far_, v->blk_slot,
               static_cast<const typename Codec<kS>::E*>(v->T), v->occ2, depth_out, normal_out, vertex_out,
               v->ctr);
}

// Raycast tile shapes the autotuner chooses from (pixels per CTA, width x height).
template <int kS, bool kNarrow>
void launch_persistent(tsdf_volume* v, const FrameParams& p, const unsigned int* near_, const unsigned int* far_,
                       int* order, float* depth_out, float* normal_out, float* vertex_out, cudaStream_t st) {
    launch_pdl(ray_order_kernel, dim3(v->num_sms), dim3(256), st, v->ctr, near_, far_, p, order);
    // exactly the CTAs that fit at once: a CTA launched later would find no rays left
    static int per_sm = 0;
    if (per_sm == 0 &&
        (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, raycast_persistent_kernel<kS, kNarrow>, 32 * kRcWarps,
                                                       0) != cudaSuccess ||
         per_sm < 1))
        per_sm = 1;
    launch_pdl(raycast_persistent_kernel<kS, kNarrow>, dim3(v->num_sms * per_sm), dim3(32 * kRcWarps), st, p, near_,
               far_, (const int*)order, v->blk_slot, static_cast<const typename Codec<kS>::E*>(v->T), v->occ2, depth_out,
               normal_out, vertex_out, v->ctr);
}

template <int kS>
void launch_march_s(tsdf_volume* v, const FrameParams& p, const unsigned int* near_, const unsigned int* far_,
                    int* order, float* depth_out, float* normal_out, float* vertex_out, cudaStream_t st) {
    if (v->lc.raycast_persistent) {
        if (v->cfg.block_capacity <= ((int64_t)1 << 23)) {
            launch_persistent<kS, true>(v, p, near_, far_, order, depth_out, normal_out, vertex_out, st);
        } else {
            launch_persistent<kS, false>(v, p, near_, far_, order, depth_out, normal_out, vertex_out, st);
        }
        return;
    }
    const int tw = v->lc.raycast_tile_w, th = v->lc.raycast_tile_h;
    if (tw == 8 && th == 8)
        launch_march_t<kS, 8, 8>(v, p, near_, far_, depth_out, normal_out, vertex_out, st);
    else if (tw == 32 && th == 4)
        launch_march_t<kS, 32, 4>(v, p, near_, far_, depth_out, normal_out, vertex_out, st);
    else if (tw == 8 && th == 16)
        launch_march_t<kS, 8, 16>(v, p, near_, far_, depth_out, normal_out, vertex_out, st);
    else if (tw == 16 && th == 16)
        launch_march_t<kS, 16, 16>(v, p, near_, far_, depth_out, normal_out, vertex_out, st);
    else
        launch_march_t<kS, 16, 8>(v, p, near_, far_, depth_out, normal_out, vertex_out, st);
}

void launch_march(tsdf_volume* v, const FrameParams& p, const unsigned int* near_, const unsigned int* far_,
                  int* order, float* depth_out, float* normal_out, float* vertex_out, cudaStream_t st) {
    switch (v->cfg.storage) {
        case TSDF_STORAGE_F16:
            launch_march_s<TSDF_STORAGE_F16>(v, p, near_, far_, order, depth_out, normal_out, vertex_out, st);
            break;
        case TSDF_STORAGE_SNORM16:
            launch_march_s<TSDF_STORAGE_SNORM16>(v, p, near_, far_, order, depth_out, normal_out, vertex_out, st);
            break;
        default:
            launch_march_s<TSDF_STORAGE_F32>(v, p, near_, far_, order, depth_out, normal_out, vertex_out, st);
            break;
    }
}

}  // namespace

cudaError_t launch_raycast(tsdf_volume* v, const FrameParams& p, float* depth_out, float* normal_out,
                           float* vertex_out, cudaStream_t st, bool rc_culled) {
    const long long npix = range_tiles(p.width, p.height);
    unsigned int* near_ = v->range;
    unsigned int* far_ = v->range + v->range_cap;
    if (!rc_culled) {   // else the integrate stage of the same pose cleared the maps and made the visible list
        launch_pdl(range_clear_kernel, dim3(v->num_sms * 4), dim3(256), st, near_, far_, npix, v->ctr);
        launch_pdl(rc_cull_kernel, dim3(v->num_sms * 8), dim3(256), st, v->ctr, v->blocks, p, v->visible_rc);
    }
    launch_pdl(raster_kernel, dim3(v->num_sms * 8), dim3(256), st, v->ctr, v->visible_rc, v->blocks, p, near_, far_);
    launch_march(v, p, near_, far_, v->ray_order, depth_out, normal_out, vertex_out, st);
    return cudaGetLastError();
}

namespace {

__global__ void __launch_bounds__(256) count_flags_kernel(const unsigned char* __restrict__ f, long long n,
                                                          unsigned long long* __restrict__ out) {
    unsigned c = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        c += f[i] != 0;
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, (unsigned long long)c);
}

template <int kS>
void launch_march_traced(tsdf_volume* v, const FrameParams& p, const unsigned int* near_, const unsigned int* far_,
                         cudaStream_t st) {
    const dim3 grid((p.width + 15) / 16, (p.height + 7) / 8);
    launch_pdl(raycast_kernel<kS, 16, 8, true>, grid, dim3(128), st, p, near_, far_, v->blk_slot,
               static_cast<const typename Codec<kS>::E*>(v->T), v->occ2, nullptr, nullptr, nullptr, v->ctr);
}

}  // namespace

cudaError_t launch_raycast_trace(tsdf_volume* v, const FrameParams& p, unsigned char* t_sector, long long n_t,
                                 unsigned char* table_sector, long long n_table, unsigned long long* counts,
                                 cudaStream_t st) {
    const TraceState ts{t_sector, table_sector, counts, storage_bytes(v->cfg.storage)};
    cudaError_t e = cudaMemcpyToSymbolAsync(g_trace, &ts, sizeof(ts), 0, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    const long long npix = range_tiles(p.width, p.height);
    unsigned int* near_ = v->range;
    unsigned int* far_ = v->range + v->range_cap;
    launch_pdl(range_clear_kernel, dim3(v->num_sms * 4), dim3(256), st, near_, far_, npix, v->ctr);
    launch_pdl(rc_cull_kernel, dim3(v->num_sms * 8), dim3(256), st, v->ctr, v->blocks, p, v->visible_rc);
    launch_pdl(raster_kernel, dim3(v->num_sms * 8), dim3(256), st, v->ctr, v->visible_rc, v->blocks, p, near_, far_);
    switch (v->cfg.storage) {
        case TSDF_STORAGE_F16: launch_march_traced<TSDF_STORAGE_F16>(v, p, near_, far_, st); break;
        case TSDF_STORAGE_SNORM16: launch_march_traced<TSDF_STORAGE_SNORM16>(v, p, near_, far_, st); break;
        default: launch_march_traced<TSDF_STORAGE_F32>(v, p, near_, far_, st); break;
    }
    count_flags_kernel<<<v->num_sms * 4, 256, 0, st>>>(t_sector, n_t, counts + 2);
    count_flags_kernel<<<v->num_sms * 4, 256, 0, st>>>(table_sector, n_table, counts + 3);
    return cudaGetLastError();
}

namespace {

// One read of pool slot `slot` behind the same index check as the raycast's
// voxel loads (tsdf_debug_check_slot: a check the host can make fail).
template <int kS>
__global__ void debug_slot_kernel(const typename Codec<kS>::E* __restrict__ T, long long slot, FrameParams p,
                                  float* __restrict__ sink) {
    if (in_bounds(p.err, slot >= 0 && slot < p.cap)) *sink = Codec<kS>::load(T + slot * kBlockVoxels, p.tsc);
}

}  // namespace

cudaError_t launch_debug_slot(tsdf_volume* v, long long slot, float* sink, cudaStream_t st) {
    const FrameParams p = make_frame_params(v, tsdf_intrinsics{1.0f, 1.0f, 0.0f, 0.0f, 1, 1}, kIdentityPose);
    switch (v->cfg.storage) {
        case TSDF_STORAGE_F16:
            debug_slot_kernel<TSDF_STORAGE_F16><<<1, 1, 0, st>>>(static_cast<const __half*>(v->T), slot, p, sink);
            break;
        case TSDF_STORAGE_SNORM16:
            debug_slot_kernel<TSDF_STORAGE_SNORM16><<<1, 1, 0, st>>>(static_cast<const short*>(v->T), slot, p, sink);
            break;
        default:
            debug_slot_kernel<TSDF_STORAGE_F32><<<1, 1, 0, st>>>(static_cast<const float*>(v->T), slot, p, sink);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_raycast_ranges(tsdf_volume* v, const FrameParams& p, unsigned int* near_, unsigned int* far_,
                                  int* order, float* depth_out, float* normal_out, float* vertex_out, cudaStream_t st) {
    const long long npix = range_tiles(p.width, p.height);
    launch_pdl(range_clear_kernel, dim3(v->num_sms * 4), dim3(256), st, near_, far_, npix, v->ctr);
    launch_pdl(rc_cull_kernel, dim3(v->num_sms * 8), dim3(256), st, v->ctr, v->blocks, p, v->visible_rc);
    launch_pdl(raster_kernel, dim3(v->num_sms * 8), dim3(256), st, v->ctr, v->visible_rc, v->blocks, p, near_, far_);
    launch_march(v, p, near_, far_, order, depth_out, normal_out, vertex_out, st);
    return cudaGetLastError();
}

}  // namespace tsdf
