// Block allocation (section "Updating Sparse Structure").
//
// The paper samples the measured surface in one kernel, reads the block
// coordinates back and allocates them on the CPU from a free list. Here the
// whole step stays on the device, with no host round trip:
//   1. alloc_mark:   one thread per pixel samples its ray at 2J+1 depths in
//                    [D - delta, D + delta]; every sample's block that the block
//                    table marks empty gets its bit set in a new-block bitmap
//                    (consecutive samples of a pixel in the same block are
//                    merged, and a bit already set is not set again, so few
//                    atomics remain).
//   2. alloc_count:  per 4096-word tile of the bitmap, the number of new blocks.
//   3. alloc_assign: each tile ranks its new blocks after all earlier tiles', so
//                    slots follow ascending block key whatever the order in
//                    which pixels were processed; writes slot and coordinates,
//                    drops blocks past the pool capacity, clears the bitmap.
//   4. alloc_finalize / init_blocks: commit the pool size and fill the new
//                    blocks with chi.
// The sample arithmetic is a fixed sequence of correctly rounded float32
// operations (explicit __fmaf_rn / __fdiv_rn; the library is built without FMA
// contraction), so the block set is reproducible bit for bit.
#include "tsdf_internal.cuh"

namespace tsdf {
namespace {

constexpr unsigned kNoKey = 0xffffffffu;

__global__ void __launch_bounds__(256) alloc_mark_kernel(const float* __restrict__ depth, AllocParams p,
                                                         const int* __restrict__ blk_slot,
                                                         unsigned int* __restrict__ newbits) {
    pdl_prologue();
    const long long n = (long long)p.width * p.height;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float d = 0.0f;
    bool valid = idx < n;
    if (valid) d = __ldg(depth + idx);
    valid = valid && depth_ok(d, p.depth_min, p.depth_max);
    float b0 = 0.0f, b1 = 0.0f, b2 = 0.0f;
    if (valid) {
        const int i = (int)(idx % p.width), j = (int)(idx / p.width);
        const float xn = __fdiv_rn(__fsub_rn((float)i, p.cx), p.fx);
        const float yn = __fdiv_rn(__fsub_rn((float)j, p.cy), p.fy);
        b0 = __fmaf_rn(p.M[0], xn, __fmaf_rn(p.M[1], yn, p.M[2]));
        b1 = __fmaf_rn(p.M[3], xn, __fmaf_rn(p.M[4], yn, p.M[5]));
        b2 = __fmaf_rn(p.M[6], xn, __fmaf_rn(p.M[7], yn, p.M[8]));
    }
    unsigned last = kNoKey;
    for (int k = 0; k <= 2 * p.J; ++k) {
        unsigned key = kNoKey;
        if (valid) {
            const float zk = __fmaf_rn((float)(k - p.J), p.dz, d);
            const float q0 = __fmaf_rn(zk, b0, p.a[0]);
            const float q1 = __fmaf_rn(zk, b1, p.a[1]);
            const float q2 = __fmaf_rn(zk, b2, p.a[2]);
            if (q0 >= 0.0f && q0 < p.G && q1 >= 0.0f && q1 < p.G && q2 >= 0.0f && q2 < p.G) {
                const unsigned bx = (unsigned)floorf(q0) >> 3;
                const unsigned by = (unsigned)floorf(q1) >> 3;
                const unsigned bz = (unsigned)floorf(q2) >> 3;
                key = bx + (unsigned)p.nb * (by + (unsigned)p.nb * bz);
            }
        }
        const bool fresh = key != kNoKey && key != last;
        if (key != kNoKey) last = key;
        if (fresh && in_bounds(p.err, (unsigned long long)key < (unsigned long long)p.nb * p.nb * p.nb) &&
            __ldg(blk_slot + key) < 0) {
            const unsigned bit = 1u << (key & 31u);
            unsigned int* w = newbits + (key >> 5);
            if (!(*(volatile unsigned int*)w & bit)) atomicOr(w, bit);
        }
    }
}

__device__ __forceinline__ unsigned block_sum(unsigned x, unsigned* smem) {
    x = warp_sum(x);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) smem[warp] = x;
    __syncthreads();
    unsigned t = 0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? smem[threadIdx.x] : 0u;
        t = warp_sum(t);
        if (threadIdx.x == 0) smem[0] = t;
    }
    __syncthreads();
    t = smem[0];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(kTileThreads) alloc_count_kernel(const uint4* __restrict__ words,
                                                                   unsigned int* __restrict__ tile_sums) {
    pdl_prologue();
    __shared__ unsigned smem[32];
    const uint4* base = words + (size_t)blockIdx.x * (kTileWords / 4);
    unsigned c = 0;
#pragma unroll
    for (int k = 0; k < kTileWords / 4 / kTileThreads; ++k) {
        const uint4 w = base[k * kTileThreads + threadIdx.x];
        c += __popc(w.x) + __popc(w.y) + __popc(w.z) + __popc(w.w);
    }
    c = block_sum(c, smem);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = c;
}

__global__ void __launch_bounds__(kTileThreads) alloc_assign_kernel(unsigned int* __restrict__ words,
                                                                    const unsigned int* __restrict__ tile_sums,
                                                                    Counters* ctr, int* __restrict__ blk_slot,
                                                                    int4* __restrict__ blocks, long long cap,
                                                                    int frame, int nb, unsigned int* __restrict__ occ2,
                                                                    int n2) {
    pdl_prologue();
    __shared__ unsigned smem[32];
    __shared__ unsigned wsum[kTileThreads / 32];
    const int tile = blockIdx.x;
    if (tile_sums[tile] == 0) return;     // uniform over the CTA
    unsigned pre = 0;
    for (int t = threadIdx.x; t < tile; t += blockDim.x) pre += tile_sums[t];
    pre = block_sum(pre, smem);
    const long long n_base = ctr->n_blocks;

    constexpr int kPer = kTileWords / kTileThreads;   // 16 contiguous words per thread
    unsigned int* w = words + (size_t)tile * kTileWords + (size_t)threadIdx.x * kPer;
    unsigned v[kPer];
    unsigned c = 0;
#pragma unroll
    for (int k = 0; k < kPer / 4; ++k) {
        const uint4 q = reinterpret_cast<const uint4*>(w)[k];
        v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
        c += __popc(q.x) + __popc(q.y) + __popc(q.z) + __popc(q.w);
    }
    // exclusive scan of c over the CTA in thread order (= word order)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    unsigned wpre = 0;
    for (int k = 0; k < warp; ++k) wpre += wsum[k];
    long long rank = n_base + (long long)pre + (long long)(wpre + incl - c);

    const unsigned key0 = ((unsigned)tile * kTileWords + (unsigned)threadIdx.x * kPer) * 32u;
    bool over = false;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        unsigned bits = v[k];
        if (!bits) continue;
        w[k] = 0u;
        while (bits) {
            const unsigned b = (unsigned)__ffs(bits) - 1u;
            bits &= bits - 1u;
            const unsigned key = key0 + 32u * (unsigned)k + b;
            if (rank < cap) {
                if (in_bounds(&ctr->error, (unsigned long long)key < (unsigned long long)nb * nb * nb)) {
                    const int bx = (int)(key % (unsigned)nb);
                    const int by = (int)((key / (unsigned)nb) % (unsigned)nb);
                    const int bz = (int)(key / ((unsigned)nb * (unsigned)nb));
                    blk_slot[key] = (int)rank;
                    blocks[rank] = make_int4(bx, by, bz, frame);
                    // coarse occupancy used by the raycast to skip empty space
                    const unsigned c2 = (unsigned)(bx / kOcc2) + (unsigned)n2 * ((unsigned)(by / kOcc2) + (unsigned)n2 * (unsigned)(bz / kOcc2));
                    atomicOr(occ2 + (c2 >> 5), 1u << (c2 & 31u));
                }
            } else {
                over = true;
            }
            ++rank;
        }
    }
    if (over) atomicOr(&ctr->error, kErrCapacity);
}

__global__ void alloc_finalize_kernel(const unsigned int* __restrict__ tile_sums, int n_tiles, Counters* ctr,
                                      long long cap) {
    pdl_prologue();
    unsigned long long s = 0;
    for (int t = threadIdx.x; t < n_tiles; t += 32) s += tile_sums[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) {
        const long long n_old = ctr->n_blocks;
        long long n_new = n_old + (long long)s;
        if (n_new > cap) {
            n_new = cap;
            ctr->error |= kErrCapacity;
        }
        ctr->n_blocks_prev = n_old;
        ctr->n_blocks = n_new;
    }
}

// Fresh blocks hold chi everywhere (Fig. 4 caption: memory is allocated for a
// block when anything but chi is to be stored in it). T is filled with the
// storage format's chi pattern, one 32-bit word (1 or 2 voxels) at a time.
__global__ void __launch_bounds__(256) init_blocks_kernel(const Counters* __restrict__ ctr,
                                                          unsigned int* __restrict__ T, float2* __restrict__ P,
                                                          int t_words, unsigned int chi_word) {
    pdl_prologue();
    const long long lo = ctr->n_blocks_prev, hi = ctr->n_blocks;
    for (long long b = lo + blockIdx.x; b < hi; b += gridDim.x) {
        for (int w = threadIdx.x; w < t_words; w += blockDim.x) T[b * t_words + w] = chi_word;
        P[b * 256 + threadIdx.x] = make_float2(0.0f, 0.0f);
    }
}

}  // namespace

cudaError_t launch_allocate(tsdf_volume* v, const float* depth, const AllocParams& p, int frame,
                            cudaStream_t st) {
    const long long n = (long long)p.width * p.height;
    if (n > 0) {
        const unsigned grid = (unsigned)((n + 255) / 256);
        launch_pdl(alloc_mark_kernel, dim3(grid), dim3(256), st, depth, p, v->blk_slot, v->newbits);
    }
    launch_pdl(alloc_count_kernel, dim3(v->n_tiles), dim3(kTileThreads), st,
               reinterpret_cast<const uint4*>(v->newbits), v->tile_sums);
    launch_pdl(alloc_assign_kernel, dim3(v->n_tiles), dim3(kTileThreads), st, v->newbits, v->tile_sums, v->ctr,
               v->blk_slot, v->blocks, v->cfg.block_capacity, frame, v->nb, v->occ2, v->n2);
    launch_pdl(alloc_finalize_kernel, dim3(1), dim3(32), st, v->tile_sums, (int)v->n_tiles, v->ctr,
               v->cfg.block_capacity);
    const int bytes = storage_bytes(v->cfg.storage);
    const unsigned chi_word = v->cfg.storage == TSDF_STORAGE_F32   ? 0x7fc00000u
                              : v->cfg.storage == TSDF_STORAGE_F16 ? 0x7e007e00u
                                                                   : 0x80008000u;
    launch_pdl(init_blocks_kernel, dim3(v->num_sms * 4), dim3(256), st, v->ctr,
               reinterpret_cast<unsigned int*>(v->T), reinterpret_cast<float2*>(v->P), kBlockVoxels * bytes / 4,
               chi_word);
    return cudaGetLastError();
}

}  // namespace tsdf
