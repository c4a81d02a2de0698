// Block eviction, import and volume shift (section "Discussion": for scenes
// larger than device memory the TSDF data of occupied blocks is evicted to
// host storage, and a shift of the volume evicts the blocks that leave it and
// rebuilds the offset array).
//
// These are rare, synchronous operations between frames, so the plan is made
// on the host from a copy of the block list (a few MB for a million blocks):
//   evict:  the blocks outside a box of block coordinates are gathered into a
//           staging buffer (decoded to float) and copied out; the pool is
//           compacted by moving the last kept blocks into the freed slots (no
//           slot is both read and written, so one kernel moves them all); the
//           block table entries of evicted and moved blocks are updated and
//           the occupancy map rebuilt.
//   shift:  the grid origin moves by whole blocks, so every voxel keeps its
//           world position; blocks whose new coordinates leave the grid are
//           evicted as above, the others are re-keyed and the block table is
//           rebuilt from the block list.
//   import: blocks with given data are appended to the pool (encoded to the
//           storage format on the device) and entered in the table.
#include <algorithm>
#include <cstring>
#include <vector>

#include "tsdf_internal.cuh"

namespace tsdf {
namespace {

// T (decoded to float) and P of the listed pool slots, block after block.
template <int kS>
__global__ void __launch_bounds__(256) gather_blocks_kernel(const int* __restrict__ slots, long long n,
                                                            const typename Codec<kS>::E* __restrict__ T,
                                                            const float* __restrict__ P, float* __restrict__ outT,
                                                            float* __restrict__ outP, float2 sc) {
    const long long quads = n * (kBlockVoxels / 4);
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < quads;
         q += (long long)gridDim.x * blockDim.x) {
        const long long b = q / (kBlockVoxels / 4);
        const int off = (int)(q % (kBlockVoxels / 4)) * 4;
        const size_t src = (size_t)slots[b] * kBlockVoxels + off;
        float t[4];
        Codec<kS>::load4(T + src, t, sc);
        *reinterpret_cast<float4*>(outT + b * kBlockVoxels + off) = make_float4(t[0], t[1], t[2], t[3]);
        *reinterpret_cast<float4*>(outP + b * kBlockVoxels + off) = *reinterpret_cast<const float4*>(P + src);
    }
}

// Pool block pairs[i].x -> pairs[i].y (the destinations are free slots that no
// pair reads).
template <int kS>
__global__ void __launch_bounds__(256) move_blocks_kernel(const int2* __restrict__ pairs, long long n,
                                                          typename Codec<kS>::E* __restrict__ T,
                                                          float* __restrict__ P) {
    using E = typename Codec<kS>::E;
    constexpr int kTWords = kBlockVoxels * (int)sizeof(E) / 16;   // 16-byte words of T per block
    constexpr int kPWords = kBlockVoxels * 4 / 16;
    const long long per = kTWords + kPWords;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n * per;
         q += (long long)gridDim.x * blockDim.x) {
        const int2 pr = pairs[q / per];
        const int w = (int)(q % per);
        if (w < kTWords) {
            const uint4* s = reinterpret_cast<const uint4*>(T + (size_t)pr.x * kBlockVoxels);
            uint4* d = reinterpret_cast<uint4*>(T + (size_t)pr.y * kBlockVoxels);
            d[w] = s[w];
        } else {
            const uint4* s = reinterpret_cast<const uint4*>(P + (size_t)pr.x * kBlockVoxels);
            uint4* d = reinterpret_cast<uint4*>(P + (size_t)pr.y * kBlockVoxels);
            d[w - kTWords] = s[w - kTWords];
        }
    }
}

// Blocks slot0 .. slot0 + n - 1 from float T (NaN = chi) and P, encoded to the
// storage format.
template <int kS>
__global__ void __launch_bounds__(256) put_blocks_kernel(const float* __restrict__ inT, const float* __restrict__ inP,
                                                         long long n, long long slot0,
                                                         typename Codec<kS>::E* __restrict__ T,
                                                         float* __restrict__ P, float2 sc) {
    const long long quads = n * (kBlockVoxels / 4);
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < quads;
         q += (long long)gridDim.x * blockDim.x) {
        const long long i = 4 * q;
        const float4 t4 = *reinterpret_cast<const float4*>(inT + i);
        const float t[4] = {t4.x, t4.y, t4.z, t4.w};
        const size_t dst = (size_t)slot0 * kBlockVoxels + (size_t)i;
        Codec<kS>::store4(T + dst, t, sc);
        *reinterpret_cast<float4*>(P + dst) = *reinterpret_cast<const float4*>(inP + i);
    }
}

// table[kv[i].x] = kv[i].y
__global__ void __launch_bounds__(256) table_scatter_kernel(const int2* __restrict__ kv, long long n,
                                                            int* __restrict__ table) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        table[kv[i].x] = kv[i].y;
}

// out[i] = table[keys[i]]
__global__ void __launch_bounds__(256) table_gather_kernel(const int* __restrict__ keys, long long n,
                                                           const int* __restrict__ table, int* __restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = table[keys[i]];
}

// Occupancy bits (cells of 4^3 blocks) of the first n pool blocks.
__global__ void __launch_bounds__(256) occ_mark_kernel(const int4* __restrict__ blocks, long long n,
                                                       unsigned int* __restrict__ occ2, int n2) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int4 b = blocks[i];
        const unsigned c2 = (unsigned)(b.x / kOcc2) + (unsigned)n2 * ((unsigned)(b.y / kOcc2) + (unsigned)n2 * (unsigned)(b.z / kOcc2));
        atomicOr(occ2 + (c2 >> 5), 1u << (c2 & 31u));
    }
}

unsigned grid_for(long long work) {
    const long long g = (work + 255) / 256;
    return (unsigned)std::max<long long>(1, std::min<long long>(g, 65535));
}

// A device buffer freed on scope exit.
struct DevBuf {
    void* p = nullptr;
    cudaError_t alloc(size_t bytes) { return bytes ? cudaMalloc(&p, bytes) : cudaSuccess; }
    ~DevBuf() { if (p) cudaFree(p); }
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

uint32_t key_of(const tsdf_volume* v, int bx, int by, int bz) {
    return (uint32_t)bx + (uint32_t)v->nb * ((uint32_t)by + (uint32_t)v->nb * (uint32_t)bz);
}

cudaError_t read_pool(tsdf_volume* v, cudaStream_t st, std::vector<int4>* blocks) {
    cudaError_t e = cudaStreamSynchronize(st);
    long long n = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&n, &v->ctr->n_blocks, sizeof(n), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    blocks->resize((size_t)n);
    if (n > 0) e = cudaMemcpy(blocks->data(), v->blocks, (size_t)n * sizeof(int4), cudaMemcpyDeviceToHost);
    return e;
}

cudaError_t launch_gather(tsdf_volume* v, const int* slots, long long n, float* outT, float* outP, cudaStream_t st) {
    const unsigned g = grid_for(n * (kBlockVoxels / 4));
    const float2 sc = make_float2((float)((double)v->cfg.truncation / 32767.0),
                                  (float)(32767.0 / (double)v->cfg.truncation));
    switch (v->cfg.storage) {
        case TSDF_STORAGE_F16:
            gather_blocks_kernel<TSDF_STORAGE_F16><<<g, 256, 0, st>>>(slots, n, static_cast<const __half*>(v->T),
                                                                      v->P, outT, outP, sc);
            break;
        case TSDF_STORAGE_SNORM16:
            gather_blocks_kernel<TSDF_STORAGE_SNORM16><<<g, 256, 0, st>>>(slots, n, static_cast<const short*>(v->T),
                                                                          v->P, outT, outP, sc);
            break;
        default:
            gather_blocks_kernel<TSDF_STORAGE_F32><<<g, 256, 0, st>>>(slots, n, static_cast<const float*>(v->T),
                                                                      v->P, outT, outP, sc);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_move(tsdf_volume* v, const int2* pairs, long long n, cudaStream_t st) {
    const long long per = kBlockVoxels * (storage_bytes(v->cfg.storage) + 4) / 16;
    const unsigned g = grid_for(n * per);
    switch (v->cfg.storage) {
        case TSDF_STORAGE_F16:
            move_blocks_kernel<TSDF_STORAGE_F16><<<g, 256, 0, st>>>(pairs, n, static_cast<__half*>(v->T), v->P);
            break;
        case TSDF_STORAGE_SNORM16:
            move_blocks_kernel<TSDF_STORAGE_SNORM16><<<g, 256, 0, st>>>(pairs, n, static_cast<short*>(v->T), v->P);
            break;
        default:
            move_blocks_kernel<TSDF_STORAGE_F32><<<g, 256, 0, st>>>(pairs, n, static_cast<float*>(v->T), v->P);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_put(tsdf_volume* v, const float* inT, const float* inP, long long n, long long slot0,
                       cudaStream_t st) {
    const unsigned g = grid_for(n * (kBlockVoxels / 4));
    const float2 sc = make_float2((float)((double)v->cfg.truncation / 32767.0),
                                  (float)(32767.0 / (double)v->cfg.truncation));
    switch (v->cfg.storage) {
        case TSDF_STORAGE_F16:
            put_blocks_kernel<TSDF_STORAGE_F16><<<g, 256, 0, st>>>(inT, inP, n, slot0, static_cast<__half*>(v->T),
                                                                   v->P, sc);
            break;
        case TSDF_STORAGE_SNORM16:
            put_blocks_kernel<TSDF_STORAGE_SNORM16><<<g, 256, 0, st>>>(inT, inP, n, slot0, static_cast<short*>(v->T),
                                                                       v->P, sc);
            break;
        default:
            put_blocks_kernel<TSDF_STORAGE_F32><<<g, 256, 0, st>>>(inT, inP, n, slot0, static_cast<float*>(v->T),
                                                                   v->P, sc);
            break;
    }
    return cudaGetLastError();
}

// The pool size (committed and "before the last allocation") and the
// occupancy map after the block list changed outside an allocation.
cudaError_t commit_pool(tsdf_volume* v, const std::vector<int4>& blocks, cudaStream_t st) {
    const long long n = (long long)blocks.size();
    cudaError_t e = cudaSuccess;
    if (n > 0) e = cudaMemcpyAsync(v->blocks, blocks.data(), (size_t)n * sizeof(int4), cudaMemcpyHostToDevice, st);
    const long long sizes[2] = {n, n};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&v->ctr->n_blocks, sizes, sizeof(sizes), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->occ2, 0, v->occ2_words * sizeof(uint32_t), st);
    if (e == cudaSuccess && n > 0) {
        occ_mark_kernel<<<grid_for(n), 256, 0, st>>>(v->blocks, n, v->occ2, v->n2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

// Evict every block for which out(b) holds, then re-key the kept ones by
// subtracting shift (block units; the whole table is rebuilt when it is
// non-zero). Outputs as tsdf_evict.
template <typename Out>
tsdf_status evict_where(tsdf_volume* v, Out out, const int32_t shift[3], int64_t max_blocks, int32_t* coords_frame,
                        float* T, float* P, int64_t* n_evicted, cudaStream_t st) {
    std::vector<int4> blocks;
    cudaError_t e = read_pool(v, st, &blocks);
    if (e != cudaSuccess) return TSDF_ERR_CUDA;
    const long long n = (long long)blocks.size();
    std::vector<int> ev;
    for (long long b = 0; b < n; ++b)
        if (out(blocks[b])) ev.push_back((int)b);
    const long long ne = (long long)ev.size();
    *n_evicted = ne;
    if (ne > max_blocks) return TSDF_ERR_CAPACITY;
    const bool rekey = shift[0] != 0 || shift[1] != 0 || shift[2] != 0;
    if (ne == 0 && !rekey) return TSDF_OK;

    // 1. the evicted blocks' data out
    if (ne > 0) {
        DevBuf d_slots, d_T, d_P;
        e = d_slots.alloc((size_t)ne * sizeof(int));
        if (e == cudaSuccess) e = d_T.alloc((size_t)ne * kBlockVoxels * sizeof(float));
        if (e == cudaSuccess) e = d_P.alloc((size_t)ne * kBlockVoxels * sizeof(float));
        if (e == cudaSuccess) e = cudaMemcpy(d_slots.p, ev.data(), (size_t)ne * sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = launch_gather(v, d_slots.as<int>(), ne, d_T.as<float>(), d_P.as<float>(), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && T)
            e = cudaMemcpy(T, d_T.p, (size_t)ne * kBlockVoxels * sizeof(float), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && P)
            e = cudaMemcpy(P, d_P.p, (size_t)ne * kBlockVoxels * sizeof(float), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return TSDF_ERR_CUDA;
        if (coords_frame)
            for (long long i = 0; i < ne; ++i) {
                const int4 b = blocks[ev[i]];
                coords_frame[4 * i] = b.x; coords_frame[4 * i + 1] = b.y;
                coords_frame[4 * i + 2] = b.z; coords_frame[4 * i + 3] = b.w;
            }
    }

    // 2. compaction: the i-th freed slot below n_keep takes the i-th kept block
    //    at or above n_keep
    const long long n_keep = n - ne;
    std::vector<int2> pairs;
    std::vector<int2> table_kv;           // table updates (rekey = false)
    std::vector<char> gone((size_t)n, 0);
    for (int b : ev) gone[b] = 1;
    {
        // ev is ascending, so its first entries are the freed slots below n_keep,
        // exactly as many as there are kept blocks at or above n_keep
        size_t h = 0;
        for (long long b = n_keep; b < n; ++b)
            if (!gone[b]) pairs.push_back(make_int2((int)b, ev[h++]));
    }
    std::vector<int4> kept(blocks.begin(), blocks.begin() + n_keep);
    for (const int2& pr : pairs) kept[pr.y] = blocks[pr.x];
    if (!rekey) {
        for (int b : ev) {
            const int4& c = blocks[b];
            table_kv.push_back(make_int2((int)key_of(v, c.x, c.y, c.z), -1));
        }
        for (const int2& pr : pairs) {
            const int4& c = blocks[pr.x];
            table_kv.push_back(make_int2((int)key_of(v, c.x, c.y, c.z), pr.y));
        }
    } else {
        for (long long b = 0; b < n_keep; ++b) {
            int4& c = kept[b];
            c.x -= shift[0]; c.y -= shift[1]; c.z -= shift[2];
            table_kv.push_back(make_int2((int)key_of(v, c.x, c.y, c.z), (int)b));
        }
    }
    if (!pairs.empty()) {
        DevBuf d_pairs;
        e = d_pairs.alloc(pairs.size() * sizeof(int2));
        if (e == cudaSuccess)
            e = cudaMemcpy(d_pairs.p, pairs.data(), pairs.size() * sizeof(int2), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = launch_move(v, d_pairs.as<int2>(), (long long)pairs.size(), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return TSDF_ERR_CUDA;
    }
    // 3. block table
    if (rekey) e = cudaMemsetAsync(v->blk_slot, 0xff, v->n_table * sizeof(int32_t), st);
    if (e == cudaSuccess && !table_kv.empty()) {
        DevBuf d_kv;
        e = d_kv.alloc(table_kv.size() * sizeof(int2));
        if (e == cudaSuccess)
            e = cudaMemcpy(d_kv.p, table_kv.data(), table_kv.size() * sizeof(int2), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            table_scatter_kernel<<<grid_for((long long)table_kv.size()), 256, 0, st>>>(
                d_kv.as<int2>(), (long long)table_kv.size(), v->blk_slot);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    // 4. block list, pool size, occupancy
    if (e == cudaSuccess) e = commit_pool(v, kept, st);
    return e == cudaSuccess ? TSDF_OK : TSDF_ERR_CUDA;
}

tsdf_status fail(tsdf_volume* v, tsdf_status s) {
    if (s == TSDF_ERR_CUDA && v->host_error == TSDF_OK) v->host_error = TSDF_ERR_CUDA;
    return s;
}

}  // namespace
}  // namespace tsdf

extern "C" {

tsdf_status tsdf_get_config(const tsdf_volume* v, tsdf_config* out) {
    if (!v || !out) return TSDF_ERR_INVALID_ARG;
    *out = v->cfg;
    return TSDF_OK;
}

tsdf_status tsdf_evict(tsdf_volume* v, const int32_t lo[3], const int32_t hi[3], int64_t max_blocks,
                       int32_t* coords_frame, float* T, float* P, int64_t* n_evicted, void* stream) {
    if (!v || !lo || !hi || !n_evicted || max_blocks < 0) return TSDF_ERR_INVALID_ARG;
    for (int r = 0; r < 3; ++r)
        if (lo[r] > hi[r]) return TSDF_ERR_INVALID_ARG;
    const int32_t a[3] = {lo[0], lo[1], lo[2]}, b[3] = {hi[0], hi[1], hi[2]};
    const int32_t none[3] = {0, 0, 0};
    cudaStream_t st = (cudaStream_t)stream;
    v->last_stream = st;
    auto out = [&](const int4& c) {
        return c.x < a[0] || c.x >= b[0] || c.y < a[1] || c.y >= b[1] || c.z < a[2] || c.z >= b[2];
    };
    return tsdf::fail(v, tsdf::evict_where(v, out, none, max_blocks, coords_frame, T, P, n_evicted, st));
}

tsdf_status tsdf_shift(tsdf_volume* v, const int32_t d[3], int64_t max_blocks, int32_t* coords_frame, float* T,
                       float* P, int64_t* n_evicted, void* stream) {
    if (!v || !d || !n_evicted || max_blocks < 0) return TSDF_ERR_INVALID_ARG;
    const int32_t nb = v->nb;
    for (int r = 0; r < 3; ++r)
        if (d[r] <= -(1 << 24) || d[r] >= (1 << 24)) return TSDF_ERR_INVALID_ARG;
    const int32_t dd[3] = {d[0], d[1], d[2]};
    cudaStream_t st = (cudaStream_t)stream;
    v->last_stream = st;
    // a block stays when its new coordinates b - d lie in [0, nb)
    auto out = [&](const int4& c) {
        return c.x - dd[0] < 0 || c.x - dd[0] >= nb || c.y - dd[1] < 0 || c.y - dd[1] >= nb || c.z - dd[2] < 0 ||
               c.z - dd[2] >= nb;
    };
    const tsdf_status s = tsdf::evict_where(v, out, dd, max_blocks, coords_frame, T, P, n_evicted, st);
    if (s != TSDF_OK) return tsdf::fail(v, s);
    // the grid moves by whole blocks: voxel i' = i - 8 d sits where voxel i sat
    const double s_m = (double)v->cfg.voxel_size;
    for (int r = 0; r < 3; ++r) v->cfg.origin[r] += (double)(tsdf::kSide * (int64_t)dd[r]) * s_m;
    return TSDF_OK;
}

tsdf_status tsdf_import(tsdf_volume* v, int64_t n, const int32_t* coords_frame, const float* T, const float* P,
                        void* stream) {
    if (!v || n < 0 || (n > 0 && (!coords_frame || !T || !P))) return TSDF_ERR_INVALID_ARG;
    if (n == 0) return TSDF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    v->last_stream = st;
    std::vector<int4> blocks;
    if (tsdf::read_pool(v, st, &blocks) != cudaSuccess) return tsdf::fail(v, TSDF_ERR_CUDA);
    const long long n0 = (long long)blocks.size();
    if (n0 + n > v->cfg.block_capacity) return TSDF_ERR_CAPACITY;
    // coordinates inside the grid, no duplicates among themselves
    std::vector<int> keys((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        const int32_t* c = coords_frame + 4 * i;
        for (int r = 0; r < 3; ++r)
            if (c[r] < 0 || c[r] >= v->nb) return TSDF_ERR_INVALID_ARG;
        keys[i] = (int)tsdf::key_of(v, c[0], c[1], c[2]);
    }
    {
        std::vector<int> sorted(keys);
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return TSDF_ERR_INVALID_ARG;
    }
    // none of them already allocated
    tsdf::DevBuf d_keys, d_slots;
    cudaError_t e = d_keys.alloc((size_t)n * sizeof(int));
    if (e == cudaSuccess) e = d_slots.alloc((size_t)n * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(d_keys.p, keys.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        tsdf::table_gather_kernel<<<tsdf::grid_for(n), 256, 0, st>>>(d_keys.as<int>(), n, v->blk_slot,
                                                                     d_slots.as<int>());
        e = cudaGetLastError();
    }
    std::vector<int> slots((size_t)n);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(slots.data(), d_slots.p, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return tsdf::fail(v, TSDF_ERR_CUDA);
    for (int s : slots)
        if (s >= 0) return TSDF_ERR_INVALID_ARG;
    // data into slots n0 .. n0 + n - 1
    tsdf::DevBuf d_T, d_P, d_kv;
    e = d_T.alloc((size_t)n * tsdf::kBlockVoxels * sizeof(float));
    if (e == cudaSuccess) e = d_P.alloc((size_t)n * tsdf::kBlockVoxels * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(d_T.p, T, (size_t)n * tsdf::kBlockVoxels * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_P.p, P, (size_t)n * tsdf::kBlockVoxels * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = tsdf::launch_put(v, d_T.as<float>(), d_P.as<float>(), n, n0, st);
    std::vector<int2> kv((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        const int32_t* c = coords_frame + 4 * i;
        // imported blocks count as allocated at the current frame
        blocks.push_back(make_int4(c[0], c[1], c[2], (int)v->frame));
        kv[i] = make_int2(keys[i], (int)(n0 + i));
    }
    if (e == cudaSuccess) e = d_kv.alloc((size_t)n * sizeof(int2));
    if (e == cudaSuccess) e = cudaMemcpy(d_kv.p, kv.data(), (size_t)n * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        tsdf::table_scatter_kernel<<<tsdf::grid_for(n), 256, 0, st>>>(d_kv.as<int2>(), n, v->blk_slot);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = tsdf::commit_pool(v, blocks, st);
    return e == cudaSuccess ? TSDF_OK : tsdf::fail(v, TSDF_ERR_CUDA);
}

}  // extern "C"
