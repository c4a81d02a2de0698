// Marching-cubes surface of the sparse TSDF (section "Scene Rendering": the
// paper's alternative renderer polygonises the non-empty blocks by marching
// cubes).
//
//   mesh_count_kernel: one CTA per allocated block (grid-stride), one thread per
//                      cell = the cube of lattice voxels i + {0,1}^3 whose lower
//                      corner is the thread's voxel; a cell with all 8 corners
//                      defined (allocated, not chi) gets its corner pattern
//                      (inside = T < 0, Eq. 1) and triangle count; the CTA's sum
//                      is the block's count.
//   mesh_scan_kernel:  one CTA: exclusive prefix sum of the block counts, so
//                      the output is ordered by block, then by cell.
//   mesh_emit_kernel:  the same traversal writes each cell's triangles at its
//                      block's offset plus the cell's rank within the CTA; a
//                      vertex lies on its edge at the linear zero of T.
//
// The case table is generated on the host from the published construction
// (no stored table): per cell face the crossed edges pair into segments, a face
// with four crossings pairing each inside corner's two edges (so the cells on
// both sides of a face agree and the surface is closed); each segment is
// directed so that the cut-off inside corner lies on the side that makes the
// normal point from inside to outside; the segments chain into loops, each
// loop starts at its smallest edge number and is split into the fan
// (v0, v_k, v_k+1). Corners c = x + 2y + 4z; edges 0-3 run along x from corners
// 0, 2, 4, 6, edges 4-7 along y from corners 0, 1, 4, 5, edges 8-11 along z
// from corners 0, 1, 2, 3.
#include <cstring>
#include <mutex>

#include "tsdf_internal.cuh"
#include "tsdf_storage.cuh"

namespace tsdf {
namespace {

constexpr int kMaxTri = 8;        // triangles per cell the table has room for (the construction gives at most 5)

struct McTable {
    unsigned char ntri[256];
    signed char tri[256][3 * kMaxTri];
};

__constant__ McTable c_mc;

int edge_corner(int e, int end) {
    const int axis = e >> 2, k = e & 3;
    static const int starts[3][4] = {{0, 2, 4, 6}, {0, 1, 4, 5}, {0, 1, 2, 3}};
    const int a = starts[axis][k];
    return end ? a + (1 << axis) : a;
}

int edge_between(int a, int b) {
    if (a > b) {
        const int t = a;
        a = b;
        b = t;
    }
    for (int e = 0; e < 12; ++e)
        if (edge_corner(e, 0) == a && edge_corner(e, 1) == b) return e;
    return -1;
}

void corner_xyz(int c, double p[3]) {
    p[0] = c & 1;
    p[1] = (c >> 1) & 1;
    p[2] = (c >> 2) & 1;
}

void build_table(McTable* t) {
    std::memset(t, 0, sizeof(*t));
    for (int cs = 0; cs < 256; ++cs) {
        int next[12];
        for (int& x : next) x = -1;
        for (int axis = 0; axis < 3; ++axis) {
            const int u = axis == 0 ? 1 : 0, v = axis == 2 ? 1 : 2;     // the face's two in-plane axes
            for (int side = 0; side < 2; ++side) {
                // corners in cyclic order (u, v) = (0,0), (1,0), (1,1), (0,1)
                int fc[4];
                const int uv[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
                for (int i = 0; i < 4; ++i) fc[i] = (side << axis) | (uv[i][0] << u) | (uv[i][1] << v);
                double nrm[3] = {0, 0, 0};
                nrm[axis] = side ? 1.0 : -1.0;
                int crossed[4], nc = 0;
                for (int i = 0; i < 4; ++i) {
                    const int a = fc[i], b = fc[(i + 1) & 3];
                    if (((cs >> a) & 1) != ((cs >> b) & 1)) crossed[nc++] = edge_between(a, b);
                }
                if (nc == 0) continue;
                int seg[2][3], ns = 0;      // (edge from, edge to, cut-off inside corner)
                if (nc == 2) {
                    int in = -1;
                    for (int i = 0; i < 4; ++i)
                        if ((cs >> fc[i]) & 1) in = fc[i];
                    seg[ns][0] = crossed[0];
                    seg[ns][1] = crossed[1];
                    seg[ns][2] = in;
                    ++ns;
                } else {
                    for (int i = 0; i < 4; ++i) {
                        if (!((cs >> fc[i]) & 1)) continue;
                        seg[ns][0] = edge_between(fc[(i + 3) & 3], fc[i]);
                        seg[ns][1] = edge_between(fc[i], fc[(i + 1) & 3]);
                        seg[ns][2] = fc[i];
                        ++ns;
                    }
                }
                for (int k = 0; k < ns; ++k) {
                    double A[3], B[3], I[3], p0[3], p1[3];
                    corner_xyz(edge_corner(seg[k][0], 0), p0);
                    corner_xyz(edge_corner(seg[k][0], 1), p1);
                    for (int d = 0; d < 3; ++d) A[d] = 0.5 * (p0[d] + p1[d]);
                    corner_xyz(edge_corner(seg[k][1], 0), p0);
                    corner_xyz(edge_corner(seg[k][1], 1), p1);
                    for (int d = 0; d < 3; ++d) B[d] = 0.5 * (p0[d] + p1[d]);
                    corner_xyz(seg[k][2], I);
                    const double ba[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
                    const double ia[3] = {I[0] - A[0], I[1] - A[1], I[2] - A[2]};
                    const double cr[3] = {ba[1] * ia[2] - ba[2] * ia[1], ba[2] * ia[0] - ba[0] * ia[2],
                                          ba[0] * ia[1] - ba[1] * ia[0]};
                    const double dn = cr[0] * nrm[0] + cr[1] * nrm[1] + cr[2] * nrm[2];
                    if (dn > 0.0)
                        next[seg[k][1]] = seg[k][0];
                    else
                        next[seg[k][0]] = seg[k][1];
                }
            }
        }
        int nt = 0;
        bool seen[12] = {false};
        for (int start = 0; start < 12; ++start) {
            if (next[start] < 0 || seen[start]) continue;
            int loop[12], nl = 0;
            for (int e = start; !seen[e]; e = next[e]) {     // start is the loop's smallest edge
                seen[e] = true;
                loop[nl++] = e;
            }
            for (int k = 1; k + 1 < nl && nt < kMaxTri; ++k) {
                t->tri[cs][3 * nt] = (signed char)loop[0];
                t->tri[cs][3 * nt + 1] = (signed char)loop[k];
                t->tri[cs][3 * nt + 2] = (signed char)loop[k + 1];
                ++nt;
            }
        }
        t->ntri[cs] = (unsigned char)nt;
    }
}

const McTable& host_table() {
    static McTable t;
    static std::once_flag once;
    std::call_once(once, [] { build_table(&t); });
    return t;
}

// The 8 corner values of the cell whose lower corner is voxel (lx, ly, lz) of
// the block at bc; false when one is undefined.
template <int kS>
__device__ __forceinline__ bool cell_values(const int* __restrict__ table, const typename Codec<kS>::E* __restrict__ T,
                                            int nb, int slot, int4 bc, int lx, int ly, int lz, float2 sc, float v[8]) {
    const int ex = lx == 7, ey = ly == 7, ez = lz == 7;
    if ((ex && bc.x + 1 >= nb) || (ey && bc.y + 1 >= nb) || (ez && bc.z + 1 >= nb)) return false;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        const int ox = dx & ex, oy = dy & ey, oz = dz & ez;      // corner in the next block along that axis
        int s = slot;
        if (ox | oy | oz)
            s = __ldg(table + (unsigned)(bc.x + ox) +
                      (unsigned)nb * ((unsigned)(bc.y + oy) + (unsigned)nb * (unsigned)(bc.z + oz)));
        if (s < 0) return false;
        const int x = ox ? 0 : lx + dx, y = oy ? 0 : ly + dy, z = oz ? 0 : lz + dz;
        v[c] = Codec<kS>::load(T + (size_t)s * kBlockVoxels + x + 8 * y + 64 * z, sc);
        if (isnan(v[c])) return false;
    }
    return true;
}

__device__ __forceinline__ int cell_case(const float v[8]) {
    int cs = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) cs |= (v[c] < 0.0f ? 1 : 0) << c;
    return cs;
}

__device__ __forceinline__ int block_sum_int(int x, int* sm) {
    x = (int)warp_sum((unsigned)x);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sm[w] = x;
    __syncthreads();
    int t = 0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (int)(blockDim.x >> 5) ? sm[threadIdx.x] : 0;
        t = (int)warp_sum((unsigned)t);
        if (threadIdx.x == 0) sm[0] = t;
    }
    __syncthreads();
    t = sm[0];
    __syncthreads();
    return t;
}

template <int kS>
__global__ void __launch_bounds__(kBlockVoxels) mesh_count_kernel(const Counters* __restrict__ ctr,
                                                                  const int4* __restrict__ blocks,
                                                                  const int* __restrict__ table,
                                                                  const typename Codec<kS>::E* __restrict__ T, int nb,
                                                                  float2 sc, int* __restrict__ counts) {
    __shared__ int sm[32];
    const long long n = ctr->n_blocks;
    const int lx = threadIdx.x & 7, ly = (threadIdx.x >> 3) & 7, lz = threadIdx.x >> 6;
    for (long long b = blockIdx.x; b < n; b += gridDim.x) {
        const int4 bc = blocks[b];
        float v[8];
        int nt = 0;
        if (cell_values<kS>(table, T, nb, (int)b, bc, lx, ly, lz, sc, v)) nt = c_mc.ntri[cell_case(v)];
        const int tot = block_sum_int(nt, sm);
        if (threadIdx.x == 0) counts[b] = tot;
    }
}

// Exclusive scan of n counts by one CTA of 1024 threads: each thread owns a
// contiguous range; *total receives the sum.
__global__ void __launch_bounds__(1024) mesh_scan_kernel(const Counters* __restrict__ ctr, const int* __restrict__ counts,
                                                         long long* __restrict__ offsets,
                                                         long long* __restrict__ total) {
    __shared__ long long part[1024];
    const long long n = ctr->n_blocks;
    const long long per = (n + 1023) / 1024;
    const long long lo = threadIdx.x * per, hi = lo + per < n ? lo + per : n;
    long long s = 0;
    for (long long i = lo; i < hi; ++i) s += counts[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {        // inclusive Hillis-Steele scan
        const long long x = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += x;
        __syncthreads();
    }
    long long run = part[threadIdx.x] - s;
    for (long long i = lo; i < hi; ++i) {
        offsets[i] = run;
        run += counts[i];
    }
    if (threadIdx.x == 1023) *total = part[1023];
}

template <int kS>
__global__ void __launch_bounds__(kBlockVoxels) mesh_emit_kernel(const Counters* __restrict__ ctr,
                                                                 const int4* __restrict__ blocks,
                                                                 const int* __restrict__ table,
                                                                 const typename Codec<kS>::E* __restrict__ T, int nb,
                                                                 float2 sc, const long long* __restrict__ offsets,
                                                                 float ox, float oy, float oz, float s,
                                                                 float* __restrict__ out) {
    __shared__ int sw[kBlockVoxels / 32];
    const long long n = ctr->n_blocks;
    const int lx = threadIdx.x & 7, ly = (threadIdx.x >> 3) & 7, lz = threadIdx.x >> 6;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (long long b = blockIdx.x; b < n; b += gridDim.x) {
        const int4 bc = blocks[b];
        float v[8];
        int nt = 0, cs = 0;
        if (cell_values<kS>(table, T, nb, (int)b, bc, lx, ly, lz, sc, v)) {
            cs = cell_case(v);
            nt = c_mc.ntri[cs];
        }
        // rank of this cell's first triangle within the CTA (cells in thread order)
        int incl = nt;
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += x;
        }
        if (lane == 31) sw[w] = incl;
        __syncthreads();
        int before = 0;
        for (int k = 0; k < w; ++k) before += sw[k];
        __syncthreads();
        long long at = offsets[b] + before + incl - nt;
        const float cx = (float)(8 * bc.x + lx), cy = (float)(8 * bc.y + ly), cz = (float)(8 * bc.z + lz);
        for (int t = 0; t < nt; ++t, ++at) {
            for (int k = 0; k < 3; ++k) {
                const int e = c_mc.tri[cs][3 * t + k];
                const int axis = e >> 2, kk = e & 3;
                const int a = axis == 0 ? 2 * kk : axis == 1 ? (kk & 1) | ((kk & 2) << 1) : kk;   // edge start corner
                const int bcorner = a + (1 << axis);
                const float f = v[a] / (v[a] - v[bcorner]);
                float p[3] = {(float)(a & 1), (float)((a >> 1) & 1), (float)((a >> 2) & 1)};
                p[axis] += f;
                out[9 * at + 3 * k] = ox + (cx + p[0]) * s;
                out[9 * at + 3 * k + 1] = oy + (cy + p[1]) * s;
                out[9 * at + 3 * k + 2] = oz + (cz + p[2]) * s;
            }
        }
    }
}

template <int kS>
cudaError_t launch_mesh_s(tsdf_volume* v, float* out, bool emit, long long* d_total, cudaStream_t st) {
    auto* T = static_cast<const typename Codec<kS>::E*>(v->T);
    const float2 sc = make_float2((float)(v->cfg.truncation / 32767.0), (float)(32767.0 / v->cfg.truncation));
    const int grid = v->num_sms * 4;
    int* counts = reinterpret_cast<int*>(v->mesh_scratch);
    long long* offsets = reinterpret_cast<long long*>(v->mesh_scratch) + (v->cfg.block_capacity + 1) / 2;
    if (!emit) {
        mesh_count_kernel<kS><<<grid, kBlockVoxels, 0, st>>>(v->ctr, v->blocks, v->blk_slot, T, v->nb, sc, counts);
        mesh_scan_kernel<<<1, 1024, 0, st>>>(v->ctr, counts, offsets, d_total);
    } else {
        const float s = v->cfg.voxel_size;
        mesh_emit_kernel<kS><<<grid, kBlockVoxels, 0, st>>>(v->ctr, v->blocks, v->blk_slot, T, v->nb, sc, offsets,
                                                            (float)v->cfg.origin[0], (float)v->cfg.origin[1],
                                                            (float)v->cfg.origin[2], s, out);
    }
    return cudaGetLastError();
}

}  // namespace

int mesh_case(int cs, signed char* edges) {
    const McTable& t = host_table();
    std::memcpy(edges, t.tri[cs], 3 * kMaxTri);
    return t.ntri[cs];
}

// Count (emit = false: counts, offsets and the total, read back to *n) or write
// the triangles (emit = true; the counts of the previous call are reused).
cudaError_t launch_mesh(tsdf_volume* v, float* out, bool emit, long long* n, cudaStream_t st) {
    if (!v->mesh_table_ready) {
        cudaError_t e = cudaMemcpyToSymbolAsync(c_mc, &host_table(), sizeof(McTable), 0, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
        v->mesh_table_ready = 1;
    }
    if (!v->mesh_scratch) {
        // counts (int) and offsets (long long) per block, and the total
        const size_t bytes = ((size_t)(v->cfg.block_capacity + 1) / 2 + (size_t)v->cfg.block_capacity + 1) * 8;
        cudaError_t e = cudaMalloc(&v->mesh_scratch, bytes);
        if (e != cudaSuccess) return e;
    }
    long long* d_total = reinterpret_cast<long long*>(v->mesh_scratch) + (v->cfg.block_capacity + 1) / 2 +
                         v->cfg.block_capacity;
    cudaError_t e;
    switch (v->cfg.storage) {
        case TSDF_STORAGE_F16: e = launch_mesh_s<TSDF_STORAGE_F16>(v, out, emit, d_total, st); break;
        case TSDF_STORAGE_SNORM16: e = launch_mesh_s<TSDF_STORAGE_SNORM16>(v, out, emit, d_total, st); break;
        default: e = launch_mesh_s<TSDF_STORAGE_F32>(v, out, emit, d_total, st); break;
    }
    if (e != cudaSuccess || emit) return e;
    e = cudaMemcpyAsync(n, d_total, sizeof(long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

}  // namespace tsdf
