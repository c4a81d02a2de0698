// tsdf_raycast_noalloc: the raycast of tsdf_raycast without any device memory
// allocation during the call.
//
// tsdf_raycast keeps its near / far range maps (one pair per 4x4-pixel tile) in
// device memory that it grows with cudaMalloc the first time it sees a larger
// image (and cudaFree of the old maps, which synchronises the device). Some callers cannot have that
// happen inside the call: a real-time loop whose memory budget is fixed up front
// and that must not stall on an allocation or on the implicit device-wide
// synchronisation of cudaFree, an application whose own allocator owns all
// device memory, or a caller recording work for later replay. For them this
// entry point takes the range maps from a fixed array that is part of the
// library's device image instead.
//
// The array, tsdf_noalloc_range, holds the near and far range maps of one
// image (one pair of words per 4x4-pixel tile, at most kNoAllocMaxTiles =
// 81,920 tiles) and the raycast's ray-order lists (kRayBuckets lists of at most
// kNoAllocMaxRayTiles = 40,960 tiles of 8x4 pixels): every image of up to
// 1280 x 1024 pixels fits. That is 1.25 MiB, held on every GPU that loads the
// library until the process exits. Images with more tiles are rejected with
// TSDF_ERR_INVALID_ARG. All calls on a
// device share the array and it keeps whatever the last call left in it; the
// kernels clear both maps at the start of every call, so nothing depends on the
// previous contents. Two calls whose work overlaps on the GPU (different
// streams, or different volumes on concurrent streams) race on the array and
// produce garbage: serialise them.
//
// Host code must not use the array's name as a device address (on the host it is
// only a stand-in symbol). The first call on each device, with that device
// current, asks the runtime for the array's device address with
// cudaGetSymbolAddress and caches it; that first call should therefore come
// before any stream capture on the device. The cached address belongs to the
// device's context as it was then: it does not survive cudaDeviceReset.
#include <mutex>

#include "tsdf_internal.cuh"

namespace {
constexpr int64_t kNoAllocMaxTiles = (1280 / tsdf::kRangeTile) * (1024 / tsdf::kRangeTile);
constexpr int64_t kNoAllocMaxRayTiles = (1280 / 8) * (1024 / 4);
constexpr int64_t kNoAllocWords = 2 * kNoAllocMaxTiles + tsdf::kRayBuckets * kNoAllocMaxRayTiles;
constexpr int kMaxDevices = 64;
}  // namespace

// near map in the first kNoAllocMaxTiles words, far map in the next
// kNoAllocMaxTiles, then the ray-order lists
static __device__ __align__(256) unsigned int tsdf_noalloc_range[kNoAllocWords];

namespace {

std::mutex g_setup_mutex;
unsigned int* g_range_addr[kMaxDevices];   // device address of tsdf_noalloc_range per device

}  // namespace

extern "C" tsdf_status tsdf_raycast_noalloc(tsdf_volume* v, const tsdf_intrinsics* K, const double pose_wc[16],
                                            float* depth_out, float* normal_out, float* vertex_out, void* stream) {
    if (!v || !tsdf::intrinsics_valid(K) || !tsdf::pose_valid(pose_wc)) return TSDF_ERR_INVALID_ARG;
    if (tsdf::range_tiles(K->width, K->height) > kNoAllocMaxTiles ||
        tsdf::ray_tiles(K->width, K->height) > kNoAllocMaxRayTiles)
        return TSDF_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSDF_ERR_CUDA;
    if (dev != v->device || dev < 0 || dev >= kMaxDevices) return TSDF_ERR_INVALID_ARG;
    unsigned int* range = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_range_addr[dev]) {
            void* ptr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&ptr, tsdf_noalloc_range);
            if (e != cudaSuccess || ptr == nullptr) {
                if (v->host_error == TSDF_OK) v->host_error = TSDF_ERR_CUDA;
                return TSDF_ERR_CUDA;
            }
            g_range_addr[dev] = static_cast<unsigned int*>(ptr);
        }
        range = g_range_addr[dev];
    }
    const tsdf::FrameParams p = tsdf::make_frame_params(v, *K, pose_wc);
    cudaStream_t st = (cudaStream_t)stream;
    v->last_stream = st;
    int* order = reinterpret_cast<int*>(range + 2 * kNoAllocMaxTiles);
    const cudaError_t e = tsdf::launch_raycast_ranges(v, p, range, range + kNoAllocMaxTiles, order, depth_out,
                                                      normal_out, vertex_out, st);
    if (e != cudaSuccess) {
        if (v->host_error == TSDF_OK) v->host_error = TSDF_ERR_CUDA;
        return TSDF_ERR_CUDA;
    }
    return TSDF_OK;
}
