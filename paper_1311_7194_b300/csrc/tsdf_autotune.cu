// Launch-shape autotuner.
//
// The integrate kernel's voxels per thread (4 or 8, i.e. 128 or 64 threads per
// 8^3 block) and persistent CTAs per SM, and the raycast kernel's pixel tile or
// its persistent state-machine form,
// change how work is spread over the GPU but not a single operation on any
// voxel or ray, so every choice gives identical results; only speed differs
// with the scene, image size and grid. tsdf_autotune times every candidate on
// frames the caller provides, with CUDA events around the stage being tuned,
// keeps the fastest, and remembers it in a JSON-lines cache keyed by GPU name,
// image size, grid size and storage format.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "tsdf_internal.cuh"

namespace {

struct Candidate {
    int vpt, ctas, tw, th;
};

const int kCtaChoices[] = {4, 8, 12, 16, 24, 32};
const int kTiles[][2] = {{16, 8}, {8, 8}, {32, 4}, {8, 16}, {16, 16}};

std::string cache_key(const tsdf_volume* v, const tsdf_intrinsics& K) {
    cudaDeviceProp prop;
    std::string name = "unknown-gpu";
    if (cudaGetDeviceProperties(&prop, v->device) == cudaSuccess) name = prop.name;
    const char* st = v->cfg.storage == TSDF_STORAGE_F16 ? "f16" : v->cfg.storage == TSDF_STORAGE_SNORM16 ? "snorm16" : "f32";
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s|%dx%d|G%d|%s", name.c_str(), K.width, K.height, v->cfg.grid_dim, st);
    return buf;
}

bool read_int(const std::string& line, const char* field, int* out) {
    const std::string pat = std::string("\"") + field + "\":";
    const size_t at = line.find(pat);
    if (at == std::string::npos) return false;
    *out = std::atoi(line.c_str() + at + pat.size());
    return true;
}

// One JSON object per line: {"key": "...", "integrate_vpt": 4, ...}
bool cache_lookup(const char* path, const std::string& key, tsdf::LaunchConfig* lc) {
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char buf[1024];
    bool found = false;
    const std::string kpat = "\"key\": \"" + key + "\"";
    while (!found && std::fgets(buf, sizeof(buf), f)) {
        const std::string line(buf);
        if (line.find(kpat) == std::string::npos) continue;
        tsdf::LaunchConfig c;
        found = read_int(line, "integrate_vpt", &c.integrate_vpt) &&
                read_int(line, "integrate_ctas_per_sm", &c.integrate_ctas_per_sm) &&
                read_int(line, "raycast_tile_w", &c.raycast_tile_w) &&
                read_int(line, "raycast_tile_h", &c.raycast_tile_h) &&
                read_int(line, "raycast_persistent", &c.raycast_persistent);
        if (found) *lc = c;
    }
    std::fclose(f);
    return found;
}

void cache_store(const char* path, const std::string& key, const tsdf::LaunchConfig& c, double int_ms, double rc_ms) {
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f,
                 "{\"key\": \"%s\", \"integrate_vpt\": %d, \"integrate_ctas_per_sm\": %d, \"raycast_tile_w\": %d, "
                 "\"raycast_tile_h\": %d, \"raycast_persistent\": %d, \"integrate_ms_per_frame\": %.6f, "
                 "\"raycast_ms_per_frame\": %.6f}\n",
                 key.c_str(), c.integrate_vpt, c.integrate_ctas_per_sm, c.raycast_tile_w, c.raycast_tile_h,
                 c.raycast_persistent, int_ms, rc_ms);
    std::fclose(f);
}

bool valid(const tsdf_launch_config& c) {
    if (c.integrate_voxels_per_thread != 4 && c.integrate_voxels_per_thread != 8) return false;
    if (c.raycast_persistent != 0 && c.raycast_persistent != 1) return false;
    if (c.integrate_ctas_per_sm < 1 || c.integrate_ctas_per_sm > 32) return false;
    for (const auto& t : kTiles)
        if (t[0] == c.raycast_tile_w && t[1] == c.raycast_tile_h) return true;
    return false;
}

}  // namespace

extern "C" {

tsdf_status tsdf_get_launch_config(const tsdf_volume* v, tsdf_launch_config* out) {
    if (!v || !out) return TSDF_ERR_INVALID_ARG;
    out->integrate_voxels_per_thread = v->lc.integrate_vpt;
    out->integrate_ctas_per_sm = v->lc.integrate_ctas_per_sm;
    out->raycast_tile_w = v->lc.raycast_tile_w;
    out->raycast_tile_h = v->lc.raycast_tile_h;
    out->raycast_persistent = v->lc.raycast_persistent;
    return TSDF_OK;
}

tsdf_status tsdf_set_launch_config(tsdf_volume* v, const tsdf_launch_config* c) {
    if (!v || !c || !valid(*c)) return TSDF_ERR_INVALID_ARG;
    v->lc = tsdf::LaunchConfig{c->integrate_voxels_per_thread, c->integrate_ctas_per_sm, c->raycast_tile_w,
                               c->raycast_tile_h, c->raycast_persistent};
    return TSDF_OK;
}

tsdf_status tsdf_autotune(tsdf_volume* v, int32_t n, const float* const* depth, const tsdf_intrinsics* K,
                          const double* poses, const char* cache_path, tsdf_launch_config* out,
                          int32_t* from_cache) {
    if (!v || n < 1 || !depth || !K || !poses) return TSDF_ERR_INVALID_ARG;
    for (int k = 0; k < n; ++k)
        if (!depth[k] || !tsdf::pose_valid(poses + 16 * k)) return TSDF_ERR_INVALID_ARG;
    if (!tsdf::intrinsics_valid(K)) return TSDF_ERR_INVALID_ARG;
    if (from_cache) *from_cache = 0;
    const std::string key = cache_key(v, *K);
    tsdf::LaunchConfig best = v->lc;
    if (cache_path && cache_lookup(cache_path, key, &best)) {
        v->lc = best;
        if (from_cache) *from_cache = 1;
        return out ? tsdf_get_launch_config(v, out) : TSDF_OK;
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float *d_out = nullptr, *n_out = nullptr, *v_out = nullptr;
    const size_t npix = (size_t)K->width * K->height;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaMalloc(&d_out, npix * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&n_out, 3 * npix * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&v_out, 3 * npix * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_out); cudaFree(n_out); cudaFree(v_out);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
        return TSDF_ERR_CUDA;
    }
    tsdf_status status = TSDF_OK;
    // integrate: fuse the frames from an empty volume, timing only the integrate calls
    double best_int = 1e30;
    for (int vpt : {4, 8}) {
        for (int ctas : kCtaChoices) {
            v->lc.integrate_vpt = vpt;
            v->lc.integrate_ctas_per_sm = ctas;
            double t_min = 1e30;
            for (int rep = 0; rep < 2 && status == TSDF_OK; ++rep) {
                status = tsdf_reset(v, st);
                double t = 0.0;
                for (int k = 0; k < n && status == TSDF_OK; ++k) {
                    status = tsdf_allocate(v, depth[k], K, poses + 16 * k, st);
                    if (status == TSDF_OK) cudaEventRecord(e0, st);
                    if (status == TSDF_OK) status = tsdf_integrate(v, depth[k], nullptr, K, poses + 16 * k, st);
                    if (status == TSDF_OK) cudaEventRecord(e1, st);
                    float ms = 0.0f;
                    if (status == TSDF_OK && cudaEventSynchronize(e1) == cudaSuccess &&
                        cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
                        t += ms;
                }
                if (t < t_min) t_min = t;
            }
            if (status == TSDF_OK && t_min < best_int) {
                best_int = t_min;
                best.integrate_vpt = vpt;
                best.integrate_ctas_per_sm = ctas;
            }
        }
    }
    // raycast: on the fused volume, at every frame's pose
    v->lc.integrate_vpt = best.integrate_vpt;
    v->lc.integrate_ctas_per_sm = best.integrate_ctas_per_sm;
    double best_rc = 1e30;
    for (int cand = 0; cand <= (int)(sizeof(kTiles) / sizeof(kTiles[0])); ++cand) {
        // every pixel-tile shape, then the persistent kernel
        const bool persistent = cand == (int)(sizeof(kTiles) / sizeof(kTiles[0]));
        const int tw = persistent ? best.raycast_tile_w : kTiles[cand][0];
        const int th = persistent ? best.raycast_tile_h : kTiles[cand][1];
        v->lc.raycast_tile_w = tw;
        v->lc.raycast_tile_h = th;
        v->lc.raycast_persistent = persistent ? 1 : 0;
        double t_min = 1e30;
        for (int rep = 0; rep < 2 && status == TSDF_OK; ++rep) {
            double t = 0.0;
            for (int k = 0; k < n && status == TSDF_OK; ++k) {
                cudaEventRecord(e0, st);
                status = tsdf_raycast(v, K, poses + 16 * k, d_out, n_out, v_out, st);
                cudaEventRecord(e1, st);
                float ms = 0.0f;
                if (status == TSDF_OK && cudaEventSynchronize(e1) == cudaSuccess &&
                    cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
                    t += ms;
            }
            if (t < t_min) t_min = t;
        }
        if (status == TSDF_OK && t_min < best_rc) {
            best_rc = t_min;
            best.raycast_tile_w = tw;
            best.raycast_tile_h = th;
            best.raycast_persistent = persistent ? 1 : 0;
        }
    }
    v->lc = best;
    if (status == TSDF_OK) status = tsdf_reset(v, st);
    if (status == TSDF_OK && cudaStreamSynchronize(st) != cudaSuccess) status = TSDF_ERR_CUDA;
    v->last_stream = nullptr;
    cudaFree(d_out); cudaFree(n_out); cudaFree(v_out);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (status != TSDF_OK) return status;
    if (cache_path) cache_store(cache_path, key, best, best_int / n, best_rc / n);
    return out ? tsdf_get_launch_config(v, out) : TSDF_OK;
}

}  // extern "C"
