// CUDA-graph driver of one fusion step: allocate -> integrate -> raycast.
//
// A step fuses K frames (K = 1: tsdf_allocate + tsdf_integrate; K > 1: the
// batched path of tsdf_integrate_batch) and raycasts the model at the last
// frame's pose. Per step the host records the step's kernels on a private
// stream under stream capture, updates one instantiated executable graph in
// place with the new kernel parameters (cudaGraphExecUpdate; the kernel
// sequence never changes shape, so the update succeeds and no re-instantiation
// is needed), and launches it on the caller's stream. The GPU then runs the
// 12 (K = 1) or 5K + 8 small kernels back to back without per-kernel launch
// gaps. Optional caller events recorded at the stage boundaries become event
// nodes of the graph, so stage times can still be measured per step.
// Every size the kernels need lives in device counters, which is what
// makes the step capturable: no host round trip, no allocation (buffers are
// sized by tsdf_graph_create).
//
// Host-input steps (tsdf_graph_launch_host) copy the step's depth maps into one
// of two device staging sets on a private copy stream and make the caller's
// stream wait for that copy only. The sets alternate per step, and a set is
// overwritten only after the step that read it (two steps back) has run, so
// the copy of step n + 1 overlaps the kernels of step n.
#include <cstdlib>
#include <cstring>

#include "tsdf_internal.cuh"

struct tsdf_graph {
    tsdf_volume* vol;
    int32_t K;
    tsdf_intrinsics intr;
    cudaStream_t cap;          // private stream the step is captured on
    cudaGraphExec_t exec;      // instantiated step, updated in place per launch
    int64_t steps;
    int64_t instantiations;
    cudaEvent_t events[4];     // optional stage-boundary events for the next launch
    // host-input steps: two staging sets of K depth maps, filled on `copy`
    cudaStream_t copy;
    float* stage;              // [2][K][width * height]
    cudaEvent_t copied[2];     // the set's copy is done
    cudaEvent_t done[2];       // the step that read the set has run
    int done_valid[2];
    int64_t host_steps;
};

namespace {

void free_host_staging(tsdf_graph* g) {
    if (g->copy) cudaStreamSynchronize(g->copy);
    for (int b = 0; b < 2; ++b) {
        if (g->copied[b]) cudaEventDestroy(g->copied[b]);
        if (g->done[b]) cudaEventDestroy(g->done[b]);
        g->copied[b] = g->done[b] = nullptr;
        g->done_valid[b] = 0;
    }
    if (g->stage) cudaFree(g->stage);
    if (g->copy) cudaStreamDestroy(g->copy);
    g->stage = nullptr;
    g->copy = nullptr;
}

// Created on the first host-input step (may allocate and synchronise).
tsdf_status ensure_host_staging(tsdf_graph* g) {
    if (g->stage) return TSDF_OK;
    const size_t npix = (size_t)g->intr.width * g->intr.height;
    cudaError_t e = cudaStreamCreateWithFlags(&g->copy, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaEventCreateWithFlags(&g->copied[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->done[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMalloc(&g->stage, 2 * (size_t)g->K * npix * sizeof(float));
    if (e == cudaSuccess) return TSDF_OK;
    const tsdf_status s = e == cudaErrorMemoryAllocation ? TSDF_ERR_OUT_OF_MEMORY : TSDF_ERR_CUDA;
    cudaGetLastError();
    free_host_staging(g);
    return s;
}

}  // namespace

extern "C" {

tsdf_status tsdf_graph_create(tsdf_volume* v, int32_t K, const tsdf_intrinsics* Kin, tsdf_graph** out) {
    if (!v || !out || K < 1 || K > tsdf::kMaxBatch || !tsdf::intrinsics_valid(Kin)) return TSDF_ERR_INVALID_ARG;
    *out = nullptr;
    cudaStream_t st = v->last_stream;
    cudaError_t e = tsdf::ensure_dtiles(v, *Kin, st);
    if (e == cudaSuccess && K > 1) e = tsdf::ensure_batch(v, *Kin, st);
    if (e == cudaSuccess) e = tsdf::ensure_range(v, *Kin, st);
    if (e != cudaSuccess) return TSDF_ERR_CUDA;
    tsdf_graph* g = (tsdf_graph*)std::calloc(1, sizeof(tsdf_graph));
    if (!g) return TSDF_ERR_OUT_OF_MEMORY;
    g->vol = v;
    g->K = K;
    g->intr = *Kin;
    if (cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking) != cudaSuccess) {
        std::free(g);
        return TSDF_ERR_CUDA;
    }
    *out = g;
    return TSDF_OK;
}

void tsdf_graph_destroy(tsdf_graph* g) {
    if (!g) return;
    if (g->vol && g->vol->last_stream) cudaStreamSynchronize(g->vol->last_stream);
    free_host_staging(g);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    cudaStreamDestroy(g->cap);
    std::free(g);
}

tsdf_status tsdf_graph_launch(tsdf_graph* g, const float* const* depth, const float* const* variance,
                              const double* poses_wc, float* depth_out, float* normal_out, float* vertex_out,
                              void* stream) {
    if (!g || !depth || !poses_wc) return TSDF_ERR_INVALID_ARG;
    tsdf_volume* v = g->vol;
    const int K = g->K;
    for (int k = 0; k < K; ++k) {
        if (!depth[k] || !tsdf::pose_valid(poses_wc + 16 * k)) return TSDF_ERR_INVALID_ARG;
        if (variance && !variance[k]) return TSDF_ERR_INVALID_ARG;
    }
    // record the step
    cudaError_t e = cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return TSDF_ERR_CUDA;
    cudaError_t le = cudaSuccess;
    if (g->events[0]) le = cudaEventRecordWithFlags(g->events[0], g->cap, cudaEventRecordExternal);
    if (K == 1) {
        const tsdf::AllocParams ap = tsdf::make_alloc_params(v, g->intr, poses_wc);
        if (le == cudaSuccess) le = tsdf::launch_allocate(v, depth[0], ap, (int)v->frame, g->cap);
        if (le == cudaSuccess && g->events[1]) le = cudaEventRecordWithFlags(g->events[1], g->cap, cudaEventRecordExternal);
        if (le == cudaSuccess)
            // the step raycasts at the pose it fuses: one cull pass makes both
            // visible lists (integrate and raycast)
            le = tsdf::launch_integrate(v, depth[0], variance ? variance[0] : nullptr,
                                        tsdf::make_frame_params(v, g->intr, poses_wc), g->cap, true);
    } else {
        tsdf::BatchParams bp;
        std::memset(&bp, 0, sizeof(bp));
        bp.K = K;
        bp.f0 = (int)v->frame;
        for (int k = 0; k < K && le == cudaSuccess; ++k) {
            const tsdf::AllocParams ap = tsdf::make_alloc_params(v, g->intr, poses_wc + 16 * k);
            le = tsdf::launch_allocate(v, depth[k], ap, (int)v->frame + k, g->cap);
            bp.fp[k] = tsdf::make_frame_params(v, g->intr, poses_wc + 16 * k);
            bp.depth[k] = depth[k];
            bp.var[k] = variance ? variance[k] : nullptr;
        }
        if (le == cudaSuccess && g->events[1]) le = cudaEventRecordWithFlags(g->events[1], g->cap, cudaEventRecordExternal);
        if (le == cudaSuccess) le = tsdf::launch_integrate_batch(v, bp, g->cap);
    }
    if (le == cudaSuccess && g->events[2]) le = cudaEventRecordWithFlags(g->events[2], g->cap, cudaEventRecordExternal);
    if (le == cudaSuccess)
        le = tsdf::launch_raycast(v, tsdf::make_frame_params(v, g->intr, poses_wc + 16 * (K - 1)), depth_out,
                                  normal_out, vertex_out, g->cap, K == 1);
    if (le == cudaSuccess && g->events[3]) le = cudaEventRecordWithFlags(g->events[3], g->cap, cudaEventRecordExternal);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(g->cap, &graph);
    if (le != cudaSuccess || e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (v->host_error == TSDF_OK) v->host_error = TSDF_ERR_CUDA;
        return TSDF_ERR_CUDA;
    }
    // refresh the executable graph in place, instantiate on first use (or if
    // the update is refused)
    if (g->exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(g->exec, graph, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(g->exec);
            g->exec = nullptr;
        }
    }
    if (!g->exec) {
        e = cudaGraphInstantiate(&g->exec, graph, 0);
        ++g->instantiations;
    }
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        g->exec = nullptr;
        if (v->host_error == TSDF_OK) v->host_error = TSDF_ERR_CUDA;
        return TSDF_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    e = cudaGraphLaunch(g->exec, st);
    if (e != cudaSuccess) {
        if (v->host_error == TSDF_OK) v->host_error = TSDF_ERR_CUDA;
        return TSDF_ERR_CUDA;
    }
    v->last_stream = st;
    v->frame += K;
    ++g->steps;
    return TSDF_OK;
}

tsdf_status tsdf_graph_launch_host(tsdf_graph* g, const float* const* depth_host, const double* poses_wc,
                                   float* depth_out, float* normal_out, float* vertex_out, void* stream) {
    if (!g || !depth_host || !poses_wc) return TSDF_ERR_INVALID_ARG;
    const int K = g->K;
    for (int k = 0; k < K; ++k)
        if (!depth_host[k] || !tsdf::pose_valid(poses_wc + 16 * k)) return TSDF_ERR_INVALID_ARG;
    tsdf_status s = ensure_host_staging(g);
    if (s != TSDF_OK) return s;
    tsdf_volume* v = g->vol;
    const size_t npix = (size_t)g->intr.width * g->intr.height;
    const int b = (int)(g->host_steps & 1);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    // the set is free once the step that read it (two host steps back) has run
    if (g->done_valid[b]) e = cudaStreamWaitEvent(g->copy, g->done[b], 0);
    const float* dev[tsdf::kMaxBatch];
    for (int k = 0; k < K && e == cudaSuccess; ++k) {
        float* d = g->stage + ((size_t)b * K + k) * npix;
        e = cudaMemcpyAsync(d, depth_host[k], npix * sizeof(float), cudaMemcpyHostToDevice, g->copy);
        dev[k] = d;
    }
    if (e == cudaSuccess) e = cudaEventRecord(g->copied[b], g->copy);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, g->copied[b], 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (v->host_error == TSDF_OK) v->host_error = TSDF_ERR_CUDA;
        return TSDF_ERR_CUDA;
    }
    s = tsdf_graph_launch(g, dev, nullptr, poses_wc, depth_out, normal_out, vertex_out, stream);
    if (s != TSDF_OK) return s;
    e = cudaEventRecord(g->done[b], st);
    if (e != cudaSuccess) {
        if (v->host_error == TSDF_OK) v->host_error = TSDF_ERR_CUDA;
        return TSDF_ERR_CUDA;
    }
    g->done_valid[b] = 1;
    ++g->host_steps;
    return TSDF_OK;
}

int64_t tsdf_graph_instantiations(const tsdf_graph* g) { return g ? g->instantiations : -1; }

tsdf_status tsdf_graph_set_events(tsdf_graph* g, void* const events[4]) {
    if (!g) return TSDF_ERR_INVALID_ARG;
    for (int i = 0; i < 4; ++i) g->events[i] = events ? (cudaEvent_t)events[i] : nullptr;
    return TSDF_OK;
}

}  // extern "C"
