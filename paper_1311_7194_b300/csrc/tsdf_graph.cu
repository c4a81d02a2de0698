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
};

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
            le = tsdf::launch_integrate(v, depth[0], variance ? variance[0] : nullptr,
                                        tsdf::make_frame_params(v, g->intr, poses_wc), g->cap);
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
                                  normal_out, vertex_out, g->cap);
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

int64_t tsdf_graph_instantiations(const tsdf_graph* g) { return g ? g->instantiations : -1; }

tsdf_status tsdf_graph_set_events(tsdf_graph* g, void* const events[4]) {
    if (!g) return TSDF_ERR_INVALID_ARG;
    for (int i = 0; i < 4; ++i) g->events[i] = events ? (cudaEvent_t)events[i] : nullptr;
    return TSDF_OK;
}

}  // extern "C"
