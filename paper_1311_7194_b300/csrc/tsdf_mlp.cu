// Learned measurement variance: inference fused into the integrate stage, and
// the kernels that train the network on the GPU.
//
// The paper weights each measurement by its variance p_k (Alg. 3) and notes
// that deviation grows with depth and that data near surface edges is poorer;
// it leaves p_k's estimation open. This network, a 27-32-32-1 perceptron with
// ReLU and bfloat16 weights, predicts out = log(p_k / p_quad) at a pixel from
// its 5x5 depth patch (differences to the centre over delta, clamped to
// [-1, 1], +1 where a neighbour is missing), depth / 4 and the incidence cosine
// from the depth map's central differences; p_k = p_quad exp(out), falling back
// to p_quad when out lies outside [-ln 4, ln 64] or is not finite. Parameters: W1[32][27],
// b1[32], W2[32][32], b2[32], W3[32], b3.
//
//   inference (tsdf_mlp.cuh): weights decoded once per CTA into shared memory
//       (read as broadcasts). The integrate stage evaluates the network inside
//       depth_tiles_mlp_kernel, where it forms the measurement map (D, p_k)
//       (tsdf_integrate with a network set and no variance map), as register
//       tiles of pixels x neurons with the same operations as mlp_eval;
//       variance_mlp_kernel writes the same p_k as a map (tsdf_mlp_variance).
//   harvest_kernel: training pairs from a measured depth map and the model's
//       raycast at the same pose: features and s = r^2 / p_quad for pixels whose
//       residual r lies within kHarvestBand truncation distances (wider than the
//       band itself, so that the heavy errors of poor pixels - near depth edges,
//       at grazing angles - are part of what the network learns).
//   mlp_grad_kernel: one warp per sample, lane j = hidden unit j: forward, the
//       Gaussian NLL (out + s exp(-out)) / 2 and its backward pass, gradients
//       summed in registers, then shared memory, then one atomic per parameter
//       per CTA.
//   mlp_adam_kernel: Adam on float32 master weights, re-rounded to bfloat16.
// Inference and training evaluate the same bfloat16 weights with float32
// arithmetic.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

#include "tsdf_mlp.cuh"

namespace tsdf {
namespace {

constexpr float kHarvestBand = 4.0f;   // residuals kept: |r| <= kHarvestBand * delta

__global__ void __launch_bounds__(128) variance_mlp_kernel(const float* __restrict__ depth, FrameParams p,
                                                           const __nv_bfloat16* __restrict__ w,
                                                           float* __restrict__ var) {
    __shared__ __align__(16) float smem[kInferFloats];
    const MlpInfer m = load_infer(w, smem);
    const int u = blockIdx.x * 16 + (threadIdx.x & 15);
    const int v = blockIdx.y * 8 + (threadIdx.x >> 4);
    if (u >= p.width || v >= p.height) return;
    var[(size_t)v * p.width + u] = learned_variance(m, depth, p, u, v);
}

__global__ void __launch_bounds__(256) features_kernel(const float* __restrict__ depth, FrameParams p, long long n,
                                                       const int* __restrict__ uv, float* __restrict__ feats,
                                                       unsigned char* __restrict__ valid) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        float f[kIn];
        const bool ok = pixel_features(depth, p, uv[2 * k], uv[2 * k + 1], f);
        for (int i = 0; i < kIn; ++i) feats[k * kIn + i] = ok ? f[i] : 0.0f;
        if (valid) valid[k] = ok ? 1 : 0;
    }
}

__global__ void __launch_bounds__(256) harvest_kernel(const float* __restrict__ depth, const float* __restrict__ pred,
                                                      FrameParams p, long long max_n, float* __restrict__ feats,
                                                      float* __restrict__ s, unsigned int* __restrict__ count) {
    const int lane = threadIdx.x & 31;
    const long long npix = (long long)p.width * p.height;
    for (long long b0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); b0 < npix;
         b0 += (long long)gridDim.x * blockDim.x) {
        const long long k = b0 + lane;
        float f[kIn];
        bool take = false;
        float sv = 0.0f;
        if (k < npix) {
            const int u = (int)(k % p.width), v = (int)(k / p.width);
            const float dh = pred[k];
            if (dh > 0.0f && pixel_features(depth, p, u, v, f)) {
                const float d = depth[k];
                const float r = d - dh;
                const float sg = __fmul_rn(__fmul_rn(p.sigma_coeff, d), d);
                const float pq = __fmul_rn(sg, sg);
                take = fabsf(r) <= kHarvestBand * p.delta && pq > 0.0f;
                sv = r * r / pq;
            }
        }
        const unsigned msk = __ballot_sync(0xffffffffu, take);
        if (!msk) continue;
        unsigned base = 0;
        if (lane == __ffs(msk) - 1) base = atomicAdd(count, (unsigned)__popc(msk));
        base = __shfl_sync(0xffffffffu, base, __ffs(msk) - 1);
        const long long at = (long long)base + __popc(msk & ((1u << lane) - 1u));
        if (take && at < max_n) {
            for (int i = 0; i < kIn; ++i) feats[at * kIn + i] = f[i];
            s[at] = sv;
        }
    }
}

__global__ void __launch_bounds__(128) forward_kernel(const __nv_bfloat16* __restrict__ w, long long n,
                                                      const float* __restrict__ feats, float* __restrict__ out) {
    __shared__ __align__(16) float smem[kInferFloats];
    const MlpInfer m = load_infer(w, smem);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        float f[kIn];
#pragma unroll
        for (int i = 0; i < kIn; ++i) f[i] = feats[k * kIn + i];
        out[k] = mlp_eval(m, f);
    }
}

__global__ void __launch_bounds__(256) mlp_grad_kernel(const __nv_bfloat16* __restrict__ w, long long n,
                                                       const int* __restrict__ idx, const float* __restrict__ feats,
                                                       const float* __restrict__ s, float* __restrict__ grad,
                                                       float* __restrict__ loss) {
    __shared__ float smem[kSmemFloats];
    __shared__ float gsum[kMlpParams];
    const MlpShared m = load_weights(w, smem);
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) gsum[i] = 0.0f;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int j = lane;                       // hidden unit of this lane
    float gW1[kIn], gW2[kHid];
#pragma unroll
    for (int i = 0; i < kIn; ++i) gW1[i] = 0.0f;
#pragma unroll
    for (int i = 0; i < kHid; ++i) gW2[i] = 0.0f;
    float gb1 = 0.0f, gb2 = 0.0f, gW3 = 0.0f, gb3 = 0.0f, L = 0.0f;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long t = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < n; t += warps) {
        const long long k = idx ? (long long)idx[t] : t;
        const float xi = lane < kIn ? feats[k * kIn + lane] : 0.0f;
        const float sk = s[k];
        float h1 = m.b1[j];
#pragma unroll
        for (int i = 0; i < kIn; ++i) h1 = fmaf(m.W1[j * kIn + i], __shfl_sync(0xffffffffu, xi, i), h1);
        const float a1 = fmaxf(h1, 0.0f);
        float h2 = m.b2[j];
#pragma unroll
        for (int i = 0; i < kHid; ++i) h2 = fmaf(m.W2[j * kW2Pitch + i], __shfl_sync(0xffffffffu, a1, i), h2);
        const float a2 = fmaxf(h2, 0.0f);
        float out = m.W3[j] * a2;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) out += __shfl_xor_sync(0xffffffffu, out, o);
        out += m.b3;
        const float e = sk * expf(-out);
        const float g = 0.5f * (1.0f - e);    // dL/dout
        L += 0.5f * (out + e);
        gb3 += g;
        gW3 = fmaf(g, a2, gW3);
        const float d2 = h2 > 0.0f ? g * m.W3[j] : 0.0f;
        gb2 += d2;
#pragma unroll
        for (int i = 0; i < kHid; ++i) gW2[i] = fmaf(d2, __shfl_sync(0xffffffffu, a1, i), gW2[i]);
        float acc = 0.0f;                     // sum over units q of W2[q][j] * d2_q
#pragma unroll
        for (int q = 0; q < kHid; ++q) acc = fmaf(m.W2[q * kW2Pitch + j], __shfl_sync(0xffffffffu, d2, q), acc);
        const float d1 = h1 > 0.0f ? acc : 0.0f;
        gb1 += d1;
#pragma unroll
        for (int i = 0; i < kIn; ++i) gW1[i] = fmaf(d1, __shfl_sync(0xffffffffu, xi, i), gW1[i]);
    }
    for (int i = 0; i < kIn; ++i) atomicAdd(&gsum[j * kIn + i], gW1[i]);
    atomicAdd(&gsum[kOffB1 + j], gb1);
    for (int i = 0; i < kHid; ++i) atomicAdd(&gsum[kOffW2 + j * kHid + i], gW2[i]);
    atomicAdd(&gsum[kOffB2 + j], gb2);
    atomicAdd(&gsum[kOffW3 + j], gW3);
    if (lane == 0) {
        atomicAdd(&gsum[kOffB3], gb3);
        atomicAdd(loss, L);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) atomicAdd(grad + i, gsum[i]);
}

__global__ void mlp_adam_kernel(float* __restrict__ w32, __nv_bfloat16* __restrict__ wq, float* __restrict__ m,
                                float* __restrict__ v, float* __restrict__ grad, float lr, float b1, float b2,
                                float eps, float gscale, float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    const float g = grad[i] * gscale;
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float wi = w32[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    w32[i] = wi;
    wq[i] = __float2bfloat16_rn(wi);
    grad[i] = 0.0f;
}

FrameParams frame_of(const tsdf_volume* v, const tsdf_intrinsics& K) {
    const double eye[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
    return make_frame_params(v, K, eye);
}

bool ok_ptr(const void* p) { return p != nullptr; }

}  // namespace

cudaError_t launch_variance_mlp(tsdf_volume* v, const float* depth, const FrameParams& p, float* var,
                                cudaStream_t st) {
    const dim3 grid((unsigned)((p.width + 15) / 16), (unsigned)((p.height + 7) / 8));
    variance_mlp_kernel<<<grid, 128, 0, st>>>(depth, p, static_cast<const __nv_bfloat16*>(v->mlp_w), var);
    return cudaGetLastError();
}

}  // namespace tsdf

using tsdf::kMlpParams;

extern "C" {

int32_t tsdf_mlp_param_count(void) { return kMlpParams; }

tsdf_status tsdf_set_variance_mlp(tsdf_volume* v, const uint16_t* bf16_weights, int64_t n) {
    if (!v) return TSDF_ERR_INVALID_ARG;
    if (!bf16_weights || n == 0) {
        if (v->last_stream) cudaStreamSynchronize(v->last_stream);
        cudaFree(v->mlp_w);
        v->mlp_w = nullptr;
        return TSDF_OK;
    }
    if (n != kMlpParams) return TSDF_ERR_INVALID_ARG;
    cudaError_t e = cudaSuccess;
    if (!v->mlp_w) e = cudaMalloc(&v->mlp_w, kMlpParams * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMemcpy(v->mlp_w, bf16_weights, kMlpParams * sizeof(uint16_t), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? TSDF_OK : TSDF_ERR_CUDA;
}

tsdf_status tsdf_mlp_variance(const tsdf_volume* v, const uint16_t* w, const float* depth, const tsdf_intrinsics* K,
                              float* var_out, void* stream) {
    if (!v || !tsdf::ok_ptr(w) || !depth || !var_out || !tsdf::intrinsics_valid(K)) return TSDF_ERR_INVALID_ARG;
    const tsdf::FrameParams p = tsdf::frame_of(v, *K);
    const dim3 grid((unsigned)((p.width + 15) / 16), (unsigned)((p.height + 7) / 8));
    tsdf::variance_mlp_kernel<<<grid, 128, 0, (cudaStream_t)stream>>>(depth, p, (const __nv_bfloat16*)w, var_out);
    return cudaGetLastError() == cudaSuccess ? TSDF_OK : TSDF_ERR_CUDA;
}

tsdf_status tsdf_mlp_features(const tsdf_volume* v, const float* depth, const tsdf_intrinsics* K, int64_t n,
                              const int32_t* uv, float* feats, uint8_t* valid, void* stream) {
    if (!v || !depth || n < 0 || (n > 0 && (!uv || !feats)) || !tsdf::intrinsics_valid(K)) return TSDF_ERR_INVALID_ARG;
    if (n == 0) return TSDF_OK;
    const tsdf::FrameParams p = tsdf::frame_of(v, *K);
    const long long blocks = (n + 255) / 256;
    tsdf::features_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, (cudaStream_t)stream>>>(
        depth, p, n, uv, feats, valid);
    return cudaGetLastError() == cudaSuccess ? TSDF_OK : TSDF_ERR_CUDA;
}

tsdf_status tsdf_mlp_harvest(const tsdf_volume* v, const float* depth, const float* pred_depth,
                             const tsdf_intrinsics* K, int64_t max_n, float* feats, float* s, uint32_t* count,
                             void* stream) {
    if (!v || !depth || !pred_depth || max_n < 0 || !feats || !s || !count || !tsdf::intrinsics_valid(K))
        return TSDF_ERR_INVALID_ARG;
    const tsdf::FrameParams p = tsdf::frame_of(v, *K);
    tsdf::harvest_kernel<<<v->num_sms * 4, 256, 0, (cudaStream_t)stream>>>(depth, pred_depth, p, max_n, feats, s,
                                                                         count);
    return cudaGetLastError() == cudaSuccess ? TSDF_OK : TSDF_ERR_CUDA;
}

tsdf_status tsdf_mlp_forward(const uint16_t* w, int64_t n, const float* feats, float* out, void* stream) {
    if (!w || n < 0 || (n > 0 && (!feats || !out))) return TSDF_ERR_INVALID_ARG;
    if (n == 0) return TSDF_OK;
    const long long blocks = (n + 127) / 128;
    tsdf::forward_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 128, 0, (cudaStream_t)stream>>>(
        (const __nv_bfloat16*)w, n, feats, out);
    return cudaGetLastError() == cudaSuccess ? TSDF_OK : TSDF_ERR_CUDA;
}

tsdf_status tsdf_mlp_loss_grad(const uint16_t* w, int64_t n, const int32_t* idx, const float* feats, const float* s,
                               float* grad, float* loss, void* stream) {
    if (!w || n < 0 || !feats || !s || !grad || !loss) return TSDF_ERR_INVALID_ARG;
    if (n == 0) return TSDF_OK;
    long long ctas = (n + 63) / 64;            // 8 warps x 8 samples per CTA
    if (ctas > 296) ctas = 296;
    tsdf::mlp_grad_kernel<<<(unsigned)ctas, 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)w, n, idx, feats,
                                                                            s, grad, loss);
    return cudaGetLastError() == cudaSuccess ? TSDF_OK : TSDF_ERR_CUDA;
}

tsdf_status tsdf_mlp_adam(float* w32, uint16_t* wbf16, float* m, float* v, float* grad, float lr, float beta1,
                          float beta2, float eps, float grad_scale, int32_t step, void* stream) {
    if (!w32 || !wbf16 || !m || !v || !grad || step < 1) return TSDF_ERR_INVALID_ARG;
    const float bc1 = (float)(1.0 - std::pow((double)beta1, step));
    const float bc2 = (float)(1.0 - std::pow((double)beta2, step));
    tsdf::mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        w32, (__nv_bfloat16*)wbf16, m, v, grad, lr, beta1, beta2, eps, grad_scale, bc1, bc2);
    return cudaGetLastError() == cudaSuccess ? TSDF_OK : TSDF_ERR_CUDA;
}

}  // extern "C"
