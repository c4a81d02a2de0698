// Inference of the learned measurement-variance network (a 27-32-32-1
// perceptron with ReLU and bfloat16 weights; see tsdf_mlp.cu): weight staging
// in shared memory, the per-pixel features, the forward pass and the variance
// it gives. Shared by the network's own kernels and by the integrate stage,
// which evaluates it where it forms each pixel's measurement (depth_tiles).
#pragma once

#include <cuda_bf16.h>

#include "tsdf_internal.cuh"

namespace tsdf {

constexpr int kIn = 27, kHid = 32;
constexpr int kOffB1 = kHid * kIn, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid;
static_assert(kOffB3 + 1 == kMlpParams, "parameter layout");
constexpr int kW2Pitch = kHid + 1;      // padded rows of W2 in shared memory (no bank conflicts)
constexpr int kSmemFloats = kOffW2 + kHid * kW2Pitch + kHid + kHid + 1;

struct MlpShared {
    float* W1;   // [32][27]
    float* b1;
    float* W2;   // [32][33]
    float* b2;
    float* W3;
    float b3;
};

__device__ __forceinline__ MlpShared load_weights(const __nv_bfloat16* __restrict__ w, float* smem) {
    for (int i = threadIdx.x; i < kOffW2; i += blockDim.x) smem[i] = __bfloat162float(w[i]);
    for (int i = threadIdx.x; i < kHid * kHid; i += blockDim.x)
        smem[kOffW2 + (i / kHid) * kW2Pitch + i % kHid] = __bfloat162float(w[kOffW2 + i]);
    float* tail = smem + kOffW2 + kHid * kW2Pitch;
    for (int i = threadIdx.x; i < 2 * kHid + 1; i += blockDim.x) tail[i] = __bfloat162float(w[kOffB2 + i]);
    __syncthreads();
    MlpShared m;
    m.W1 = smem;
    m.b1 = smem + kOffB1;
    m.W2 = smem + kOffW2;
    m.b2 = tail;
    m.W3 = tail + kHid;
    m.b3 = tail[2 * kHid];
    return m;
}

// Features of pixel (u, v); false when its depth is not a valid measurement.
__device__ __forceinline__ bool pixel_features(const float* __restrict__ depth, const FrameParams& p, int u, int v,
                                               float f[kIn]) {
    auto D = [&](int x, int y, float* d) {
        if (x < 0 || y < 0 || x >= p.width || y >= p.height) return false;
        *d = __ldg(depth + (size_t)y * p.width + x);
        return depth_ok(*d, p.depth_min, p.depth_max);
    };
    float d0;
    if (!D(u, v, &d0)) return false;
    const float inv_delta = 1.0f / p.delta;
    int i = 0;
#pragma unroll
    for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
        for (int dx = -2; dx <= 2; ++dx, ++i) {
            float d;
            f[i] = D(u + dx, v + dy, &d) ? fminf(1.0f, fmaxf(-1.0f, (d - d0) * inv_delta)) : 1.0f;
        }
    f[25] = d0 * 0.25f;
    f[26] = 0.0f;
    float dl, dr, du, dd;
    if (D(u - 1, v, &dl) && D(u + 1, v, &dr) && D(u, v - 1, &du) && D(u, v + 1, &dd)) {
        const float xn = ((float)u - p.cx) / p.fx, yn = ((float)v - p.cy) / p.fy;
        const float xl = ((float)(u - 1) - p.cx) / p.fx, xr = ((float)(u + 1) - p.cx) / p.fx;
        const float yu = ((float)(v - 1) - p.cy) / p.fy, yd = ((float)(v + 1) - p.cy) / p.fy;
        const float a0 = dr * xr - dl * xl, a1 = (dr - dl) * yn, a2 = dr - dl;          // P(u+1) - P(u-1)
        const float b0 = (dd - du) * xn, b1 = dd * yd - du * yu, b2 = dd - du;          // P(v+1) - P(v-1)
        const float n0 = a1 * b2 - a2 * b1, n1 = a2 * b0 - a0 * b2, n2 = a0 * b1 - a1 * b0;
        const float P0 = d0 * xn, P1 = d0 * yn, P2 = d0;
        const float ln = sqrtf(n0 * n0 + n1 * n1 + n2 * n2), lp = sqrtf(P0 * P0 + P1 * P1 + P2 * P2);
        if (ln > 0.0f && lp > 0.0f) f[26] = fabsf(n0 * P0 + n1 * P1 + n2 * P2) / (ln * lp);
    }
    return true;
}

__device__ __forceinline__ float mlp_eval(const MlpShared& m, const float f[kIn]) {
    float a1[kHid];
#pragma unroll
    for (int j = 0; j < kHid; ++j) {
        float acc = m.b1[j];
#pragma unroll
        for (int i = 0; i < kIn; ++i) acc = fmaf(m.W1[j * kIn + i], f[i], acc);
        a1[j] = fmaxf(acc, 0.0f);
    }
    float out = m.b3;
#pragma unroll
    for (int j = 0; j < kHid; ++j) {
        float acc = m.b2[j];
#pragma unroll
        for (int i = 0; i < kHid; ++i) acc = fmaf(m.W2[j * kW2Pitch + i], a1[i], acc);
        out = fmaf(m.W3[j], fmaxf(acc, 0.0f), out);
    }
    return out;
}

// p_k of pixel (u, v) under the network: p_quad exp(out), or p_quad when out
// lies outside [-ln 4, ln 64] or is not finite (a measurement may be up to 64
// times noisier than the quadratic model says - a sensor far poorer at depth
// edges - or 4 times less noisy); 0 (no measurement) when the pixel's depth is
// not a valid measurement.
__device__ __forceinline__ float learned_variance(const MlpShared& m, const float* __restrict__ depth,
                                                  const FrameParams& p, int u, int v) {
    float f[kIn];
    if (!pixel_features(depth, p, u, v, f)) return 0.0f;
    const float d = __ldg(depth + (size_t)v * p.width + u);
    const float sg = __fmul_rn(__fmul_rn(p.sigma_coeff, d), d);
    const float pq = __fmul_rn(sg, sg);
    const float out = mlp_eval(m, f);
    return (out >= -1.3862943611198906f && out <= 4.1588830833596715f) ? pq * expf(out) : pq;   // false for NaN
}

}  // namespace tsdf
