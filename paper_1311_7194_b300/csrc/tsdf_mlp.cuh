// Inference of the learned measurement-variance network (a 27-32-32-1
// perceptron with ReLU and bfloat16 weights; see tsdf_mlp.cu): weight staging
// in shared memory, the per-pixel features, the forward pass and the variance
// it gives. Shared by the network's own kernels and by the integrate stage,
// which evaluates it where it forms each pixel's measurement
// (depth_tiles_mlp_kernel, with the same operations as mlp_eval).
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

// The inference layout: W1 and W2 transposed ([input][neuron], rows of 32
// floats, 16-byte aligned), so one vector load from shared memory gives four
// neurons' weights of the same input (a broadcast: every lane reads the same
// address) and two paired multiply-adds consume them. kInferFloats floats.
constexpr int kOffW2t = kHid * kIn + kHid, kOffB2t = kOffW2t + kHid * kHid;
constexpr int kInferFloats = kOffB2t + 2 * kHid + 1;
static_assert(kHid % 4 == 0 && (kHid * kIn) % 4 == 0 && kOffW2t % 4 == 0, "16-byte aligned rows");

struct MlpInfer {
    const float* W1t;   // [27][32]
    const float* b1;
    const float* W2t;   // [32][32]
    const float* b2;
    const float* W3;
    float b3;
};

// smem: kInferFloats floats, 16-byte aligned.
__device__ __forceinline__ MlpInfer load_infer(const __nv_bfloat16* __restrict__ w, float* smem) {
    for (int e = threadIdx.x; e < kHid * kIn; e += blockDim.x)
        smem[(e % kIn) * kHid + e / kIn] = __bfloat162float(w[e]);              // W1[j][i] -> W1t[i][j]
    for (int j = threadIdx.x; j < kHid; j += blockDim.x) smem[kHid * kIn + j] = __bfloat162float(w[kOffB1 + j]);
    for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x)
        smem[kOffW2t + (e % kHid) * kHid + e / kHid] = __bfloat162float(w[kOffW2 + e]);   // W2[j][i] -> W2t[i][j]
    for (int i = threadIdx.x; i < 2 * kHid + 1; i += blockDim.x) smem[kOffB2t + i] = __bfloat162float(w[kOffB2 + i]);
    __syncthreads();
    MlpInfer m;
    m.W1t = smem;
    m.b1 = smem + kHid * kIn;
    m.W2t = smem + kOffW2t;
    m.b2 = smem + kOffB2t;
    m.W3 = smem + kOffB2t + kHid;
    m.b3 = smem[kOffB2t + 2 * kHid];
    return m;
}

// Features of pixel (u, v); false when its depth is not a valid measurement.
// D(x, y, &d) reads the depth at pixel (x, y) into d and tells whether it is
// a valid measurement (false outside the image).
template <class DepthAt>
__device__ __forceinline__ bool features_from(DepthAt D, const FrameParams& p, int u, int v, float f[kIn]) {
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

__device__ __forceinline__ bool pixel_features(const float* __restrict__ depth, const FrameParams& p, int u, int v,
                                               float f[kIn]) {
    auto D = [&](int x, int y, float* d) {
        if (x < 0 || y < 0 || x >= p.width || y >= p.height) return false;
        *d = __ldg(depth + (size_t)y * p.width + x);
        return depth_ok(*d, p.depth_min, p.depth_max);
    };
    return features_from(D, p, u, v, f);
}

// The network's output for features f. Each neuron's sum runs over its inputs
// in order, one fused multiply-add each (two neurons per paired instruction,
// which rounds both as the scalar one), and the output sums the neurons in
// order: the same operations as a plain loop over the row-major weights.
__device__ __forceinline__ float mlp_eval(const MlpInfer& m, const float f[kIn]) {
    // the weights stay in shared memory: without this barrier the compiler
    // treats their loads as invariant across the caller's pixel loop, hoists
    // all of them and spills them to local memory
    asm volatile("" ::: "memory");
    float2 acc[kHid / 2];
#pragma unroll
    for (int j = 0; j < kHid / 2; ++j) acc[j] = make_float2(m.b1[2 * j], m.b1[2 * j + 1]);
#pragma unroll
    for (int i = 0; i < kIn; ++i) {
        const float2 x = make_float2(f[i], f[i]);
        const float4* w = reinterpret_cast<const float4*>(m.W1t + i * kHid);
#pragma unroll
        for (int q = 0; q < kHid / 4; ++q) {
            const float4 w4 = w[q];
            acc[2 * q] = __ffma2_rn(make_float2(w4.x, w4.y), x, acc[2 * q]);
            acc[2 * q + 1] = __ffma2_rn(make_float2(w4.z, w4.w), x, acc[2 * q + 1]);
        }
    }
    float a1[kHid];
#pragma unroll
    for (int j = 0; j < kHid / 2; ++j) {
        a1[2 * j] = fmaxf(acc[j].x, 0.0f);
        a1[2 * j + 1] = fmaxf(acc[j].y, 0.0f);
    }
    // the second layer in two halves of 16 neurons (registers)
    float out = m.b3;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float2 acc2[kHid / 4];
#pragma unroll
        for (int j = 0; j < kHid / 4; ++j) acc2[j] = make_float2(m.b2[h * kHid / 2 + 2 * j], m.b2[h * kHid / 2 + 2 * j + 1]);
#pragma unroll
        for (int i = 0; i < kHid; ++i) {
            const float2 x = make_float2(a1[i], a1[i]);
            const float4* w = reinterpret_cast<const float4*>(m.W2t + i * kHid + h * kHid / 2);
#pragma unroll
            for (int q = 0; q < kHid / 8; ++q) {
                const float4 w4 = w[q];
                acc2[2 * q] = __ffma2_rn(make_float2(w4.x, w4.y), x, acc2[2 * q]);
                acc2[2 * q + 1] = __ffma2_rn(make_float2(w4.z, w4.w), x, acc2[2 * q + 1]);
            }
        }
#pragma unroll
        for (int j = 0; j < kHid / 4; ++j) {
            out = fmaf(m.W3[h * kHid / 2 + 2 * j], fmaxf(acc2[j].x, 0.0f), out);
            out = fmaf(m.W3[h * kHid / 2 + 2 * j + 1], fmaxf(acc2[j].y, 0.0f), out);
        }
    }
    return out;
}

// p_k of pixel (u, v) under the network: p_quad exp(out), or p_quad when out
// lies outside [-ln 4, ln 64] or is not finite (a measurement may be up to 64
// times noisier than the quadratic model says - a sensor far poorer at depth
// edges - or 4 times less noisy); 0 (no measurement) when the pixel's depth is
// not a valid measurement.
__device__ __forceinline__ float learned_variance(const MlpInfer& m, const float* __restrict__ depth,
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
