// Storage formats of the distance T (the paper keeps T in 8 bits and sizes its
// memory study at 2 bytes per voxel; section "Volumetric Scene Representation",
// Fig. 6 caption). The variance P always stays float32 and all arithmetic is
// float32: a format only changes how T is held between launches.
//   F32:     float, chi = NaN.
//   F16:     IEEE half, round to nearest even, chi = NaN.
//   SNORM16: int16 q = rint(T * (32767 / delta)) in [-32767, 32767],
//            chi = -32768; T = q * (delta / 32767) (both scales rounded once
//            to float from double).
// decode() turns chi into NaN in every format, so chi propagates through sums
// (a trilinear sample with a chi corner is NaN) exactly as with float storage.
#pragma once

#include <cuda_fp16.h>

#include "tsdf.h"

namespace tsdf {

template <int S>
struct Codec;

template <>
struct Codec<TSDF_STORAGE_F32> {
    using E = float;
    static constexpr int kBytes = 4;
    __device__ static float load(const E* p, float2) { return __ldg(p); }
    __device__ static void load4(const E* p, float v[4], float2) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    __device__ static void store4(E* p, const float v[4], float2) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};

template <>
struct Codec<TSDF_STORAGE_F16> {
    using E = __half;
    static constexpr int kBytes = 2;
    __device__ static float load(const E* p, float2) { return __half2float(__ldg(p)); }
    __device__ static void load4(const E* p, float v[4], float2) {
        const uint2 t = *reinterpret_cast<const uint2*>(p);
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&t.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&t.y));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    __device__ static void store4(E* p, const float v[4], float2) {
        const __half2 a = __floats2half2_rn(v[0], v[1]);
        const __half2 b = __floats2half2_rn(v[2], v[3]);
        uint2 t;
        t.x = *reinterpret_cast<const unsigned int*>(&a);
        t.y = *reinterpret_cast<const unsigned int*>(&b);
        *reinterpret_cast<uint2*>(p) = t;
    }
};

template <>
struct Codec<TSDF_STORAGE_SNORM16> {
    using E = short;
    static constexpr int kBytes = 2;
    // sc.x = delta / 32767 decodes, sc.y = 32767 / delta encodes
    __device__ static float decode(short q, float2 sc) {
        return q == (short)-32768 ? __int_as_float(0x7fc00000) : (float)q * sc.x;
    }
    __device__ static short encode(float f, float2 sc) {
        if (isnan(f)) return (short)-32768;
        const float q = rintf(__fmul_rn(f, sc.y));
        return (short)fminf(fmaxf(q, -32767.0f), 32767.0f);
    }
    __device__ static float load(const E* p, float2 sc) { return decode(__ldg(p), sc); }
    __device__ static void load4(const E* p, float v[4], float2 sc) {
        const short4 t = *reinterpret_cast<const short4*>(p);
        v[0] = decode(t.x, sc); v[1] = decode(t.y, sc); v[2] = decode(t.z, sc); v[3] = decode(t.w, sc);
    }
    __device__ static void store4(E* p, const float v[4], float2 sc) {
        *reinterpret_cast<short4*>(p) =
            make_short4(encode(v[0], sc), encode(v[1], sc), encode(v[2], sc), encode(v[3], sc));
    }
};

inline int storage_bytes(int storage) { return storage == TSDF_STORAGE_F32 ? 4 : 2; }

}  // namespace tsdf
