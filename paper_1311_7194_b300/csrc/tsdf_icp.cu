// Point-to-plane registration of a depth frame to the raycast model maps
// (section "Registration", Eqs. 2-8).
//
//   icp_reduce_kernel: one thread per pixel (grid-stride): back-project the
//                      frame pixel, its normal from the central differences of
//                      its back-projected neighbours, move both into the world
//                      with the current pose estimate, match the point to the
//                      model pixel nearest its projection into the model camera,
//                      reject by distance and normal deviation, and accumulate
//                      the Eq. 4 sums (J J^T, J r with J = (p x n, n), r =
//                      (p - q).n), sum r^2, the count and the box of the
//                      matched points; lanes in float, a CTA's warps in
//                      double.
//   icp_final_kernel:  the CTAs' partial sums in a fixed order, in double.
// The paper does matching, rejection and the first reduction level in one
// kernel and the further levels in another; so does this file. The 6x6 solve
// runs on the host in double: the sums are restated in the box of the matched
// points shrunk to the unit cube (Eqs. 5-7), the system's eigenvectors with
// eigenvalue / pairs <= theta are dropped (Eq. 8), and the motion is applied
// to the pose.
//
// Scaling: with c^ = S^-1 (c - m x n), the residual (p - q).n + r.c + t.n
// becomes (p - q).n + (S r).c^ + (t + r x m).n, so the scaled system is solved
// for r^ = S r and t^ = t + r x m and the motion recovered as r = S^-1 r^,
// t = t^ - r x m. The scaled sums follow from the plain ones (M = [m]x):
//   sum c^ c^T = S^-1 (Acc - Acn M^T - M Acn^T + M Ann M^T) S^-1
//   sum c^ n^T = S^-1 (Acn - M Ann),  sum c^ r = S^-1 (bc - M bn),
// so one pass over the pixels suffices although m and S come from that pass.
#include <cmath>
#include <cstring>

#include "tsdf_internal.cuh"

namespace tsdf {
namespace {

constexpr int kIcpThreads = 256;
constexpr int kSums = 29;     // 21 of J J^T (upper triangle, row major), 6 of J r, sum r^2, count

struct IcpFrame {
    float fx, fy, cx, cy;
    int width, height;
    float R[9], t[3];          // current pose estimate, camera -> world
    float Rm[9], tm[3];        // model camera -> world
    float dist_max, cos_min, depth_min, depth_max;
};

__device__ __forceinline__ bool depth_valid(float d, const IcpFrame& f) {
    return isfinite(d) && d > 0.0f && d >= f.depth_min && d <= f.depth_max;
}

__device__ __forceinline__ void backproject(const IcpFrame& f, int u, int v, float d, float X[3]) {
    X[0] = ((float)u - f.cx) / f.fx * d;
    X[1] = ((float)v - f.cy) / f.fy * d;
    X[2] = d;
}

// The contribution of pixel (u, v), or false when it has no accepted pair.
__device__ __forceinline__ bool pixel_pair(const IcpFrame& f, const float* __restrict__ depth,
                                           const float* __restrict__ mv, const float* __restrict__ mn, int u, int v,
                                           float p[3], float q[3], float n[3]) {
    if (u < 1 || v < 1 || u >= f.width - 1 || v >= f.height - 1) return false;
    const int i = v * f.width + u;
    const float d = __ldg(depth + i);
    const float dl = __ldg(depth + i - 1), dr = __ldg(depth + i + 1);
    const float du = __ldg(depth + i - f.width), dd = __ldg(depth + i + f.width);
    if (!(depth_valid(d, f) && depth_valid(dl, f) && depth_valid(dr, f) && depth_valid(du, f) && depth_valid(dd, f)))
        return false;
    float X[3], Xl[3], Xr[3], Xu[3], Xd[3];
    backproject(f, u, v, d, X);
    backproject(f, u - 1, v, dl, Xl);
    backproject(f, u + 1, v, dr, Xr);
    backproject(f, u, v - 1, du, Xu);
    backproject(f, u, v + 1, dd, Xd);
    const float ax = Xr[0] - Xl[0], ay = Xr[1] - Xl[1], az = Xr[2] - Xl[2];
    const float bx = Xd[0] - Xu[0], by = Xd[1] - Xu[1], bz = Xd[2] - Xu[2];
    float ns[3] = {ay * bz - az * by, az * bx - ax * bz, ax * by - ay * bx};
    const float nn = sqrtf(ns[0] * ns[0] + ns[1] * ns[1] + ns[2] * ns[2]);
    if (!(nn > 0.0f)) return false;
    const float sg = (ns[0] * X[0] + ns[1] * X[1] + ns[2] * X[2]) > 0.0f ? -1.0f / nn : 1.0f / nn;
    for (int k = 0; k < 3; ++k) ns[k] *= sg;
    float nw[3];
    for (int r = 0; r < 3; ++r) {
        p[r] = f.R[3 * r] * X[0] + f.R[3 * r + 1] * X[1] + f.R[3 * r + 2] * X[2] + f.t[r];
        nw[r] = f.R[3 * r] * ns[0] + f.R[3 * r + 1] * ns[1] + f.R[3 * r + 2] * ns[2];
    }
    // into the model camera: R_m^T (p - t_m)
    const float ex = p[0] - f.tm[0], ey = p[1] - f.tm[1], ez = p[2] - f.tm[2];
    const float xm = f.Rm[0] * ex + f.Rm[3] * ey + f.Rm[6] * ez;
    const float ym = f.Rm[1] * ex + f.Rm[4] * ey + f.Rm[7] * ez;
    const float zm = f.Rm[2] * ex + f.Rm[5] * ey + f.Rm[8] * ez;
    if (!(zm > 0.0f)) return false;
    const float uf = floorf(f.fx * xm / zm + f.cx + 0.5f), vf = floorf(f.fy * ym / zm + f.cy + 0.5f);
    if (!(uf >= 0.0f && uf < (float)f.width && vf >= 0.0f && vf < (float)f.height)) return false;
    const int j = 3 * ((int)vf * f.width + (int)uf);
    for (int k = 0; k < 3; ++k) {
        q[k] = __ldg(mv + j + k);
        n[k] = __ldg(mn + j + k);
    }
    if (!(isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]) && isfinite(n[0]) && isfinite(n[1]) && isfinite(n[2])))
        return false;
    const float dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
    if (!(dx * dx + dy * dy + dz * dz <= f.dist_max * f.dist_max)) return false;
    return nw[0] * n[0] + nw[1] * n[1] + nw[2] * n[2] >= f.cos_min;
}

__device__ __forceinline__ double warp_sum_d(double x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__global__ void __launch_bounds__(kIcpThreads) icp_reduce_kernel(IcpFrame f, const float* __restrict__ depth,
                                                                 const float* __restrict__ mv,
                                                                 const float* __restrict__ mn,
                                                                 double* __restrict__ part, float* __restrict__ pbox) {
    __shared__ double ssum[kIcpThreads / 32][kSums];
    __shared__ float sbox[kIcpThreads / 32][6];
    float acc[kSums];
#pragma unroll
    for (int k = 0; k < kSums; ++k) acc[k] = 0.0f;
    float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
    const long long n_pix = (long long)f.width * f.height;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_pix;
         i += (long long)gridDim.x * blockDim.x) {
        float p[3], q[3], n[3];
        if (!pixel_pair(f, depth, mv, mn, (int)(i % f.width), (int)(i / f.width), p, q, n)) continue;
        const float J[6] = {p[1] * n[2] - p[2] * n[1], p[2] * n[0] - p[0] * n[2], p[0] * n[1] - p[1] * n[0],
                            n[0], n[1], n[2]};
        const float r = (p[0] - q[0]) * n[0] + (p[1] - q[1]) * n[1] + (p[2] - q[2]) * n[2];
        int k = 0;
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = a; b < 6; ++b) acc[k++] += J[a] * J[b];
#pragma unroll
        for (int a = 0; a < 6; ++a) acc[21 + a] += J[a] * r;
        acc[27] += r * r;
        acc[28] += 1.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], fminf(p[a], q[a]));
            hi[a] = fmaxf(hi[a], fmaxf(p[a], q[a]));
        }
    }
    // FP64 arithmetic is scarce on this GPU: the 32 lanes' sums are formed in
    // float (a few pixels each) and only the warps' sums are added in double
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kSums; ++k) {
        float s = acc[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) ssum[warp][k] = (double)s;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float l = lo[a], h = hi[a];
        for (int o = 16; o > 0; o >>= 1) {
            l = fminf(l, __shfl_xor_sync(0xffffffffu, l, o));
            h = fmaxf(h, __shfl_xor_sync(0xffffffffu, h, o));
        }
        if (lane == 0) {
            sbox[warp][a] = l;
            sbox[warp][3 + a] = h;
        }
    }
    __syncthreads();
    if (threadIdx.x < kSums) {
        double s = 0.0;
        for (int w = 0; w < kIcpThreads / 32; ++w) s += ssum[w][threadIdx.x];
        part[(size_t)blockIdx.x * kSums + threadIdx.x] = s;
    } else if (threadIdx.x >= 32 && threadIdx.x < 38) {
        const int a = threadIdx.x - 32;
        float b = a < 3 ? 3.0e38f : -3.0e38f;
        for (int w = 0; w < kIcpThreads / 32; ++w) b = a < 3 ? fminf(b, sbox[w][a]) : fmaxf(b, sbox[w][a]);
        pbox[(size_t)blockIdx.x * 6 + a] = b;
    }
}

// kSums + 1 CTAs: CTA k < kSums adds the CTAs' partial k (thread j taking CTAs
// j, j + 256, ..., then a fixed shuffle tree and the warps in order: the same
// order every run); the last CTA reduces the box.
__global__ void __launch_bounds__(kIcpThreads) icp_final_kernel(const double* __restrict__ part,
                                                                const float* __restrict__ pbox, int n_parts,
                                                                double* __restrict__ out, float* __restrict__ box) {
    __shared__ double sw[kIcpThreads / 32];
    __shared__ float sb[kIcpThreads / 32][6];
    const int k = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (k < kSums) {
        double s = 0.0;
        for (int b = threadIdx.x; b < n_parts; b += kIcpThreads) s += part[(size_t)b * kSums + k];
        s = warp_sum_d(s);
        if (lane == 0) sw[warp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kIcpThreads / 32; ++w) t += sw[w];
            out[k] = t;
        }
    } else {
        float v[6] = {3.0e38f, 3.0e38f, 3.0e38f, -3.0e38f, -3.0e38f, -3.0e38f};
        for (int b = threadIdx.x; b < n_parts; b += kIcpThreads)
            for (int a = 0; a < 6; ++a)
                v[a] = a < 3 ? fminf(v[a], pbox[(size_t)b * 6 + a]) : fmaxf(v[a], pbox[(size_t)b * 6 + a]);
        for (int a = 0; a < 6; ++a) {
            float x = v[a];
            for (int o = 16; o > 0; o >>= 1) {
                const float y = __shfl_xor_sync(0xffffffffu, x, o);
                x = a < 3 ? fminf(x, y) : fmaxf(x, y);
            }
            if (lane == 0) sb[warp][a] = x;
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            const int a = threadIdx.x;
            float x = sb[0][a];
            for (int w = 1; w < kIcpThreads / 32; ++w) x = a < 3 ? fminf(x, sb[w][a]) : fmaxf(x, sb[w][a]);
            box[a] = x;
        }
    }
}

// ---------------------------------------------------------------------------
// host side, double precision
// ---------------------------------------------------------------------------

// Eigen-decomposition of a symmetric 6x6 matrix by cyclic Jacobi rotations
// (Golub & Van Loan, "Matrix Computations", symmetric Jacobi method): on return
// lam holds the eigenvalues and the columns of V the eigenvectors.
void jacobi6(const double A_in[36], double lam[6], double V[36]) {
    double A[36];
    std::memcpy(A, A_in, sizeof(A));
    for (int i = 0; i < 36; ++i) V[i] = (i % 7 == 0) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                tot += A[6 * i + j] * A[6 * i + j];
                if (i != j) off += A[6 * i + j] * A[6 * i + j];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < 5; ++p)
            for (int q = p + 1; q < 6; ++q) {
                const double apq = A[6 * p + q];
                if (apq == 0.0) continue;
                const double theta = (A[6 * q + q] - A[6 * p + p]) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 6; ++k) {      // A <- A J (columns p, q)
                    const double akp = A[6 * k + p], akq = A[6 * k + q];
                    A[6 * k + p] = c * akp - s * akq;
                    A[6 * k + q] = s * akp + c * akq;
                }
                for (int k = 0; k < 6; ++k) {      // A <- J^T A (rows p, q)
                    const double apk = A[6 * p + k], aqk = A[6 * q + k];
                    A[6 * p + k] = c * apk - s * aqk;
                    A[6 * q + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 6; ++k) {      // V <- V J
                    const double vkp = V[6 * k + p], vkq = V[6 * k + q];
                    V[6 * k + p] = c * vkp - s * vkq;
                    V[6 * k + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < 6; ++i) lam[i] = A[7 * i];
}

void cross3(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// exp([r]x) by Rodrigues' formula, row major.
void rotation(const double r[3], double R[9]) {
    const double a = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0) ? 1.0 : 0.0;
    if (a < 1e-300) return;
    const double k[3] = {r[0] / a, r[1] / a, r[2] / a};
    const double K[9] = {0, -k[2], k[1], k[2], 0, -k[0], -k[1], k[0], 0};
    double K2[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int l = 0; l < 3; ++l) s += K[3 * i + l] * K[3 * l + j];
            K2[3 * i + j] = s;
        }
    const double sa = std::sin(a), ca = 1.0 - std::cos(a);
    for (int i = 0; i < 9; ++i) R[i] += sa * K[i] + ca * K2[i];
}

// The motion (r, t) of one iteration from the plain sums, the box, theta.
// Returns the number of eigen-directions kept.
int solve_motion(const double* s, const float* box, double theta, double r_out[3], double t_out[3]) {
    double A[36];
    int k = 0;
    for (int a = 0; a < 6; ++a)
        for (int b = a; b < 6; ++b) {
            A[6 * a + b] = s[k];
            A[6 * b + a] = s[k];
            ++k;
        }
    const double bc[3] = {s[21], s[22], s[23]}, bn[3] = {s[24], s[25], s[26]};
    const double N = s[28];
    double m[3], S[3];
    for (int a = 0; a < 3; ++a) {
        m[a] = 0.5 * ((double)box[a] + (double)box[3 + a]);
        S[a] = std::fmax((double)box[3 + a] - (double)box[a], 1e-9);
    }
    const double M[9] = {0, -m[2], m[1], m[2], 0, -m[0], -m[1], m[0], 0};   // M n = m x n
    double Acc[9], Acn[9], Ann[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            Acc[3 * i + j] = A[6 * i + j];
            Acn[3 * i + j] = A[6 * i + 3 + j];
            Ann[3 * i + j] = A[6 * (3 + i) + 3 + j];
        }
    auto mul = [](const double* X, const double* Y, double* Z, bool yt) {   // Z = X Y or X Y^T
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double v = 0.0;
                for (int l = 0; l < 3; ++l) v += X[3 * i + l] * (yt ? Y[3 * j + l] : Y[3 * l + j]);
                Z[3 * i + j] = v;
            }
    };
    double AcnMt[9], MAcnT[9], MAnn[9], MAnnMt[9], AcnT[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) AcnT[3 * i + j] = Acn[3 * j + i];
    mul(Acn, M, AcnMt, true);
    mul(M, AcnT, MAcnT, false);
    mul(M, Ann, MAnn, false);
    mul(MAnn, M, MAnnMt, true);
    double C[36], b[6];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const double cc = (Acc[3 * i + j] - AcnMt[3 * i + j] - MAcnT[3 * i + j] + MAnnMt[3 * i + j]) / (S[i] * S[j]);
            const double cn = (Acn[3 * i + j] - MAnn[3 * i + j]) / S[i];
            C[6 * i + j] = cc;
            C[6 * i + 3 + j] = cn;
            C[6 * (3 + j) + i] = cn;
            C[6 * (3 + i) + 3 + j] = Ann[3 * i + j];
        }
    for (int i = 0; i < 3; ++i) {
        double mb = 0.0;
        for (int l = 0; l < 3; ++l) mb += M[3 * i + l] * bn[l];
        b[i] = -(bc[i] - mb) / S[i];
        b[3 + i] = -bn[i];
    }
    double lam[6], V[36];
    jacobi6(C, lam, V);
    double x[6] = {0, 0, 0, 0, 0, 0};
    int rank = 0;
    for (int e = 0; e < 6; ++e) {
        if (!(lam[e] / std::fmax(N, 1.0) > theta)) continue;
        ++rank;
        double vb = 0.0;
        for (int i = 0; i < 6; ++i) vb += V[6 * i + e] * b[i];
        for (int i = 0; i < 6; ++i) x[i] += V[6 * i + e] * vb / lam[e];
    }
    for (int a = 0; a < 3; ++a) r_out[a] = x[a] / S[a];
    double rxm[3];
    cross3(r_out, m, rxm);
    for (int a = 0; a < 3; ++a) t_out[a] = x[3 + a] - rxm[a];
    return rank;
}

}  // namespace

cudaError_t launch_icp_sums(tsdf_volume* v, const float* depth, const tsdf_intrinsics& K, const double pose[16],
                            const float* mv, const float* mn, const double model_pose[16], const tsdf_icp_params& prm,
                            double* host_sums, float* host_box, cudaStream_t st) {
    IcpFrame f;
    f.fx = K.fx; f.fy = K.fy; f.cx = K.cx; f.cy = K.cy;
    f.width = K.width; f.height = K.height;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            f.R[3 * r + c] = (float)pose[4 * r + c];
            f.Rm[3 * r + c] = (float)model_pose[4 * r + c];
        }
        f.t[r] = (float)pose[4 * r + 3];
        f.tm[r] = (float)model_pose[4 * r + 3];
    }
    f.dist_max = prm.dist_max;
    f.cos_min = prm.normal_cos_min;
    f.depth_min = v->cfg.depth_min;
    f.depth_max = v->cfg.depth_max;
    // one wave: exactly the CTAs that can be resident at once (the kernel's
    // registers fit 3 CTAs of 256 threads on an SM; a grid of 4 per SM ran
    // its last quarter as a second wave)
    static int per_sm = 0;
    if (per_sm == 0 &&
        (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, icp_reduce_kernel, kIcpThreads, 0) != cudaSuccess ||
         per_sm < 1))
        per_sm = 1;
    const int grid = v->num_sms * per_sm;
    if (!v->icp_part) {
        cudaError_t e = cudaMalloc(&v->icp_part, (size_t)grid * (kSums + 3) * sizeof(double) + 64 * sizeof(double));
        if (e != cudaSuccess) return e;
    }
    // the sums and the box lie next to each other on the device (kSums doubles,
    // one spare, then 6 floats): one copy into pinned memory reads both
    constexpr size_t kOutWords = kSums + 4;
    if (!v->icp_host) {
        cudaError_t e = cudaMallocHost(&v->icp_host, kOutWords * sizeof(double));
        if (e != cudaSuccess) {
            v->icp_host = nullptr;
            return e;
        }
    }
    double* part = v->icp_part;
    float* pbox = reinterpret_cast<float*>(part + (size_t)grid * kSums);          // grid * 6 floats
    double* out = part + (size_t)grid * (kSums + 3);                              // kSums doubles
    float* box = reinterpret_cast<float*>(out + kSums + 1);                       // 6 floats
    icp_reduce_kernel<<<grid, kIcpThreads, 0, st>>>(f, depth, mv, mn, part, pbox);
    icp_final_kernel<<<kSums + 1, kIcpThreads, 0, st>>>(part, pbox, grid, out, box);
    cudaError_t e = cudaMemcpyAsync(v->icp_host, out, kOutWords * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
        std::memcpy(host_sums, v->icp_host, kSums * sizeof(double));
        std::memcpy(host_box, v->icp_host + kSums + 1, 6 * sizeof(float));
    }
    return e == cudaSuccess ? cudaGetLastError() : e;
}

int icp_solve(const double* sums, const float* box, double theta, double r[3], double t[3]) {
    return solve_motion(sums, box, theta, r, t);
}

void icp_apply(const double r[3], const double t[3], double pose[16]) {
    double R[9];
    rotation(r, R);
    double out[16];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 4; ++j) {
            double s = 0.0;
            for (int l = 0; l < 3; ++l) s += R[3 * i + l] * pose[4 * l + j];
            out[4 * i + j] = s + (j == 3 ? t[i] : 0.0);
        }
    }
    for (int j = 0; j < 4; ++j) out[12 + j] = pose[12 + j];
    std::memcpy(pose, out, sizeof(out));
}

}  // namespace tsdf
