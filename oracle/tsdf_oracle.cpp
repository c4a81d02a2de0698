// CPU oracle for sparse TSDF fusion (Trifonov, "Real-time High Resolution Fusion of
// Depth Maps on GPU", arXiv 1311.7194).
//
// TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
// restatement of what the fusion hot path computes. It shares no code, header,
// table or constant with the CUDA library: it exists to check that library.
// Only the test suite, the package's smoke check and the benchmark's CPU-baseline
// leg load it; no product code path may call it.
//
// Arithmetic is IEEE double throughout (compiled with -ffp-contract=off), except
// the allocation sampling, where a floating-point computation decides an integer
// (a block coordinate): there both sides take the decision in single precision
// with the same sequence of correctly rounded operations, so block sets are
// comparable bit for bit.
//
// What each part follows:
//   * Eq. 1 (section "Volumetric Scene Representation"): T is the signed distance,
//     positive outside, replaced by the mark chi when |distance| > delta.
//   * Section "Updating Sparse Structure": the surface is sampled and the blocks
//     containing the samples are allocated; only those blocks (and blocks allocated
//     before) carry values.
//   * Section "Integration of Measurements", last paragraph: T_k(x) comes from
//     projecting x into the measured depth map; chi when there is no measurement.
//   * Alg. 3 (Kalman filter for TSDF estimation): predict P+Q, gain K, correct T,
//     shrink P, then chi if |T| > delta.
//   * Alg. 1 (scene TSDF estimation): T <- (1 - w_k) T + w_k T_k, chi if |T| > delta.
//   * Alg. 2 (weighted scene TSDF estimation): T <- (W T + w_k T_k) / (W + w_k),
//     W <- min(W + w_k, W_max), chi if |T| > delta; the weight W is kept where
//     Alg. 3 keeps P.
//   * Section "Integration of Measurements", last paragraph: optionally, T_k
//     refined by gradient (Gauss-Newton) steps in the depth map (refine_tk).
//   * Eq. 9: averaging N measurements of deviation sigma leaves variance sigma^2/N
//     (used by the tests as a closed-form pin).
//   * Section "Scene Rendering": the depth/normal map of the fused surface is found
//     by casting rays through the voxel field; here with a fine fixed-step march and
//     bisection, which is the exact first zero crossing that the GPU's coarse
//     march with refinement approximates.
//
// Readings where the paper is silent (camera model, pixel rounding, definition of
// T_k as a z-difference, sampling density of the allocation, raycast crossing rule)
// are stated at each function.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <unordered_map>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

// Volume settings. Lengths in metres. Values the CUDA library takes as float are
// float here too, and are widened exactly to double where the oracle computes.
struct ov_params {
    float voxel_size;           // s
    float truncation;           // delta (Eq. 1)
    double origin[3];           // world position of voxel (0,0,0)
    int32_t grid_dim;           // G voxels per axis (multiple of 8)
    int64_t block_capacity;     // pool size in blocks
    float process_variance;     // Q (Alg. 3)
    float depth_min, depth_max; // measured depth outside this range = no measurement
    float raycast_near, raycast_far;
    float sigma_coeff;          // sensor deviation a: sigma = a * D^2, p_k = sigma^2
    int32_t alloc_half_samples; // J; 0 = ceil(2 delta / s)
    double amb_px;              // pixel-rounding ambiguity margin, pixels
    double amb_trunc;           // truncation-test ambiguity margin, fraction of delta
    int32_t store_values;       // 0 = allocation bookkeeping only
    int32_t update_rule;        // 0 = Alg. 3 (Kalman), 1 = Alg. 1 (running average),
                                // 2 = Alg. 2 (weighted average with W_max)
    float update_weight;        // w_k of Alg. 1 / Alg. 2 (the same for every measurement)
    float weight_max;           // W_max of Alg. 2
    int32_t refine_steps;       // Gauss-Newton steps refining T_k in the depth map (0 = off)
};

struct ov_intr {
    float fx, fy, cx, cy;
    int32_t width, height;
};

}  // extern "C"

namespace {

constexpr int M = 8;             // voxels per block axis
constexpr int M3 = M * M * M;

struct Block {
    int32_t b[3];
    int32_t alloc_frame;
    std::vector<double> T, P;    // distance and variance per voxel
    std::vector<uint8_t> chi;    // 1 = chi (no isosurface nearby)
    std::vector<uint8_t> amb;    // 1 = an FP32 implementation may legitimately differ
};

struct Volume {
    ov_params p;
    int32_t nb;                                   // blocks per axis
    std::unordered_map<uint32_t, int32_t> index;  // block key -> position in blocks
    std::vector<Block> blocks;
};

uint32_t block_key(int64_t bx, int64_t by, int64_t bz, int32_t nb) {
    return (uint32_t)(bx + (int64_t)nb * (by + (int64_t)nb * bz));
}

// A measured depth is usable when it is a finite positive number within the
// sensor range (reading of "if no measurement is available ... chi").
bool depth_valid(float d, const ov_params& p) {
    return std::isfinite(d) && d > 0.0f && d >= p.depth_min && d <= p.depth_max;
}

// --------------------------------------------------------------------------
// Allocation (section "Updating Sparse Structure")
// --------------------------------------------------------------------------
// Reading of the sampling density: every valid pixel is sampled at 2J+1 depths
// spaced delta/J along its viewing ray, covering [D - delta, D + delta], with
// J = ceil(2 delta / s) so that consecutive samples are at most s/2 apart along z.
// Per-frame constants are computed in double and rounded once to float; the
// per-sample arithmetic is a fixed sequence of single-precision operations:
//   xn = (i - cx) / fx,  yn = (j - cy) / fy
//   b_r = fma(Mr0, xn, fma(Mr1, yn, Mr2))        with M = R / s
//   z_k = fma(k - J, delta/J, D)
//   q_r = fma(z_k, b_r, a_r)                       with a = (t - origin) / s
// q is the sample position in voxel units; the sample lies in the grid when
// 0 <= q_r < G, and its block is floor(q) / 8 (floor division).
struct AllocConsts {
    float Mr[3][3];
    float a[3];
    float dz;
    int J;
    float G;
};

AllocConsts alloc_consts(const ov_params& p, const double* pose) {
    AllocConsts c;
    const double s = (double)p.voxel_size;
    const double delta = (double)p.truncation;
    c.J = p.alloc_half_samples > 0 ? p.alloc_half_samples
                                   : (int)std::ceil(2.0 * delta / s - 1e-6);
    c.dz = (float)(delta / (double)c.J);
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) c.Mr[r][k] = (float)(pose[4 * r + k] / s);
        c.a[r] = (float)((pose[4 * r + 3] - p.origin[r]) / s);
    }
    c.G = (float)p.grid_dim;
    return c;
}

// The sorted, duplicate-free keys of every block a frame's surface samples touch.
std::vector<uint32_t> frame_blocks(const ov_params& p, const float* depth, const ov_intr& in,
                                   const double* pose) {
    const AllocConsts c = alloc_consts(p, pose);
    const int32_t nb = p.grid_dim / M;
    std::vector<uint32_t> keys;
#pragma omp parallel
    {
        std::vector<uint32_t> local;
#pragma omp for schedule(static)
        for (int j = 0; j < in.height; ++j) {
            for (int i = 0; i < in.width; ++i) {
                const float d = depth[(int64_t)j * in.width + i];
                if (!depth_valid(d, p)) continue;
                const float xn = ((float)i - in.cx) / in.fx;
                const float yn = ((float)j - in.cy) / in.fy;
                float b[3];
                for (int r = 0; r < 3; ++r)
                    b[r] = std::fmaf(c.Mr[r][0], xn, std::fmaf(c.Mr[r][1], yn, c.Mr[r][2]));
                for (int k = 0; k <= 2 * c.J; ++k) {
                    const float zk = std::fmaf((float)(k - c.J), c.dz, d);
                    float q[3];
                    bool inside = true;
                    for (int r = 0; r < 3; ++r) {
                        q[r] = std::fmaf(zk, b[r], c.a[r]);
                        inside = inside && (q[r] >= 0.0f) && (q[r] < c.G);
                    }
                    if (!inside) continue;
                    const int64_t vx = (int64_t)std::floor(q[0]);
                    const int64_t vy = (int64_t)std::floor(q[1]);
                    const int64_t vz = (int64_t)std::floor(q[2]);
                    local.push_back(block_key(vx / M, vy / M, vz / M, nb));
                }
            }
        }
#pragma omp critical
        keys.insert(keys.end(), local.begin(), local.end());
    }
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    return keys;
}

void key_to_block(uint32_t key, int32_t nb, int32_t b[3]) {
    b[0] = (int32_t)(key % (uint32_t)nb);
    b[1] = (int32_t)((key / (uint32_t)nb) % (uint32_t)nb);
    b[2] = (int32_t)(key / ((uint32_t)nb * (uint32_t)nb));
}

// New blocks join the pool in ascending key order; when the pool is full the
// remaining (highest-key) new blocks of the frame are not allocated.
void add_blocks(Volume& v, const std::vector<uint32_t>& keys, int32_t frame, int64_t* n_new,
                int32_t* overflow) {
    int64_t added = 0;
    int32_t over = 0;
    for (uint32_t key : keys) {
        if (v.index.count(key)) continue;
        if ((int64_t)v.blocks.size() >= v.p.block_capacity) {
            over = 1;
            continue;
        }
        Block blk;
        key_to_block(key, v.nb, blk.b);
        blk.alloc_frame = frame;
        if (v.p.store_values) {
            blk.T.assign(M3, 0.0);
            blk.P.assign(M3, 0.0);
            blk.chi.assign(M3, 1);   // a fresh block holds chi everywhere
            blk.amb.assign(M3, 0);
        }
        v.index.emplace(key, (int32_t)v.blocks.size());
        v.blocks.push_back(std::move(blk));
        ++added;
    }
    if (n_new) *n_new = added;
    if (overflow) *overflow = over;
}

// --------------------------------------------------------------------------
// Projective measurement T_k(x) (Fusion, last paragraph of "Integration of
// Measurements") and Alg. 3.
// --------------------------------------------------------------------------
// Readings: the voxel centre x = origin + i s is moved into the camera frame with
// the inverse pose, x_c = R^T (x - t); its pixel is the nearest one,
// u = floor(fx x_c/z_c + cx + 1/2), v likewise; T_k = D(u,v) - z_c, the signed
// distance along the optical axis, positive in front of the measured surface
// (outside, Eq. 1). T_k is chi when z_c <= 0, the pixel is outside the image, the
// depth is not a valid measurement, its variance is not a positive finite number,
// or |T_k| > delta. p_k is the given variance map, else (a D^2)^2.
struct Frame {
    const float* depth;
    const float* var;   // may be null
    ov_intr in;
    double R[3][3], t[3];
};

Frame make_frame(const float* depth, const float* var, const ov_intr& in, const double* pose) {
    Frame f;
    f.depth = depth;
    f.var = var;
    f.in = in;
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) f.R[r][k] = pose[4 * r + k];
        f.t[r] = pose[4 * r + 3];
    }
    return f;
}

struct Meas {
    bool valid;
    bool amb;     // a decision above was within rounding distance of its boundary
    double Tk, pk;
};

// Where x + 1/2 lies within `margin` of an integer, rounding x to the nearest
// integer could go either way under a few units of rounding error; returns the
// other candidate (or the same value when the decision is clear).
double other_rounding(double x, double margin) {
    const double u0 = std::floor(x + 0.5);
    const double r = x + 0.5 - u0;
    if (r < margin) return u0 - 1.0;
    if (1.0 - r < margin) return u0 + 1.0;
    return u0;
}

struct PixMeas {
    bool valid;
    bool trunc_amb;
    double Tk, pk;
};

PixMeas pixel_measure(const ov_params& p, const Frame& f, double u, double v, double z) {
    PixMeas m{false, false, 0.0, 0.0};
    if (u < 0.0 || v < 0.0 || u >= (double)f.in.width || v >= (double)f.in.height) return m;
    const int64_t pix = (int64_t)v * f.in.width + (int64_t)u;
    const float D = f.depth[pix];
    if (!depth_valid(D, p)) return m;
    const double Dd = (double)D;
    double pk;
    if (f.var) {
        pk = (double)f.var[pix];
    } else {
        const double sigma = (double)p.sigma_coeff * Dd * Dd;
        pk = sigma * sigma;
    }
    if (!(std::isfinite(pk) && pk > 0.0)) return m;
    const double Tk = Dd - z;
    const double delta = (double)p.truncation;
    m.trunc_amb = std::fabs(std::fabs(Tk) - delta) <= p.amb_trunc * delta;
    if (std::fabs(Tk) > delta) return m;
    m.valid = true;
    m.Tk = Tk;
    m.pk = pk;
    return m;
}

// Section "Integration of Measurements", last paragraph: a finer T_k by a few
// gradient steps in the depth map towards the local minimum of the distance
// between the measured surface and x. Reading: the measured surface is the
// depth map back-projected, S(u, v) = D~(u, v) ((u - cx)/fx, (v - cy)/fy, 1),
// with D~ the bilinear interpolation of the four pixels around (u, v); the
// steps are Gauss-Newton steps on |S(u, v) - X|^2 from the voxel's projection;
// an evaluation needs all four pixels valid and within delta of each other (no
// depth edge). T_k is the distance |S - X| at the last valid evaluation, signed
// by the side of S's tangent plane X lies on (positive on the camera side:
// outside, Eq. 1), or stays the z-difference when no evaluation is valid. *amb is set when an evaluation point lies within amb_px
// of a pixel-cell line, where float rounding could pick another cell.
struct SurfEval {
    bool ok;
    double S[3], Ju[3], Jv[3];
};

SurfEval surface_eval(const ov_params& p, const Frame& f, double u, double v) {
    SurfEval e{false, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    const double fi = std::floor(u), fj = std::floor(v);
    if (!(fi >= 0.0 && fj >= 0.0 && fi + 1.0 < (double)f.in.width && fj + 1.0 < (double)f.in.height)) return e;
    const int64_t i = (int64_t)fi, j = (int64_t)fj, W = f.in.width;
    const float d00 = f.depth[j * W + i], d10 = f.depth[j * W + i + 1];
    const float d01 = f.depth[(j + 1) * W + i], d11 = f.depth[(j + 1) * W + i + 1];
    if (!(depth_valid(d00, p) && depth_valid(d10, p) && depth_valid(d01, p) && depth_valid(d11, p))) return e;
    // the depth-edge test is a branch decided by float values: it is taken in
    // float32, as the library takes it
    const float lo32 = std::min(std::min(d00, d10), std::min(d01, d11));
    const float hi32 = std::max(std::max(d00, d10), std::max(d01, d11));
    if (hi32 - lo32 > p.truncation) return e;
    const double D00 = d00, D10 = d10, D01 = d01, D11 = d11;
    const double a = u - fi, b = v - fj;
    const double D = (1 - a) * (1 - b) * D00 + a * (1 - b) * D10 + (1 - a) * b * D01 + a * b * D11;
    const double Du = (1 - b) * (D10 - D00) + b * (D11 - D01);
    const double Dv = (1 - a) * (D01 - D00) + a * (D11 - D10);
    const double fx = f.in.fx, fy = f.in.fy;
    const double ray[3] = {(u - (double)f.in.cx) / fx, (v - (double)f.in.cy) / fy, 1.0};
    for (int k = 0; k < 3; ++k) {
        e.S[k] = D * ray[k];
        e.Ju[k] = Du * ray[k];
        e.Jv[k] = Dv * ray[k];
    }
    e.Ju[0] += D / fx;
    e.Jv[1] += D / fy;
    e.ok = true;
    return e;
}

bool near_cell_line(double x, double margin) {
    const double r = x - std::floor(x);
    return r < margin || 1.0 - r < margin;
}

double refine_tk(const ov_params& p, const Frame& f, const double X[3], double uf, double vf, double Tk0,
                 bool* amb) {
    double u = uf, v = vf, dist = -1.0, side = 1.0;
    for (int k = 0; k <= p.refine_steps; ++k) {
        if (near_cell_line(u, p.amb_px) || near_cell_line(v, p.amb_px)) *amb = true;
        const SurfEval e = surface_eval(p, f, u, v);
        if (!e.ok) break;
        const double r[3] = {e.S[0] - X[0], e.S[1] - X[1], e.S[2] - X[2]};
        dist = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        // tangent-plane normal Ju x Jv turned to the camera (at the origin)
        double n[3] = {e.Ju[1] * e.Jv[2] - e.Ju[2] * e.Jv[1], e.Ju[2] * e.Jv[0] - e.Ju[0] * e.Jv[2],
                       e.Ju[0] * e.Jv[1] - e.Ju[1] * e.Jv[0]};
        if (n[0] * e.S[0] + n[1] * e.S[1] + n[2] * e.S[2] > 0.0)
            for (double& c : n) c = -c;
        side = (-r[0] * n[0] - r[1] * n[1] - r[2] * n[2]) >= 0.0 ? 1.0 : -1.0;   // (X - S).n
        if (k == p.refine_steps) break;
        const double a11 = e.Ju[0] * e.Ju[0] + e.Ju[1] * e.Ju[1] + e.Ju[2] * e.Ju[2];
        const double a12 = e.Ju[0] * e.Jv[0] + e.Ju[1] * e.Jv[1] + e.Ju[2] * e.Jv[2];
        const double a22 = e.Jv[0] * e.Jv[0] + e.Jv[1] * e.Jv[1] + e.Jv[2] * e.Jv[2];
        const double g1 = e.Ju[0] * r[0] + e.Ju[1] * r[1] + e.Ju[2] * r[2];
        const double g2 = e.Jv[0] * r[0] + e.Jv[1] * r[1] + e.Jv[2] * r[2];
        const double det = a11 * a22 - a12 * a12;
        if (!(det > 0.0)) break;
        u -= (a22 * g1 - a12 * g2) / det;
        v -= (a11 * g2 - a12 * g1) / det;
    }
    if (dist < 0.0) return Tk0;
    return side * dist;
}

Meas measure(const ov_params& p, const Frame& f, int64_t ix, int64_t iy, int64_t iz) {
    Meas m{false, false, 0.0, 0.0};
    const double s = (double)p.voxel_size;
    const double x[3] = {p.origin[0] + (double)ix * s, p.origin[1] + (double)iy * s,
                         p.origin[2] + (double)iz * s};
    const double d[3] = {x[0] - f.t[0], x[1] - f.t[1], x[2] - f.t[2]};
    double xc[3];
    for (int k = 0; k < 3; ++k) xc[k] = f.R[0][k] * d[0] + f.R[1][k] * d[1] + f.R[2][k] * d[2];
    const double z = xc[2];
    if (!(z > 0.0)) {
        m.amb = std::fabs(z) < 1e-6;
        return m;
    }
    const double uf = (double)f.in.fx * xc[0] / z + (double)f.in.cx;
    const double vf = (double)f.in.fy * xc[1] / z + (double)f.in.cy;
    const double u0 = std::floor(uf + 0.5), v0 = std::floor(vf + 0.5);
    const PixMeas m0 = pixel_measure(p, f, u0, v0, z);
    m.valid = m0.valid;
    m.amb = m0.trunc_amb;
    m.Tk = m0.Tk;
    m.pk = m0.pk;
    // The nearest pixel is ambiguous within rounding error of a half-pixel line:
    // the voxel is flagged when another candidate pixel would measure differently.
    const double ua = other_rounding(uf, p.amb_px), va = other_rounding(vf, p.amb_px);
    const double cu[3] = {ua, u0, ua}, cv[3] = {v0, va, va};
    for (int c = 0; c < 3; ++c) {
        if (cu[c] == u0 && cv[c] == v0) continue;
        const PixMeas mc = pixel_measure(p, f, cu[c], cv[c], z);
        if (mc.valid != m0.valid || (m0.valid && (mc.Tk != m0.Tk || mc.pk != m0.pk)) ||
            mc.trunc_amb)
            m.amb = true;
    }
    if (m.valid && p.refine_steps > 0) {
        m.Tk = refine_tk(p, f, xc, uf, vf, m.Tk, &m.amb);
        // a refined T_k near +-delta makes the chi test after the update a close call
        const double delta = (double)p.truncation;
        if (std::fabs(std::fabs(m.Tk) - delta) <= p.amb_trunc * delta) m.amb = true;
    }
    return m;
}

// Alg. 3, one measurement into one voxel.
void kalman_update(double& T, double& P, uint8_t& chi, double Tk, double pk, double Q,
                   double delta) {
    if (chi) {
        T = Tk;
        P = pk;
        chi = 0;
    } else {
        P = P + Q;                    // predict
        const double K = P / (P + pk);
        T = T + K * (Tk - T);         // correct
        P = (1.0 - K) * P;
    }
    if (std::fabs(T) > delta) chi = 1;
}

// Alg. 1: a fixed-weight running average of the measurements. P is not used.
void average_update(double& T, uint8_t& chi, double Tk, double w, double delta) {
    if (chi) {
        T = Tk;
        chi = 0;
    } else {
        T = (1.0 - w) * T + w * Tk;
    }
    if (std::fabs(T) > delta) chi = 1;
}

// Alg. 2: the weighted average, with the weight sum W (held in P) bounded by W_max.
void weighted_update(double& T, double& W, uint8_t& chi, double Tk, double w, double Wmax, double delta) {
    if (chi) {
        T = Tk;
        W = w;
        chi = 0;
    } else {
        T = (W * T + w * Tk) / (W + w);
        W = std::min(W + w, Wmax);
    }
    if (std::fabs(T) > delta) chi = 1;
}

// One measurement into one voxel by the volume's update rule.
void update_voxel(const ov_params& p, double& T, double& P, uint8_t& chi, double Tk, double pk) {
    const double delta = (double)p.truncation;
    if (p.update_rule == 1)
        average_update(T, chi, Tk, (double)p.update_weight, delta);
    else if (p.update_rule == 2)
        weighted_update(T, P, chi, Tk, (double)p.update_weight, (double)p.weight_max, delta);
    else
        kalman_update(T, P, chi, Tk, pk, (double)p.process_variance, delta);
}

// --------------------------------------------------------------------------
// Raycast (section "Scene Rendering")
// --------------------------------------------------------------------------
// Readings: the ray of pixel (u,v) is o + z d with o the camera centre and
// d = R ((u-cx)/fx, (v-cy)/fy, 1), so z is camera depth. The field along it is
// the trilinear interpolation of T over the 8 lattice voxels around the point; it
// is undefined when any of them is unallocated, chi or outside the grid. The
// surface is the first + to - crossing between consecutive defined samples of a
// march of step 0.05 s from raycast_near to raycast_far, bisected to 1e-12 m; a
// - to + crossing first means the ray met a back face and is a miss. The normal is
// the normalised central difference of the field at the hit (+-1 voxel along the
// world axes), turned towards the camera.

int32_t lookup(const Volume& v, int64_t bx, int64_t by, int64_t bz) {
    if (bx < 0 || by < 0 || bz < 0 || bx >= v.nb || by >= v.nb || bz >= v.nb) return -1;
    auto it = v.index.find(block_key(bx, by, bz, v.nb));
    return it == v.index.end() ? -1 : it->second;
}

bool voxel_value(const Volume& v, int64_t ix, int64_t iy, int64_t iz, double* out) {
    const int32_t bi = lookup(v, ix >> 3, iy >> 3, iz >> 3);
    if (bi < 0) return false;
    const Block& b = v.blocks[bi];
    const int li = (int)((ix & 7) + 8 * (iy & 7) + 64 * (iz & 7));
    if (b.chi[li]) return false;
    *out = b.T[li];
    return true;
}

bool trilinear(const Volume& v, const double p[3], double* out) {
    const double s = (double)v.p.voxel_size;
    double q[3], fr[3];
    int64_t base[3];
    for (int r = 0; r < 3; ++r) {
        q[r] = (p[r] - v.p.origin[r]) / s;
        const double fl = std::floor(q[r]);
        if (!(fl >= 0.0 && fl + 1.0 < (double)v.p.grid_dim)) return false;
        base[r] = (int64_t)fl;
        fr[r] = q[r] - fl;
    }
    double c[2][2][2];
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx)
                if (!voxel_value(v, base[0] + dx, base[1] + dy, base[2] + dz, &c[dz][dy][dx]))
                    return false;
    double acc = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                const double w = (dx ? fr[0] : 1.0 - fr[0]) * (dy ? fr[1] : 1.0 - fr[1]) *
                                 (dz ? fr[2] : 1.0 - fr[2]);
                acc += w * c[dz][dy][dx];
            }
    *out = acc;
    return true;
}

struct RayOut {
    double depth, vertex[3], normal[3];
    int32_t flags;   // 1 hit, 2 bisection met an undefined sample, 4 normal undefined,
                     // 8 crossing not unique within delta/2 (see crossing_unique)
};

// Whether the ray's sign change at camera depth zc is the only one, and the
// field is defined throughout, within one coarse step (delta/2) on either side.
// Where it is not, a march that samples the ray every delta/2 (the two-stage
// raycast of section "Scene Rendering") may legitimately report another zero
// crossing close by; such pixels are flagged.
bool crossing_unique(const Volume& v, const double o[3], const double d[3], double zc, double step) {
    const double h = 0.5 * (double)v.p.truncation;
    bool prev_def = false;
    double f_prev = 0.0;
    int changes = 0;
    for (double z = zc - h; z <= zc + h; z += step) {
        double p[3] = {o[0] + z * d[0], o[1] + z * d[1], o[2] + z * d[2]};
        double f;
        if (!trilinear(v, p, &f)) return false;
        if (prev_def && ((f_prev > 0.0 && f <= 0.0) || (f_prev <= 0.0 && f > 0.0))) ++changes;
        prev_def = true;
        f_prev = f;
    }
    return changes <= 1;
}

RayOut cast_ray(const Volume& v, const ov_intr& in, const double* pose, int32_t u, int32_t w) {
    const double nan = std::numeric_limits<double>::quiet_NaN();
    RayOut out{0.0, {nan, nan, nan}, {nan, nan, nan}, 0};
    const double s = (double)v.p.voxel_size;
    const double dc[3] = {((double)u - (double)in.cx) / (double)in.fx,
                          ((double)w - (double)in.cy) / (double)in.fy, 1.0};
    double o[3], d[3];
    for (int r = 0; r < 3; ++r) {
        o[r] = pose[4 * r + 3];
        d[r] = pose[4 * r] * dc[0] + pose[4 * r + 1] * dc[1] + pose[4 * r + 2] * dc[2];
    }
    auto at = [&](double z, double p[3]) {
        for (int r = 0; r < 3; ++r) p[r] = o[r] + z * d[r];
    };
    const double z0 = (double)v.p.raycast_near, z1 = (double)v.p.raycast_far;
    const double step = 0.05 * s;
    int64_t i = 0;
    bool prev_def = false;
    double f_prev = 0.0, z_prev = 0.0;
    double zl = 0.0, zr = 0.0;
    bool found = false;
    for (;;) {
        const double z = z0 + (double)i * step;
        if (z > z1) break;
        double p[3];
        at(z, p);
        // Samples whose lower lattice corner lies in an unallocated block are
        // undefined; skipping them to the block's exit changes nothing.
        int64_t bc[3];
        for (int r = 0; r < 3; ++r) bc[r] = (int64_t)std::floor(std::floor((p[r] - v.p.origin[r]) / s) / 8.0);
        if (lookup(v, bc[0], bc[1], bc[2]) < 0) {
            double zexit = std::numeric_limits<double>::infinity();
            for (int r = 0; r < 3; ++r) {
                const double dq = d[r] / s;
                const double q0 = (o[r] - v.p.origin[r]) / s;
                if (dq > 0) zexit = std::min(zexit, (8.0 * (double)(bc[r] + 1) - q0) / dq);
                if (dq < 0) zexit = std::min(zexit, (8.0 * (double)bc[r] - q0) / dq);
            }
            int64_t inext = i + 1;
            if (std::isfinite(zexit)) {
                const double k = std::floor((zexit - z0) / step) - 1.0;
                if (k > (double)inext) inext = (int64_t)std::min(k, 9.0e15);
            }
            i = inext;
            prev_def = false;
            continue;
        }
        double f;
        const bool def = trilinear(v, p, &f);
        if (def && prev_def) {
            if (f_prev > 0.0 && f <= 0.0) {
                zl = z_prev;
                zr = z;
                found = true;
                break;
            }
            if (f_prev < 0.0 && f > 0.0) {        // back face first: miss
                if (!crossing_unique(v, o, d, z, step)) out.flags |= 8;
                break;
            }
        }
        prev_def = def;
        f_prev = f;
        z_prev = z;
        ++i;
    }
    if (!found) return out;
    for (int it = 0; it < 200 && zr - zl > 1e-12; ++it) {
        const double zm = 0.5 * (zl + zr);
        double p[3], f;
        at(zm, p);
        if (!trilinear(v, p, &f)) {
            out.flags |= 2;
            break;
        }
        if (f > 0.0) zl = zm; else zr = zm;
    }
    const double zs = 0.5 * (zl + zr);
    out.flags |= 1;
    if (!crossing_unique(v, o, d, zs, step)) out.flags |= 8;
    out.depth = zs;
    double p[3];
    at(zs, p);
    for (int r = 0; r < 3; ++r) out.vertex[r] = p[r];
    double g[3];
    bool ok = true;
    for (int r = 0; r < 3 && ok; ++r) {
        double pp[3] = {p[0], p[1], p[2]}, pm[3] = {p[0], p[1], p[2]};
        pp[r] += s;
        pm[r] -= s;
        double fp, fm;
        ok = trilinear(v, pp, &fp) && trilinear(v, pm, &fm);
        if (ok) g[r] = (fp - fm) / (2.0 * s);
    }
    const double gn = ok ? std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]) : 0.0;
    if (!ok || !(gn > 0.0)) {
        out.flags |= 4;
        return out;
    }
    double sgn = (g[0] * d[0] + g[1] * d[1] + g[2] * d[2]) > 0.0 ? -1.0 : 1.0;
    for (int r = 0; r < 3; ++r) out.normal[r] = sgn * g[r] / gn;
    return out;
}

// --------------------------------------------------------------------------
// Eviction and volume shift (section "Discussion")
// --------------------------------------------------------------------------
// The paper names both for scenes beyond device memory: the TSDF data of the
// occupied blocks is evicted to other storage, and a shift of the volume evicts
// the blocks that leave it and rebuilds the offset array. Readings:
//   * eviction removes every block whose block coordinates lie outside a box
//     [lo, hi) and hands out its coordinates, allocation frame and values;
//   * a shift by d moves the grid by whole blocks: origin' = origin + 8 s d, so
//     voxel i' = i - 8 d sits where voxel i sat; blocks whose new coordinates
//     b - d leave [0, nb) are evicted first;
//   * an imported block is allocated at the given frame with the given values.

bool outside_box(const Block& b, const int32_t lo[3], const int32_t hi[3]) {
    for (int r = 0; r < 3; ++r)
        if (b.b[r] < lo[r] || b.b[r] >= hi[r]) return true;
    return false;
}

void rebuild_index(Volume& v) {
    v.index.clear();
    for (size_t i = 0; i < v.blocks.size(); ++i)
        v.index.emplace(block_key(v.blocks[i].b[0], v.blocks[i].b[1], v.blocks[i].b[2], v.nb), (int32_t)i);
}

// Removes the blocks outside [lo, hi); writes them in ascending key order.
int64_t evict_box(Volume& v, const int32_t lo[3], const int32_t hi[3], int32_t* coords_frame, double* T,
                  double* P) {
    std::vector<std::pair<uint32_t, size_t>> gone;
    for (size_t i = 0; i < v.blocks.size(); ++i)
        if (outside_box(v.blocks[i], lo, hi))
            gone.emplace_back(block_key(v.blocks[i].b[0], v.blocks[i].b[1], v.blocks[i].b[2], v.nb), i);
    std::sort(gone.begin(), gone.end());
    const double nan = std::numeric_limits<double>::quiet_NaN();
    for (size_t n = 0; n < gone.size(); ++n) {
        const Block& b = v.blocks[gone[n].second];
        if (coords_frame) {
            for (int r = 0; r < 3; ++r) coords_frame[4 * n + r] = b.b[r];
            coords_frame[4 * n + 3] = b.alloc_frame;
        }
        if (!v.p.store_values) continue;
        for (int l = 0; l < M3; ++l) {
            if (T) T[n * M3 + l] = b.chi[l] ? nan : b.T[l];
            if (P) P[n * M3 + l] = b.chi[l] ? nan : b.P[l];
        }
    }
    std::vector<Block> kept;
    kept.reserve(v.blocks.size() - gone.size());
    for (Block& b : v.blocks)
        if (!outside_box(b, lo, hi)) kept.push_back(std::move(b));
    v.blocks = std::move(kept);
    rebuild_index(v);
    return (int64_t)gone.size();
}

}  // namespace

// ==========================================================================
// C interface for the test suite (ctypes)
// ==========================================================================
extern "C" {

void* ov_create(const ov_params* p) {
    if (!p || p->grid_dim <= 0 || p->grid_dim % M != 0) return nullptr;
    Volume* v = new Volume();
    v->p = *p;
    v->nb = p->grid_dim / M;
    return v;
}

void ov_destroy(void* h) { delete static_cast<Volume*>(h); }

int64_t ov_num_blocks(const void* h) { return (int64_t)static_cast<const Volume*>(h)->blocks.size(); }

int32_t ov_alloc_half_samples(const ov_params* p) {
    double pose[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
    return alloc_consts(*p, pose).J;
}

// Keys of the blocks one frame's surface samples touch (before any pool limit).
int64_t ov_frame_blocks(const ov_params* p, const float* depth, const ov_intr* in,
                        const double* pose, uint32_t* keys_out, int64_t max_out) {
    std::vector<uint32_t> keys = frame_blocks(*p, depth, *in, pose);
    const int64_t n = std::min<int64_t>((int64_t)keys.size(), max_out);
    if (keys_out) std::memcpy(keys_out, keys.data(), (size_t)n * sizeof(uint32_t));
    return (int64_t)keys.size();
}

void ov_allocate(void* h, const float* depth, const ov_intr* in, const double* pose,
                 int32_t frame, int64_t* n_new, int32_t* overflow) {
    Volume& v = *static_cast<Volume*>(h);
    add_blocks(v, frame_blocks(v.p, depth, *in, pose), frame, n_new, overflow);
}

// The update rule (Alg. 3 by default) over every voxel of every allocated block
// (no culling).
void ov_integrate(void* h, const float* depth, const float* var, const ov_intr* in,
                  const double* pose) {
    Volume& v = *static_cast<Volume*>(h);
    if (!v.p.store_values) return;
    const Frame f = make_frame(depth, var, *in, pose);
    const int64_t nblk = (int64_t)v.blocks.size();
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t bi = 0; bi < nblk; ++bi) {
        Block& b = v.blocks[bi];
        for (int l = 0; l < M3; ++l) {
            const int64_t ix = (int64_t)M * b.b[0] + (l & 7);
            const int64_t iy = (int64_t)M * b.b[1] + ((l >> 3) & 7);
            const int64_t iz = (int64_t)M * b.b[2] + (l >> 6);
            const Meas m = measure(v.p, f, ix, iy, iz);
            if (m.amb) b.amb[l] = 1;
            if (!m.valid) continue;
            update_voxel(v.p, b.T[l], b.P[l], b.chi[l], m.Tk, m.pk);
        }
    }
}

// Blocks in ascending key order: coords_frame (n x 4: bx, by, bz, alloc_frame),
// T and P (n x 512, NaN where chi), amb (n x 512). Any output may be null.
void ov_export(const void* h, int32_t* coords_frame, double* T, double* P, uint8_t* amb) {
    const Volume& v = *static_cast<const Volume*>(h);
    std::vector<std::pair<uint32_t, int32_t>> order;
    order.reserve(v.index.size());
    for (const auto& kv : v.index) order.emplace_back(kv.first, kv.second);
    std::sort(order.begin(), order.end());
    const double nan = std::numeric_limits<double>::quiet_NaN();
    for (size_t n = 0; n < order.size(); ++n) {
        const Block& b = v.blocks[order[n].second];
        if (coords_frame) {
            for (int r = 0; r < 3; ++r) coords_frame[4 * n + r] = b.b[r];
            coords_frame[4 * n + 3] = b.alloc_frame;
        }
        if (!v.p.store_values) continue;
        for (int l = 0; l < M3; ++l) {
            if (T) T[n * M3 + l] = b.chi[l] ? nan : b.T[l];
            if (P) P[n * M3 + l] = b.chi[l] ? nan : b.P[l];
            if (amb) amb[n * M3 + l] = b.amb[l];
        }
    }
}

// Number of blocks outside the block box [lo, hi).
int64_t ov_count_outside(const void* h, const int32_t* lo, const int32_t* hi) {
    const Volume& v = *static_cast<const Volume*>(h);
    int64_t n = 0;
    for (const Block& b : v.blocks) n += outside_box(b, lo, hi);
    return n;
}

// Evicts the blocks outside [lo, hi) into the buffers (ascending key order,
// layout of ov_export); returns their number.
int64_t ov_evict(void* h, const int32_t* lo, const int32_t* hi, int32_t* coords_frame, double* T, double* P) {
    return evict_box(*static_cast<Volume*>(h), lo, hi, coords_frame, T, P);
}

// Shifts the grid by d blocks; the blocks that leave it are written as by
// ov_evict (coordinates before the shift).
int64_t ov_shift(void* h, const int32_t* d, int32_t* coords_frame, double* T, double* P) {
    Volume& v = *static_cast<Volume*>(h);
    int32_t lo[3], hi[3];
    for (int r = 0; r < 3; ++r) {
        lo[r] = d[r];
        hi[r] = d[r] + v.nb;
    }
    const int64_t n = evict_box(v, lo, hi, coords_frame, T, P);
    for (Block& b : v.blocks)
        for (int r = 0; r < 3; ++r) b.b[r] -= d[r];
    rebuild_index(v);
    for (int r = 0; r < 3; ++r) v.p.origin[r] += (double)((int64_t)M * d[r]) * (double)v.p.voxel_size;
    return n;
}

// Adds n blocks with the given values (NaN T = chi) at allocation frame
// `frame`. Returns 0, or -1 (nothing added) when a block lies outside the grid,
// is given twice or is already allocated, or the pool would overflow.
int32_t ov_import(void* h, int64_t n, const int32_t* coords_frame, const double* T, const double* P, int32_t frame) {
    Volume& v = *static_cast<Volume*>(h);
    std::vector<uint32_t> keys;
    for (int64_t i = 0; i < n; ++i) {
        const int32_t* c = coords_frame + 4 * i;
        for (int r = 0; r < 3; ++r)
            if (c[r] < 0 || c[r] >= v.nb) return -1;
        keys.push_back(block_key(c[0], c[1], c[2], v.nb));
        if (v.index.count(keys.back())) return -1;
    }
    std::vector<uint32_t> sorted(keys);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return -1;
    if ((int64_t)v.blocks.size() + n > v.p.block_capacity) return -1;
    for (int64_t i = 0; i < n; ++i) {
        Block blk;
        for (int r = 0; r < 3; ++r) blk.b[r] = coords_frame[4 * i + r];
        blk.alloc_frame = frame;
        if (v.p.store_values) {
            blk.T.assign(M3, 0.0);
            blk.P.assign(M3, 0.0);
            blk.chi.assign(M3, 1);
            blk.amb.assign(M3, 0);
            for (int l = 0; l < M3; ++l) {
                const double t = T[i * M3 + l];
                if (std::isnan(t)) continue;
                blk.chi[l] = 0;
                blk.T[l] = t;
                blk.P[l] = P[i * M3 + l];
            }
        }
        v.index.emplace(keys[i], (int32_t)v.blocks.size());
        v.blocks.push_back(std::move(blk));
    }
    return 0;
}

// The volume's origin (it moves with ov_shift).
void ov_origin(const void* h, double* out) {
    const Volume& v = *static_cast<const Volume*>(h);
    for (int r = 0; r < 3; ++r) out[r] = v.p.origin[r];
}

void ov_raycast(const void* h, const ov_intr* in, const double* pose, int64_t n,
                const int32_t* uv, double* depth, double* vertex, double* normal,
                int32_t* flags) {
    const Volume& v = *static_cast<const Volume*>(h);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < n; ++k) {
        const RayOut r = cast_ray(v, *in, pose, uv[2 * k], uv[2 * k + 1]);
        depth[k] = r.depth;
        for (int c = 0; c < 3; ++c) {
            vertex[3 * k + c] = r.vertex[c];
            normal[3 * k + c] = r.normal[c];
        }
        flags[k] = r.flags;
    }
}

// Trilinear field at n world points (n x 3): value, or NaN where undefined.
void ov_field(const void* h, int64_t n, const double* points, double* f) {
    const Volume& v = *static_cast<const Volume*>(h);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        double val;
        f[k] = trilinear(v, points + 3 * k, &val) ? val : std::numeric_limits<double>::quiet_NaN();
    }
}

// Per-voxel replay of a whole sequence: for each listed voxel (ix, iy, iz) whose
// block joined the pool at frame alloc_frame[k], apply every frame from that one
// on with the volume's update rule. Gives the same values ov_integrate would, one
// voxel at a time.
void ov_replay_voxels(const ov_params* p, int32_t n_frames, const float* const* depths,
                      const float* const* vars, const ov_intr* in, const double* poses,
                      int64_t n, const int32_t* voxels, const int32_t* alloc_frame,
                      double* T_out, double* P_out, uint8_t* amb_out) {
    const double nan = std::numeric_limits<double>::quiet_NaN();
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < n; ++k) {
        double T = 0.0, P = 0.0;
        uint8_t chi = 1, amb = 0;
        for (int32_t fi = std::max(0, alloc_frame[k]); fi < n_frames; ++fi) {
            const Frame f = make_frame(depths[fi], vars ? vars[fi] : nullptr, *in, poses + 16 * fi);
            const Meas m = measure(*p, f, voxels[3 * k], voxels[3 * k + 1], voxels[3 * k + 2]);
            if (m.amb) amb = 1;
            if (m.valid) update_voxel(*p, T, P, chi, m.Tk, m.pk);
        }
        T_out[k] = chi ? nan : T;
        P_out[k] = chi ? nan : P;
        amb_out[k] = amb;
    }
}

// Dense brute force: the update rule applied to every voxel of a G^3 grid, no
// allocation.
void* ov_dense_create(const ov_params* p) {
    if (!p || p->grid_dim <= 0) return nullptr;
    Volume* v = new Volume();
    v->p = *p;
    v->nb = p->grid_dim;     // here: voxels per axis
    const size_t n = (size_t)p->grid_dim * p->grid_dim * p->grid_dim;
    v->blocks.resize(1);
    v->blocks[0].T.assign(n, 0.0);
    v->blocks[0].P.assign(n, 0.0);
    v->blocks[0].chi.assign(n, 1);
    v->blocks[0].amb.assign(n, 0);
    return v;
}

void ov_dense_integrate(void* h, const float* depth, const float* var, const ov_intr* in,
                        const double* pose) {
    Volume& v = *static_cast<Volume*>(h);
    const Frame f = make_frame(depth, var, *in, pose);
    const int64_t G = v.p.grid_dim;
    Block& b = v.blocks[0];
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t iz = 0; iz < G; ++iz)
        for (int64_t iy = 0; iy < G; ++iy)
            for (int64_t ix = 0; ix < G; ++ix) {
                const size_t l = (size_t)(ix + G * (iy + G * iz));
                const Meas m = measure(v.p, f, ix, iy, iz);
                if (m.amb) b.amb[l] = 1;
                if (m.valid) update_voxel(v.p, b.T[l], b.P[l], b.chi[l], m.Tk, m.pk);
            }
}

// Read n voxels (ix, iy, iz) of a dense grid: T, P (NaN where chi), amb.
void ov_dense_read(const void* h, int64_t n, const int32_t* voxels, double* T, double* P,
                   uint8_t* amb) {
    const Volume& v = *static_cast<const Volume*>(h);
    const int64_t G = v.p.grid_dim;
    const Block& b = v.blocks[0];
    const double nan = std::numeric_limits<double>::quiet_NaN();
    for (int64_t k = 0; k < n; ++k) {
        const size_t l = (size_t)(voxels[3 * k] + G * (voxels[3 * k + 1] + G * (int64_t)voxels[3 * k + 2]));
        T[k] = b.chi[l] ? nan : b.T[l];
        P[k] = b.chi[l] ? nan : b.P[l];
        amb[k] = b.amb[l];
    }
}

// Count of dense voxels that are not chi, and of those lying in blocks absent
// from the sparse volume h (the misses the sampling allocation tolerates).
void ov_dense_coverage(const void* dense, const void* sparse, int64_t* n_valid, int64_t* n_missed) {
    const Volume& d = *static_cast<const Volume*>(dense);
    const Volume& s = *static_cast<const Volume*>(sparse);
    const int64_t G = d.p.grid_dim;
    int64_t nv = 0, nm = 0;
    for (int64_t iz = 0; iz < G; ++iz)
        for (int64_t iy = 0; iy < G; ++iy)
            for (int64_t ix = 0; ix < G; ++ix) {
                if (d.blocks[0].chi[(size_t)(ix + G * (iy + G * iz))]) continue;
                ++nv;
                if (lookup(s, ix >> 3, iy >> 3, iz >> 3) < 0) ++nm;
            }
    *n_valid = nv;
    *n_missed = nm;
}

// --------------------------------------------------------------------------
// Learned measurement variance (an addition to the paper: it motivates
// per-measurement variances - deviation growing with depth, poorer data near
// surface edges - and leaves their estimation open). A 27-32-32-1 perceptron
// with ReLU predicts out = log(p_k / p_quad) at a pixel from
//   f[0..24] = (D(u + d) - D(u)) / delta clamped to [-1, 1] over the 5x5
//              neighbourhood d (row-major, dy then dx); +1 where the neighbour
//              is outside the image or not a valid measurement,
//   f[25]    = D(u) / 4,
//   f[26]    = |cos| of the angle between the viewing ray and the surface
//              normal from the depth map's central differences (0 when a
//              4-neighbour is invalid);
// the variance is p_quad exp(out), or p_quad when |out| > ln 4 or out is not
// finite. Training minimises the Gaussian negative log-likelihood of fusion
// residuals r: L = (log p + r^2 / p) / 2, i.e. (out + s exp(-out)) / 2 up to a
// constant, s = r^2 / p_quad. Parameters, in order: W1[32][27], b1[32],
// W2[32][32], b2[32], W3[32], b3 (1985 values).
// --------------------------------------------------------------------------
constexpr int kIn = 27, kHid = 32;
constexpr int kParams = kHid * kIn + kHid + kHid * kHid + kHid + kHid + 1;

int32_t ov_mlp_param_count(void) { return kParams; }

// Features of n pixels (uv: n x 2); valid[k] = 0 when the centre depth is not a
// valid measurement (the network is then not used).
void ov_mlp_features(const float* depth, const ov_intr* in, const ov_params* p, int64_t n, const int32_t* uv,
                     double* feat, uint8_t* valid) {
    const double delta = (double)p->truncation;
    auto D = [&](int64_t u, int64_t v, double* out) {
        if (u < 0 || v < 0 || u >= in->width || v >= in->height) return false;
        const float d = depth[v * in->width + u];
        if (!depth_valid(d, *p)) return false;
        *out = (double)d;
        return true;
    };
    auto point = [&](int64_t u, int64_t v, double d, double P[3]) {
        P[0] = d * ((double)u - (double)in->cx) / (double)in->fx;
        P[1] = d * ((double)v - (double)in->cy) / (double)in->fy;
        P[2] = d;
    };
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        const int64_t u = uv[2 * k], v = uv[2 * k + 1];
        double* f = feat + kIn * k;
        double d0;
        valid[k] = D(u, v, &d0) ? 1 : 0;
        if (!valid[k]) {
            for (int i = 0; i < kIn; ++i) f[i] = 0.0;
            continue;
        }
        int i = 0;
        for (int dy = -2; dy <= 2; ++dy)
            for (int dx = -2; dx <= 2; ++dx, ++i) {
                double d;
                f[i] = D(u + dx, v + dy, &d) ? std::fmax(-1.0, std::fmin(1.0, (d - d0) / delta)) : 1.0;
            }
        f[25] = d0 / 4.0;
        double dl, dr, du, dd;
        f[26] = 0.0;
        if (D(u - 1, v, &dl) && D(u + 1, v, &dr) && D(u, v - 1, &du) && D(u, v + 1, &dd)) {
            double Pl[3], Pr[3], Pu[3], Pd[3], P0[3];
            point(u - 1, v, dl, Pl); point(u + 1, v, dr, Pr); point(u, v - 1, du, Pu); point(u, v + 1, dd, Pd);
            point(u, v, d0, P0);
            const double a[3] = {Pr[0] - Pl[0], Pr[1] - Pl[1], Pr[2] - Pl[2]};
            const double b[3] = {Pd[0] - Pu[0], Pd[1] - Pu[1], Pd[2] - Pu[2]};
            const double nn[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
            const double ln = std::sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
            const double lp = std::sqrt(P0[0] * P0[0] + P0[1] * P0[1] + P0[2] * P0[2]);
            if (ln > 0.0 && lp > 0.0) f[26] = std::fabs(nn[0] * P0[0] + nn[1] * P0[1] + nn[2] * P0[2]) / (ln * lp);
        }
    }
}

namespace {
struct MlpAct {
    double h1[kHid], a1[kHid], h2[kHid], a2[kHid], out;
};

void mlp_forward(const double* w, const double* x, MlpAct* t) {
    const double* W1 = w;
    const double* b1 = W1 + kHid * kIn;
    const double* W2 = b1 + kHid;
    const double* b2 = W2 + kHid * kHid;
    const double* W3 = b2 + kHid;
    const double b3 = W3[kHid];
    for (int j = 0; j < kHid; ++j) {
        double acc = b1[j];
        for (int i = 0; i < kIn; ++i) acc += W1[j * kIn + i] * x[i];
        t->h1[j] = acc;
        t->a1[j] = acc > 0.0 ? acc : 0.0;
    }
    for (int j = 0; j < kHid; ++j) {
        double acc = b2[j];
        for (int i = 0; i < kHid; ++i) acc += W2[j * kHid + i] * t->a1[i];
        t->h2[j] = acc;
        t->a2[j] = acc > 0.0 ? acc : 0.0;
    }
    double acc = b3;
    for (int j = 0; j < kHid; ++j) acc += W3[j] * t->a2[j];
    t->out = acc;
}
}  // namespace

void ov_mlp_forward(const double* w, int64_t n, const double* feat, double* out) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        MlpAct t;
        mlp_forward(w, feat + kIn * k, &t);
        out[k] = t.out;
    }
}

// Sum over the n samples of L = (out + s exp(-out)) / 2 and its gradient with
// respect to every parameter (backpropagation, written out layer by layer).
void ov_mlp_loss_grad(const double* w, int64_t n, const double* feat, const double* s, double* grad, double* loss) {
    const double* W2 = w + kHid * kIn + kHid;
    const double* W3 = W2 + kHid * kHid + kHid;
    for (int i = 0; i < kParams; ++i) grad[i] = 0.0;
    double total = 0.0;
    double* gW1 = grad;
    double* gb1 = gW1 + kHid * kIn;
    double* gW2 = gb1 + kHid;
    double* gb2 = gW2 + kHid * kHid;
    double* gW3 = gb2 + kHid;
    double* gb3 = gW3 + kHid;
    for (int64_t k = 0; k < n; ++k) {
        const double* x = feat + kIn * k;
        MlpAct t;
        mlp_forward(w, x, &t);
        const double e = s[k] * std::exp(-t.out);
        total += 0.5 * (t.out + e);
        const double g = 0.5 * (1.0 - e);            // dL/dout
        double d2[kHid], d1[kHid];
        *gb3 += g;
        for (int j = 0; j < kHid; ++j) {
            gW3[j] += g * t.a2[j];
            d2[j] = t.h2[j] > 0.0 ? g * W3[j] : 0.0;
        }
        for (int j = 0; j < kHid; ++j) {
            gb2[j] += d2[j];
            for (int i = 0; i < kHid; ++i) gW2[j * kHid + i] += d2[j] * t.a1[i];
        }
        for (int i = 0; i < kHid; ++i) {
            double acc = 0.0;
            for (int j = 0; j < kHid; ++j) acc += W2[j * kHid + i] * d2[j];
            d1[i] = t.h1[i] > 0.0 ? acc : 0.0;
        }
        for (int j = 0; j < kHid; ++j) {
            gb1[j] += d1[j];
            for (int i = 0; i < kIn; ++i) gW1[j * kIn + i] += d1[j] * x[i];
        }
    }
    *loss = total;
}

// Per-pixel variance map with the network (float output, 0 where the depth is
// not valid): p_quad exp(out), or p_quad where out lies outside
// [-ln 4, ln 64] or is not finite (a measurement may be up to 64 times noisier
// than the quadratic model says - a sensor far poorer at depth edges - or 4
// times less noisy).
void ov_mlp_variance_map(const double* w, const float* depth, const ov_intr* in, const ov_params* p, float* var) {
    const int64_t n = (int64_t)in->width * in->height;
    std::vector<int32_t> uv(2 * n);
    for (int64_t k = 0; k < n; ++k) {
        uv[2 * k] = (int32_t)(k % in->width);
        uv[2 * k + 1] = (int32_t)(k / in->width);
    }
    std::vector<double> feat(kIn * n), out(n);
    std::vector<uint8_t> valid(n);
    ov_mlp_features(depth, in, p, n, uv.data(), feat.data(), valid.data());
    ov_mlp_forward(w, n, feat.data(), out.data());
    const double lo = -std::log(4.0), hi = std::log(64.0);
    for (int64_t k = 0; k < n; ++k) {
        if (!valid[k]) {
            var[k] = 0.0f;
            continue;
        }
        const double d = (double)depth[k];
        const double sg = (double)p->sigma_coeff * d * d;
        const double pq = sg * sg;
        var[k] = (float)((std::isfinite(out[k]) && out[k] >= lo && out[k] <= hi) ? pq * std::exp(out[k]) : pq);
    }
}

int32_t ov_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

}  // extern "C"
