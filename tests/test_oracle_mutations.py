"""Plant plausible mistakes in copies of the oracle and check that the pins catch
each one: evidence that the pins constrain every part of the oracle.

Each mutation is a textual edit of ```oracle/tsdf_oracle.cpp`` compiled into a
temporary library; the pins run against it in a child process (so a mutation that
crashed would fail the child, not this test run). The real oracle is untouched.
"""
import concurrent.futures
import json
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, text in the oracle, planted replacement)
MUTATIONS = [
    ("kalman_correct_sign", "T = T + K * (Tk - T);", "T = T + K * (T - Tk);"),
    ("refine_step_sign", "u -= (a22 * g1 - a12 * g2) / det;", "u += (a22 * g1 - a12 * g2) / det;"),
    ("refine_jacobian_scale", "e.Ju[0] += D / fx;", "e.Ju[0] += D;"),
    ("refine_side_unoriented", "side = (-r[0] * n[0] - r[1] * n[1] - r[2] * n[2]) >= 0.0 ? 1.0 : -1.0;",
     "side = 1.0;"),
    ("alg1_weights_swapped", "T = (1.0 - w) * T + w * Tk;", "T = w * T + (1.0 - w) * Tk;"),
    ("alg2_no_weight_bound", "W = std::min(W + w, Wmax);", "W = W + w;"),
    ("alg2_first_weight", "T = Tk;\n        W = w;", "T = Tk;\n        W = 1.0;"),
    ("kalman_variance_shrink", "P = (1.0 - K) * P;", "P = K * P;"),
    ("kalman_predict_sign", "P = P + Q;                    // predict", "P = P - Q;"),
    ("kalman_gain", "const double K = P / (P + pk);", "const double K = pk / (P + pk);"),
    ("first_measurement_variance", "T = Tk;\n        P = pk;", "T = Tk;\n        P = pk * pk;"),
    ("camera_rotation_transposed",
     "xc[k] = f.R[0][k] * d[0] + f.R[1][k] * d[1] + f.R[2][k] * d[2];",
     "xc[k] = f.R[k][0] * d[0] + f.R[k][1] * d[1] + f.R[k][2] * d[2];"),
    ("tk_sign", "const double Tk = Dd - z;", "const double Tk = z - Dd;"),
    ("pixel_floor_not_round", "const double u0 = std::floor(uf + 0.5), v0 = std::floor(vf + 0.5);",
     "const double u0 = std::floor(uf), v0 = std::floor(vf);"),
    ("pixel_index_uv_swapped", "const int64_t pix = (int64_t)v * f.in.width + (int64_t)u;",
     "const int64_t pix = (int64_t)u * f.in.height + (int64_t)v;"),
    ("truncation_doubled", "if (std::fabs(Tk) > delta) return m;", "if (std::fabs(Tk) > 2.0 * delta) return m;"),
    ("variance_is_sigma", "pk = sigma * sigma;", "pk = sigma;"),
    ("voxel_centre_offset", "p.origin[2] + (double)iz * s};", "p.origin[2] + ((double)iz + 0.5) * s};"),
    ("alloc_rotation_transposed", "c.Mr[r][k] = (float)(pose[4 * r + k] / s);",
     "c.Mr[r][k] = (float)(pose[4 * k + r] / s);"),
    ("alloc_half_samples", "std::ceil(2.0 * delta / s - 1e-6)", "std::ceil(0.5 * delta / s - 1e-6)"),
    ("alloc_block_axes_swapped", "block_key(vx / M, vy / M, vz / M, nb)", "block_key(vy / M, vx / M, vz / M, nb)"),
    ("alloc_origin_sign", "c.a[r] = (float)((pose[4 * r + 3] - p.origin[r]) / s);",
     "c.a[r] = (float)((pose[4 * r + 3] + p.origin[r]) / s);"),
    ("alloc_order_descending", "for (uint32_t key : keys) {",
     "for (auto it_ = keys.rbegin(); it_ != keys.rend(); ++it_) { const uint32_t key = *it_;"),
    ("trilinear_weight_swapped", "const double w = (dx ? fr[0] : 1.0 - fr[0])",
     "const double w = (dx ? 1.0 - fr[0] : fr[0])"),
    ("raycast_crossing_reversed", "if (f_prev > 0.0 && f <= 0.0) {", "if (f_prev < 0.0 && f >= 0.0) {"),
    ("normal_orientation", "> 0.0 ? -1.0 : 1.0;", "> 0.0 ? 1.0 : -1.0;"),
    ("ray_direction_transposed",
     "d[r] = pose[4 * r] * dc[0] + pose[4 * r + 1] * dc[1] + pose[4 * r + 2] * dc[2];",
     "d[r] = pose[r] * dc[0] + pose[4 + r] * dc[1] + pose[8 + r] * dc[2];"),
    ("normal_axis_permuted", "pp[r] += s;\n        pm[r] -= s;",
     "pp[(r + 1) % 3] += s;\n        pm[(r + 1) % 3] -= s;"),
    ("mlp_relu_grad_dropped", "d2[j] = t.h2[j] > 0.0 ? g * W3[j] : 0.0;", "d2[j] = g * W3[j];"),
    ("mlp_backward_w2_transposed", "for (int j = 0; j < kHid; ++j) acc += W2[j * kHid + i] * d2[j];",
     "for (int j = 0; j < kHid; ++j) acc += W2[i * kHid + j] * d2[j];"),
    ("mlp_loss_grad_sign", "const double g = 0.5 * (1.0 - e);", "const double g = 0.5 * (e - 1.0);"),
    ("mlp_invalid_neighbour", "? std::fmax(-1.0, std::fmin(1.0, (d - d0) / delta)) : 1.0;",
     "? std::fmax(-1.0, std::fmin(1.0, (d - d0) / delta)) : 0.0;"),
    ("mlp_depth_feature", "f[25] = d0 / 4.0;", "f[25] = d0 / 2.0;"),
    ("mlp_variance_exp_sign", "pq * std::exp(out[k])", "pq * std::exp(-out[k])"),
    ("mlp_fallback_limit", "lo = -std::log(4.0), hi = std::log(64.0);", "lo = -std::log(4.0), hi = std::log(16.0);"),
    ("mlp_fallback_low_limit", "lo = -std::log(4.0), hi = std::log(64.0);", "lo = -std::log(16.0), hi = std::log(64.0);"),
    ("mlp_first_layer_relu", "t->a1[j] = acc > 0.0 ? acc : 0.0;", "t->a1[j] = acc;"),
    ("shift_origin_sign", "v.p.origin[r] += (double)((int64_t)M * d[r]) * (double)v.p.voxel_size;",
     "v.p.origin[r] -= (double)((int64_t)M * d[r]) * (double)v.p.voxel_size;"),
    ("shift_rekey_sign", "for (int r = 0; r < 3; ++r) b.b[r] -= d[r];", "for (int r = 0; r < 3; ++r) b.b[r] += d[r];"),
    ("evict_box_upper_inclusive", "if (b.b[r] < lo[r] || b.b[r] >= hi[r]) return true;",
     "if (b.b[r] < lo[r] || b.b[r] > hi[r]) return true;"),
    ("import_drops_values", "blk.chi[l] = 0;\n                blk.T[l] = t;", "blk.chi[l] = 0;\n                blk.T[l] = 0.0;"),
    ("import_allows_allocated", "if (v.index.count(keys.back())) return -1;", "(void)0;"),
    ("replay_one_frame_late", "fi = std::max(0, alloc_frame[k]);", "fi = std::max(0, alloc_frame[k] + 1);"),
    ("replay_ignores_allocation_frame", "fi = std::max(0, alloc_frame[k]);", "fi = 0;"),
    ("crossing_two_changes_unique", "return changes <= 1;", "return changes <= 2;"),
    ("crossing_always_unique", "return changes <= 1;", "return true;"),
    ("crossing_window_doubled", "const double h = 0.5 * (double)v.p.truncation;",
     "const double h = (double)v.p.truncation;"),
    ("crossing_skips_undefined", "if (!trilinear(v, p, &f)) return false;", "if (!trilinear(v, p, &f)) continue;"),
]


@pytest.fixture(scope="module")
def variants(tmp_path_factory):
    src = oracle.source_text()
    d = tmp_path_factory.mktemp("oracle_mutants")
    jobs = {}
    with concurrent.futures.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        for name, old, new in MUTATIONS:
            assert src.count(old) == 1, f"mutation {name}: anchor text not found once"
            jobs[name] = ex.submit(oracle.compile_variant, src.replace(old, new), str(d / f"lib_{name}.so"))
        return {k: v.result() for k, v in jobs.items()}


def _run_pins(lib_path):
    """The pins against one variant, in a process of its own (a planted mistake
    may crash the oracle); stops at the first pin that fails."""
    code = ("import sys, json; sys.path.insert(0, %r); sys.path.insert(0, %r); import pins; "
            "print(json.dumps(pins.run_all(%r, stop_at_first=True)))" % (ROOT, os.path.join(ROOT, "tests"), lib_path))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    return subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, env=env)


@pytest.fixture(scope="module")
def outcomes(variants):
    """Every variant's pin run, and one of the unmodified oracle, the processes
    side by side."""
    runs = dict(variants, unmodified=oracle.build())
    with concurrent.futures.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        jobs = {name: ex.submit(_run_pins, path) for name, path in runs.items()}
        return {k: v.result() for k, v in jobs.items()}


def test_unmodified_oracle_passes_the_same_run(outcomes):
    """The harness itself: the oracle as committed, run the same way, exits
    cleanly with no failing pin (so a crash below means the planted mistake)."""
    r = outcomes["unmodified"]
    assert r.returncode == 0, r.stderr[-2000:]
    assert json.loads(r.stdout.strip().splitlines()[-1]) == []


@pytest.mark.parametrize("name", [m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(outcomes, name):
    r = outcomes[name]
    if r.returncode != 0:
        return      # the planted mistake crashed the oracle: caught
    failed = json.loads(r.stdout.strip().splitlines()[-1])
    assert failed, f"no pin caught the planted mistake {name}"
