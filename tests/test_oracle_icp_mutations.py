"""Plant plausible mistakes in copies of the registration oracle
(``oracle/icp.py``) and check that the registration pins catch each one. Each
copy is imported as ``oracle.icp`` in a child process; the real module is
untouched."""
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "icp.py")

# (name, text in the oracle, planted replacement)
MUTATIONS = [
    ("cross_product_order", "c_hat = (np.cross(p, n) - np.cross(m[None, :], n)) / S[None, :]",
     "c_hat = (np.cross(n, p) - np.cross(m[None, :], n)) / S[None, :]"),
    ("printed_translation_recovery", "t = x[3:] - np.cross(r, m)", "t = x[3:] + np.cross(r, m)"),
    ("printed_rotation_recovery", "r = x[:3] / S", "r = x[:3] * S"),
    ("residual_sign", "return J.T @ J, -(J.T @ r), m, S", "return J.T @ J, (J.T @ r), m, S"),
    ("projection_floor", "um = np.floor(intr.fx * xm[..., 0] / xm[..., 2] + intr.cx + 0.5)",
     "um = np.floor(intr.fx * xm[..., 0] / xm[..., 2] + intr.cx)"),
    ("model_camera_transposed", "xm = (p - tm) @ Rm ", "xm = (p - tm) @ Rm.T "),
    ("update_on_the_right", "return inc @ pose, {", "return pose @ inc, {"),
    ("frame_normal_unrotated", "ns = nf @ R.T", "ns = nf"),
    ("eigen_threshold_inverted", "keep = lam / max(N, 1) > theta", "keep = lam / max(N, 1) < theta"),
]

CHILD = textwrap.dedent("""
    import importlib.util, sys
    sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
    import oracle
    spec = importlib.util.spec_from_file_location("oracle.icp", {path!r})
    mod = importlib.util.module_from_spec(spec)
    sys.modules["oracle.icp"] = mod; oracle.icp = mod
    spec.loader.exec_module(mod)
    import pins
    failed = []
    for pin in (pins.pin_icp_recovers_a_known_motion, pins.pin_icp_scaled_equals_unscaled,
                pins.pin_icp_plane_keeps_unobservable_motion_out):
        try:
            pin()
        except Exception:
            failed.append(pin.__name__)
    print("FAILED:" + ",".join(failed))
""")


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_icp_pins_catch_mutation(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    path = tmp_path / "icp.py"
    path.write_text(src.replace(old, new))
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), path=str(path))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    line = [l for l in r.stdout.splitlines() if l.startswith("FAILED:")]
    assert line, r.stdout + r.stderr
    assert line[0] != "FAILED:", f"no pin caught {name}"
