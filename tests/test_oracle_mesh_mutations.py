"""Plant plausible mistakes in copies of the marching-cubes oracle
(``oracle/mesh.py``) and check that the mesh pins catch each one."""
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mesh.py")

MUTATIONS = [
    ("orientation_flipped", "if np.dot(np.cross(B - A, I - A), n) > 0:", "if np.dot(np.cross(B - A, I - A), n) < 0:"),
    ("inside_is_positive", "inside = tuple(bool(x < 0) for x in v8)", "inside = tuple(bool(x > 0) for x in v8)"),
    ("interpolation_from_the_wrong_end", "t = v8[a] / (v8[a] - v8[b])", "t = v8[b] / (v8[b] - v8[a])"),
    ("ambiguous_face_one_segment", "        if len(crossed) == 2:", "        if len(crossed) >= 2:"),
    ("fan_skips_a_triangle", "for k in range(1, len(loop) - 1):", "for k in range(1, max(1, len(loop) - 2)):"),
]

CHILD = textwrap.dedent("""
    import importlib.util, sys
    sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
    import oracle
    spec = importlib.util.spec_from_file_location("oracle.mesh", {path!r})
    mod = importlib.util.module_from_spec(spec)
    sys.modules["oracle.mesh"] = mod; oracle.mesh = mod
    spec.loader.exec_module(mod)
    import pins
    failed = []
    for pin in pins.MESH_PINS:
        try:
            pin()
        except Exception:
            failed.append(pin.__name__)
    print("FAILED:" + ",".join(failed))
""")


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mesh_pins_catch_mutation(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    path = tmp_path / "mesh.py"
    path.write_text(src.replace(old, new))
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), path=str(path))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    line = [l for l in r.stdout.splitlines() if l.startswith("FAILED:")]
    assert line, r.stdout + r.stderr
    assert line[0] != "FAILED:", f"no pin caught {name}"
