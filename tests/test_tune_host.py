"""Host logic of the autotuner (no GPU): the candidate grid, the first
candidate being the library's defaults, and the -D form of a tuned file."""
import json

from paper_1802_03980_gb300 import tune


def test_candidates_are_the_grid_product_in_order():
    grid = {"A": [1, 2], "B": [3, 4, 5]}
    c = tune.candidates(grid)
    assert len(c) == 6
    assert c[0] == {"A": 1, "B": 3} and c[-1] == {"A": 2, "B": 5}
    assert len({tuple(sorted(x.items())) for x in c}) == 6


def test_default_grid_starts_with_the_library_defaults():
    # the first entry of each list is the value the kernels compile with
    # when no define is given (the tuner's reference candidate), as the
    # sources' #ifndef / #define blocks set it
    import os
    import re
    csrc = os.path.join(os.path.dirname(tune.__file__), "csrc")
    text = "".join(open(os.path.join(csrc, f)).read() for f in os.listdir(csrc)
                   if f.endswith((".cu", ".cuh")))
    defaults = {}
    for name in tune.GRID:
        m = re.search(r"#ifndef %s\s*\n#define %s (\d+)" % (name, name), text)
        assert m, name
        defaults[name] = int(m.group(1))
    assert tune.candidates(tune.GRID)[0] == defaults


def test_tuned_defines_reads_a_tuned_file(tmp_path):
    p = tmp_path / "tuned.json"
    p.write_text(json.dumps({"defines": {"KF_PREFETCH": 1, "KF_ASSOC_U": 4}}))
    assert tune.tuned_defines(str(p)) == ["KF_ASSOC_U=4", "KF_PREFETCH=1"]
    assert tune.tuned_defines(str(tmp_path / "missing.json")) == []


def test_pose_error_of_equal_and_shifted_poses():
    import numpy as np
    a = np.tile(np.eye(4), (3, 1, 1))
    b = a.copy()
    b[1, 0, 3] += 2e-6
    rot, tr = tune._pose_err(a, b)
    assert rot == 0.0 and abs(tr - 2e-6) < 1e-12
