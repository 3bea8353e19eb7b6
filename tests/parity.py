"""Parity report shared by the GPU tests: relative L2 error and max-abs error
(relative to the largest reference value) of a CUDA result against the
oracle, printed for every check, appended as a JSON line to the file named by
NEDNER_PARITY_LOG when that is set, and asserted against the tolerance."""
import json
import os
import sys

import numpy as np


def errors(got, want):
    got = np.asarray(got)
    want = np.asarray(want)
    d = np.abs(got - want)
    scale = max(float(np.abs(want).max()) if want.size else 0.0, 1e-300)
    rel = float(np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300))
    return rel, float(d.max()) / scale if d.size else 0.0


def check(got, want, tol, label=None):
    """Assert rel-L2(got, want) <= tol; report rel-L2 and max-abs."""
    rel, mx = errors(got, want)
    if label is None:
        label = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    print("%s: rel-L2 %.3e, max-abs %.3e of max |ref| (tol %.1e)" % (label, rel, mx, tol), file=sys.stderr)
    path = os.environ.get("NEDNER_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": label, "rel_l2": rel, "max_abs_rel": mx, "tol": tol}) + "\n")
    assert rel <= tol, (label, rel, mx)
    return rel, mx
