"""The bounds-checking build (`build(debug_bounds=True)`, TERA_DEBUG_BOUNDS):
the library's kernels with every write of a record, code or sort entry
checked against the range its pair or buffer owns (a violation latches
TERA_EBOUNDS and skips the write).  Chains of the parity tests (batched with
and without id columns, all pairs, one launch per subdomain, the predictor
path) run through libtera_debug.so in a child process (the library is chosen
when the binding loads) and must equal the oracle with the status clean."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.join(ROOT, "tests")

CHILD = r"""
import sys
sys.path[:0] = [{root!r}, {tests!r}]
from paper_2509_24063_gb300 import _lib
assert _lib.DEBUG_BOUNDS and _lib.LIB_PATH.endswith("libtera_debug.so"), _lib.LIB_PATH
import paper_2509_24063_gb300 as tera
from synth import Workload
import test_gpu_parity as par
import test_gpu_predictor as pred
wl = Workload("t", 60000, (0.0,) * 3, (200.0, 150.0, 150.0), (4, 3, 3), 15.0, 4,
              p_grow=0.1, p_divide=0.02, p_die=0.02, seed=41)
print("batched", flush=True)
par.run_chain(tera, wl, 4, path="batched")
print("batched without id columns", flush=True)
par.run_chain(tera, wl, 4, path="batched", id_columns=False)
print("all pairs", flush=True)
par.run_chain(tera, wl, 3, path="all_pairs")
print("per subdomain", flush=True)
par.run_chain(tera, wl, 3, per_subdomain=True)
print("predictor", flush=True)
pred.run_pred_chain(tera, pred.drift(n=30000, iters=4, seed=8), pred.velocity_network(),
                    "batched")
print("bounds-checked chains equal the oracle")
"""


def test_bounds_checking_build_runs_the_chains_clean():
    from paper_2509_24063_gb300 import build
    build.build(debug_bounds=True)
    env = dict(os.environ, TERA_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, tests=TESTS)], env=env,
                       capture_output=True, text=True, timeout=1200, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
    assert "bounds-checked chains equal the oracle" in r.stdout
