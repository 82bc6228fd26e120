"""The checked build (libssj_checked.so, -DSSJ_CHECKED): every index of the plan and verify
kernels is tested against its array's extent, and an out-of-bounds one sets device error bit 4
instead of faulting.  Parity tests run in a child process on that build must pass with no
check firing (a fired check turns a verification into SSJ_EDEVICE, so it fails them)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROBE = r"""
import numpy as np, oracle, synth
import paper_1812_09141_gb300 as ssj
assert ssj.LIB_PATH.endswith("libssj_checked.so"), ssj.LIB_PATH
ctx = ssj.ssj_create(0)
spec = synth.long_sets(n=600)
spec.plant_frac, spec.plant_edits = 0.3, 10
c = synth.collection(spec)
h = ssj.ssj_load_collection(ctx, c.offsets, c.tokens)
for gran in (0, ssj.SSJ_FORCE_THREAD, ssj.SSJ_FORCE_LANE, ssj.SSJ_FORCE_WARP, ssj.SSJ_FORCE_BLOCK,
             ssj.SSJ_FORCE_INDEX):
    pr, co, ci = ssj.feeder_all(c.offsets, c.tokens, 3, 5, n_threads=4)
    got = ssj.triples_to_array(ssj.ssj_verify_batch(ctx, h, h, 3, 5, pr, co, ci, flags=gran))
    want = oracle.sort_triples(oracle.allpairs_self(c.offsets, c.tokens, 3, 5)[0])
    assert np.array_equal(got, want), gran
    assert ssj.ssj_device_error(ctx) == 0
print("checked build ok")
"""


def _child(args, timeout):
    env = dict(os.environ, SSJ_LIBRARY="checked")
    return subprocess.run([sys.executable, *args], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=timeout)


def test_checked_build_loads_and_matches_the_oracle():
    from paper_1812_09141_gb300 import _build
    _build.build()
    r = _child(["-c", "import sys; sys.path.insert(0, '.'); sys.path.insert(0, 'tests')\n" + PROBE], 600)
    assert r.returncode == 0 and "checked build ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]


def test_parity_suites_on_the_checked_build():
    r = _child(["-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "tests/test_gpu_parity.py",
                "tests/test_gpu_multi.py", "tests/test_gpu_sim.py", "-k",
                "not full_ and not serving and not bandwidth and not autotuned"], 1500)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
