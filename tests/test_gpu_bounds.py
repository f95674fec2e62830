"""Memory safety of every kernel, checked by the bounds-checked build
(libtlbm_debug.so, TLBM_DEBUG_BOUNDS): the cases of bounds_cases.py run on it
in a child process, where every global load and store of the step, in-place,
staged, batch, transfer, initial-state and reduction kernels is checked against
the handle's population buffers.  No access may leave them, and the checked
build must compute bitwise what the release build computes."""
import json
import os
import subprocess
import sys

import pytest

import bounds_cases

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def T():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_03160_gb300 import tlbm

    tlbm.lib()
    return tlbm


def test_no_kernel_access_leaves_the_population_buffers(T, tmp_path):
    out = tmp_path / "debug.json"
    env = dict(os.environ, TLBM_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_cases.py"), str(out)], env=env,
                       capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    dbg = json.loads(out.read_text())
    rel = bounds_cases.run(T, str(tmp_path))
    assert set(dbg) == set(rel)
    assert all(v["violations"] is not None for v in dbg.values()), "the child did not load the checked build"
    assert all(v["violations"] is None for v in rel.values())
    bad = {k: v["violations"] for k, v in dbg.items() if v["violations"] != 0}
    assert not bad, bad
    differ = [k for k in rel if rel[k]["hash"] != dbg[k]["hash"] or rel[k]["red"] != dbg[k]["red"]]
    assert not differ, differ
    assert len(rel) > 250
