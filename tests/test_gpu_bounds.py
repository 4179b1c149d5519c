"""The bounds-check build: every index of the step kernels stays within its extent.

The library is built a second time with -DAHS_BOUNDS_CHECK (_ahs_check.so).  There
every global offset of the step kernels' tile loaders, rings and stores, and every
shared-memory index of their tiles, is checked against the extent it addresses; an
index outside it is counted and replaced by 0, so no access leaves its array and no
kernel traps.  A fresh process (bounds_check_run.py) runs every step path -- plain
and measuring steps of the one-site and paired kernels, both tile heights, short
and ragged z-chunks, in-place momenta with the Gauss pre-pass, compensated and FP64
precision, two steps per pass, a batch, the winding field and the allocation-free
measurement -- on sides smaller than a tile, odd and even (4, 5, 7, 65, 66), and
expects the count to stay zero; a self-test then shows the counter counts.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_no_index_leaves_its_extent():
    from paper_2005_14454_gb300 import build
    lib = build.build(variant="check")
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_check_run.py"), lib],
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["paths"] >= 40
    assert res["errors"] == 0, res
    assert res["selftest"] == 2, res      # one counted index per kernel translation unit
