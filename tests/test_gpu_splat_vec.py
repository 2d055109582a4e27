"""The splat's other load form (16-byte depth loads, eight consecutive source
pixels per lane, kept for measurements and chosen by FVV_SPLAT_VEC=1 when
the library loads) against the oracle.  The switch is read once per process,
so the check runs in a child process.  The 333 x 187 cameras leave a ragged
vector at the end of every row; the layered form takes the same loads."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

_CHILD = r"""
import sys
sys.path[:0] = [{root!r}, {tests!r}]
import oracle
import synthetic as S
from fvv_helpers import assert_parity, gpu_run, lib
oracle.build()
wl = S.workload("plain_9cam_1280x720", scale=0.26)
views = [wl["views"][i] for i in (20, 140, 260)]
gs = gpu_run(wl["cams"], wl["rgb"], wl["depth"], views, wl["look_at"])
for g, v in zip(gs, views):
    assert_parity(g, oracle.synthesize(wl["cams"], wl["rgb"], wl["depth"], v, wl["look_at"]), "vector splat")
print("ok", len(gs))
"""


def test_vector_splat_matches_the_oracle(oracle_mod):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    tests = os.path.dirname(os.path.abspath(__file__))
    env = dict(os.environ, FVV_SPLAT_VEC="1")
    r = subprocess.run([sys.executable, "-c", _CHILD.format(root=root, tests=tests)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert r.stdout.strip().endswith("ok 3")
