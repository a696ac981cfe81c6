"""The bounds-checked build (-DMG_CHECKED; libmg_checked.so) on small grids
against the oracle.  In that build every device index the kernels take from a
host table (the messenger constants' row ranges and offsets, the shell id of
each |m|^2) is compared with its buffer before use; a violation would skip the
access and surface as MG_EBOUNDS.  The run happens in a fresh process with
MG_CHECKED=1 so that the binding loads the checked library; it must finish
with parity at the usual tolerances and no status raised."""
import json
import os
import subprocess
import sys

import pytest

from gpu_helpers import TOL, need_gpu

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_matches_the_oracle_with_no_bounds_fault():
    need_gpu()  # builds both libraries
    env = dict(os.environ, MG_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_build_child.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["library"] == "libmg_checked.so"
    for key, err in res.items():
        if key == "library":
            continue
        tol = TOL[32] if key.endswith("_32") else TOL[64]
        assert err <= tol, (key, err)
