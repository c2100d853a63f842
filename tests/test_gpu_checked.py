"""The checked library variant (compiled with FEM_CHECKED): the kernels check
element ids taken from permutations and the output offsets of mixed-degree
plans against their extents, skip a failing access and report FEM_ECHECKED.
Runs in a child process that loads libfem_gb300_checked.so; a plan whose
output bound the test hook shortens by one value has its last block refused,
every other element still matches the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_mixed_plans():
    import torch
    from paper_1310_1191_gb300 import build
    assert torch.cuda.is_available()
    build.build(checked=True)
    env = dict(os.environ, FEM_GB300_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "_checked_child.py")], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert r.stdout.strip().splitlines()[-1] == "OK 4", r.stdout[-2000:]


def test_shrink_hook_refused_by_normal_build():
    import torch
    from paper_1310_1191_gb300 import _lib, build, inputs
    assert torch.cuda.is_available()
    build.build()
    _lib.load()
    assert os.path.basename(_lib._lib._name) == "libfem_gb300.so"
    t = _lib.fem_tables_build(_lib.FEM_PRISM6, 1, 3)
    plan = _lib.fem_plan_create(t, inputs.mixed_degrees(16).clip(1, 3), _lib.FEM_F64)
    with pytest.raises(_lib.FemError) as ei:
        _lib.fem_debug_shrink_bound(plan)
    assert ei.value.code == _lib.FEM_EUNSUPPORTED
    plan.close()
    t.close()
