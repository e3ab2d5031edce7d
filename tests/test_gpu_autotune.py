"""The autotuner times real candidates, stores the winner per size class, round-trips JSON."""
import json

import numpy as np
import pytest

import oracle
from gpu_util import assert_same, gpu_assemble, to_dev
from paper_1406_1066_gb300 import fsparse, inputs

pytestmark = pytest.mark.gpu


def test_autotune_roundtrip(tmp_path):
    t = inputs.mesh3d(14, 5)
    fsparse.fsparse_tune_clear()
    best = fsparse.autotune(to_dev(t.ii), to_dev(t.jj), to_dev(t.s), t.m, t.n, reps=1)
    assert fsparse.fsparse_get_config(t.L, t.m, t.n) == best
    path = tmp_path / "tune.json"
    fsparse.fsparse_tune_save(str(path))
    assert len(json.loads(path.read_text())["entries"]) == 1
    fsparse.fsparse_tune_clear()
    fsparse.fsparse_tune_load(str(path))
    assert fsparse.fsparse_get_config(t.L, t.m, t.n) == best
    g = gpu_assemble(t.ii, t.jj, t.s, t.m, t.n)   # the tuned configuration is still exact
    assert_same(g, oracle.assemble(t.ii, t.jj, t.s, t.m, t.n))
    fsparse.fsparse_tune_clear()
