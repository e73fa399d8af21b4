"""C-ABI checks that need no GPU: the library loads, exports every function
include/hz.h declares, validates arguments, and its host-side geometry
(GLL node positions) matches the oracle's."""

import os
import re
import subprocess

import numpy as np
import pytest

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "hz.h")).read()
    return sorted(set(re.findall(r"^HZ_API\s+\w+\s+(hz_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_symbol():
    import paper_2606_21695_gb300 as hz

    path = hz.library_path()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(hz_\w+)$", out, flags=re.M))
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = [n for n in declared if n not in exported]
    assert not missing, missing
    assert sorted(hz.exported_names()) == declared


def test_mesh_validation_errors():
    import paper_2606_21695_gb300 as hz

    with pytest.raises(hz.HzError) as e:
        hz.hz_mesh_create(0, 1, 0, 1, 10, 10, 2, 3, 5)  # 3 does not divide 10
    assert e.value.status == hz.HZ_ERR_INVALID_ARG
    with pytest.raises(hz.HzError):
        hz.hz_mesh_create(0, 1, 0, 1, 8, 8, 0, 4, 4)  # degree 0
    with pytest.raises(hz.HzError):
        hz.hz_mesh_create(0, 1, 0, 1, 8, 8, 8, 4, 4)  # degree beyond the compiled range
    with pytest.raises(hz.HzError):
        hz.hz_mesh_create(1, 0, 0, 1, 8, 8, 2, 4, 4)  # empty box
    with pytest.raises(hz.HzError):
        hz.hz_mesh_create(0, float("nan"), 0, 1, 8, 8, 2, 4, 4)


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 6, 7])
def test_node_coordinates_match_oracle(P):
    import paper_2606_21695_gb300 as hz
    from oracle import sem

    box = (-0.5, 1.5, 0.25, 1.0)
    m = hz.hz_mesh_create(*box, 6, 4, P, 3, 2)
    try:
        assert hz.hz_mesh_num_nodes(m) == (6 * P + 1) * (4 * P + 1)
        xy = hz.hz_mesh_node_coords(m)
    finally:
        hz.hz_mesh_destroy(m)
    om = sem.Mesh(*box, 6, 4, P, 3, 2)
    X, Y = om.coords()
    np.testing.assert_allclose(xy[:, 0], X.ravel(), rtol=0, atol=1e-15)
    np.testing.assert_allclose(xy[:, 1], Y.ravel(), rtol=0, atol=1e-15)


def test_problem_create_without_device_fails_cleanly():
    import torch

    import paper_2606_21695_gb300 as hz

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    m = hz.hz_mesh_create(0, 1, 0, 1, 4, 4, 2, 2, 2)
    try:
        with pytest.raises(hz.HzError) as e:
            hz.hz_problem_create(m, 0)
        assert e.value.status in (hz.HZ_ERR_CUDA, hz.HZ_ERR_INVALID_ARG)
    finally:
        hz.hz_mesh_destroy(m)
