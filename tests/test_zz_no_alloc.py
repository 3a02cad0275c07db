"""lbm_reduce_noalloc: the reduction entry point for callers that cannot
allocate device memory (its scratch is a static device array inside the
library).  It must return what lbm_reduce returns, call after call, on the
same bound state, bit for bit (the same kernels run in the same order).
This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    from paper_1601_06984_gb300 import build, lbm as L
    build.build()
    return L


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_lbm_reduce_on_two_calls(lbm, precision):
    from paper_1601_06984_gb300 import workloads as W
    m = W.config_sphere_small()
    om = W.omega_coarse_from_finest(1.6, 3)
    s = lbm.Sim(m, 19, om, precision=precision, u_in=(0.04, 0, 0))
    s.init(*W.uniform_fields(m, 1.0, (0.04, 0.0, 0.0)), W.pdf_perturbation(m, 19, 1e-4))
    s.step(2)
    ref = s.reduce()
    first = lbm.lbm_reduce_noalloc(s)
    second = lbm.lbm_reduce_noalloc(s)
    # the same kernels in the same order on the same state: bit for bit equal
    assert np.array_equal(first, ref) and np.array_equal(second, ref)
    assert ref[4] != 0.0  # the sphere's drag is part of the comparison
    # the state moves on; the static scratch must not keep the old result
    s.step(1)
    ref2 = s.reduce()
    third = lbm.lbm_reduce_noalloc(s)
    assert np.array_equal(third, ref2)
    assert not np.array_equal(ref2, ref)


def test_noalloc_rejects_deeper_hierarchies(lbm):
    from paper_1601_06984_gb300 import workloads as W
    # nine levels: each level refines the central half of the previous one
    boxes, lo = [], 0
    for k in range(8):
        lo = 2 * (lo + 8)
        boxes.append(((lo, lo), (lo + 32, lo + 32)))
    m = W.nested_boxes(2, 5, (32, 32), boxes, (0, 0, 0, 0))
    s = lbm.Sim(m, 9, 1.9, precision=lbm.FP64)
    s.init(*W.uniform_fields(m))
    assert len(s.mesh_info()) == 9
    with pytest.raises(lbm.LBMError, match="at most 8"):
        lbm.lbm_reduce_noalloc(s)
    assert np.isfinite(s.reduce()).all()
