"""dg_apply_sumfact_static: the operator with its face-trace scratch in libtpp's
static device array, for callers that cannot allocate device scratch.

Its output is compared with dg_apply_sumfact on two calls in a row (the static
array keeps the previous call's contents), and a problem larger than the
array is rejected.  Collected last so that a failure here comes after every
other test has run."""
import numpy as np
import pytest

import synthetic
from tests.gpu_util import make_pair, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,nel,h", [(16, (4, 4), 1.0), (31, (64, 64), 1.0), (5, (3, 5), 1.0 / 3)])
def test_static_scratch_operator_matches(n, nel, h):
    ctx, dg = make_pair(n, nel, 0.05, synthetic.fourier_velocity(1705, 2), h=h, max_restart=2)
    for seed in (11, 12):                 # two calls in a row, different inputs
        x = to_dev(synthetic.rhs(seed, dg.ndof))
        y_ref = to_host(ctx.dg_apply_sumfact(x))
        y = to_host(ctx.dg_apply_sumfact_static(x))
        # same tolerance as the operator parity tests
        assert rel(y, y_ref) <= 1e-12
        assert np.abs(y - y_ref).max() <= 1e-11 * np.abs(y_ref).max()


def test_static_scratch_rejects_oversize():
    from paper_1704_04549_gb300 import TppError
    # 128 x 64 elements at n = 32: 8192 * 4 * 32 = 1,048,576 trace values > 524,288
    ctx, dg = make_pair(32, (128, 64), 0.05, synthetic.constant_velocity([1.0, 0.5]), h=1.0,
                        max_restart=1)
    x = to_dev(np.ones(dg.ndof))
    with pytest.raises(TppError, match="static scratch"):
        ctx.dg_apply_sumfact_static(x)
