"""Host-side checks of the mixed-degree batch inputs (no GPU)."""
import numpy as np

import synthetic


def test_mixed_degree_groups_generator():
    """The mixed-degree batch: degrees in range, every element in exactly one group."""
    groups = synthetic.mixed_degree_batch(e2d=500, e3d=60)
    ids = np.sort(np.concatenate([g.ids for g in groups]))
    assert np.array_equal(ids, np.arange(560))
    for g in groups:
        assert (g.dim == 2 and 5 <= g.n <= 31) or (g.dim == 3 and 4 <= g.n <= 13)
        assert g.centres.shape == (len(g.ids), g.dim)
        assert np.all((g.centres >= 0) & (g.centres < 1))
