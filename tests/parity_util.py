"""Comparison of one CompaSO result with the CPU oracle (test helper).

Integer outputs (kernel sums, labels, nucleus ids, sizes, R^2) must be
identical; the FP64 centres of mass and R_Delta within 1e-9 relative."""
import numpy as np

import oracle as O

BOX = 1 << 21


def assert_matches_oracle(res, pos, ids, u, **kw):
    """res: outputs of one request (numpy dict with sigma, l0, l1, l2, halos)
    for the particles (pos, ids); the oracle runs on the same input."""
    o = O.find_groups(pos, ids, O.params(u, **kw))
    for k in ("sigma", "l0", "l1", "l2"):
        a, b = res[k], o[k]
        if not np.array_equal(a, b):
            bad = np.nonzero(a != b)[0]
            raise AssertionError("%s differs from the oracle at %d of %d entries" % (k, bad.size, a.size))
    H, Ho = res["halos"], o["halos"]
    assert len(H) == len(Ho), (len(H), len(Ho))
    for f in ("nucleus_id", "N", "R2", "l2max_id", "l2max_N", "l2_top5_N", "n_l2", "l0_id"):
        assert np.array_equal(H[f], Ho[f]), f
    for f in ("com", "l2max_com", "R_delta"):
        np.testing.assert_allclose(H[f], Ho[f], rtol=1e-9, atol=1e-9 * BOX)
    return o
