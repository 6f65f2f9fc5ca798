"""Pins of the shared weight of several orbital pairs (k-points on one grid):
for SSM it is the weight of the concatenated orbital sets (Eq. weight function
2 summed over all columns), for one pair it is that pair's weight, and it is
the sum of the pairs' weights in any grouping up to rounding."""
import numpy as np

import oracle as O
from paper_2208_07731_gb300 import workload as W


def _pairs(count, n_orb=4):
    out = []
    for b in range(count):
        w = W.small_workload(n=8, L=6.0, n_orb=n_orb, n_mu=16, iters=1, ecut=6.0, seed=40 + b)
        out.append(tuple(x.numpy() for x in W.make_pair(w)))
    return out


def test_shared_ssm_weight_is_the_concatenated_sets_weight():
    pairs = _pairs(3)
    phi = np.concatenate([p for p, _ in pairs], axis=1)
    psi = np.concatenate([q for _, q in pairs], axis=1)
    for alpha in (1.0, 2.0, 3.0):
        np.testing.assert_allclose(O.shared_weights(pairs, "ssm", alpha), O.weights(phi, psi, "ssm", alpha),
                                   rtol=1e-14)


def test_one_pair_is_its_own_weight():
    pairs = _pairs(1)
    assert np.array_equal(O.shared_weights(pairs, "psm"), O.weights(*pairs[0], "psm"))


def test_order_changes_only_rounding():
    pairs = _pairs(4)
    a = O.shared_weights(pairs)
    b = O.shared_weights(pairs[::-1])
    np.testing.assert_allclose(a, b, rtol=1e-15)
