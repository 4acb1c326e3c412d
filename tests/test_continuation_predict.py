"""The library's continuation predictor (host code, no GPU) takes the same decisions and
weights as the oracle's reading of Sec. 4.3."""
import numpy as np
import pytest

from oracle import continuation as ct


@pytest.fixture(scope="module")
def predict():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_16635_gb300.rsc import continuation_predict
    return continuation_predict


def test_matches_oracle_on_random_histories(predict):
    rng = np.random.default_rng(7)
    modes = set()
    for trial in range(400):
        k = 2 + trial % 2
        Ra = list(100.0 + np.cumsum(rng.uniform(-3, 3, k))[::-1])
        s = list(rng.uniform(0.1, 2.0) + rng.normal(0, 0.3, k))
        its = int(rng.integers(1, 9))
        gamma = float(rng.choice([0.5, 5.0, 50.0]))
        scale = float(rng.choice([1.0, 0.5, 0.25]))
        m0, r0, w0 = ct.predict(Ra, s, its, 4, gamma, scale)
        m1, r1, w1 = predict(Ra, s, its, 4, gamma, scale)
        modes.add(m1)
        assert m0 == m1
        assert abs(r0 - r1) <= 1e-12 * abs(r0)
        assert np.allclose(w0, w1, rtol=1e-12, atol=1e-12)
    assert modes == {0, 1}


def test_rejects_a_single_point(predict):
    from paper_2508_16635_gb300 import RscError
    with pytest.raises(RscError):
        predict([100.0], [1.0], 3, 4, 20.0)
