"""Host logic of the hybrid field optimisation (Sec. 3.4) and pins for the oracle's Adam
and geometric loss.  CPU only."""
import numpy as np

import oracle
from paper_2602_06991_b300.hybrid import HybridSchedule


def test_schedule_pattern():
    s = HybridSchedule(4)
    assert [s.is_semantic(i) for i in range(8)] == [False, False, False, True] * 2
    assert HybridSchedule(1).is_semantic(0) and HybridSchedule(1).semantic_fraction() == 1.0
    assert s.semantic_fraction() == 0.25


def test_adam_first_steps_closed_form():
    """With bias correction, a constant gradient g gives m_hat = g and v_hat = g^2 at every
    step, so each step moves p by lr g / (|g| + eps) -- the sign step of Adam."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p = np.array([1.0, 1.0, 1.0, 1.0])
    m = v = np.zeros(4)
    lr, eps = 0.01, 1e-8
    for t in (1, 2, 3):
        p2, m, v = oracle.adam_step(p, g, m, v, lr, 0.9, 0.999, eps, t)
        np.testing.assert_allclose(p2, p - lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)
        p = p2
    np.testing.assert_allclose(m, (1 - 0.9 ** 3) * g, rtol=1e-12)


def test_loss_geo_closed_form():
    C = np.array([[0.5, 0.5, 0.5], [0.0, 1.0, 0.2]])
    Cgt = np.array([[0.5, 0.4, 0.7], [0.1, 1.0, 0.1]])
    D, Dgt = np.array([2.0, 3.0]), np.array([2.5, 3.0])
    loss, dC, dD = oracle.loss_geo(C, Cgt, D, Dgt, 1.0, 0.5)
    np.testing.assert_allclose(loss, ((0.0 + 0.1 + 0.2) / 3 + 0.5 * 0.5 + (0.1 + 0.0 + 0.1) / 3 + 0.0) / 2, rtol=1e-14)
    np.testing.assert_array_equal(np.sign(dC), [[0, 1, -1], [-1, 0, 1]])
    np.testing.assert_array_equal(dD, [-0.25, 0.0])
