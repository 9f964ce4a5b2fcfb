"""Host-side statistics of recorded delay traces (the paper's delays,
Section 3, summarised as histograms, means and lag-1 autocorrelations),
checked on traces whose statistics are known by construction."""
from __future__ import annotations

import numpy as np

from paper_1510_08982_gb300 import experiments, inputs


def test_delay_statistics_on_constructed_traces():
    # one boundary; side 0 alternates 0, 2, 0, 2 and side 1 is 1, 1, 2, 2
    tr = np.array([[[0, 1]], [[2, 1]], [[0, 2]], [[2, 2]]], dtype=np.uint8)
    st = experiments.delay_statistics(tr, 3)
    assert st["histogram"].tolist() == [2, 2, 4]
    assert st["per_side"].tolist() == [[2, 0, 2], [0, 2, 2]]
    assert abs(st["mean"] - 10 / 8) < 1e-15
    # side 0: x = -1, 1, -1, 1: sum x_k x_{k-1} = -3, sum x^2 = 4 -> -0.75
    # side 1: x = -.5, -.5, .5, .5: products .25, -.25, .25 -> .25, sum x^2 = 1 -> 0.25
    assert abs(st["lag1_autocorrelation"] - (-0.75 + 0.25) / 2) < 1e-15


def test_delay_statistics_of_iid_delays():
    """Seeded i.i.d. uniform delays: flat histogram, mean (q-1)/2, no lag-1
    correlation (within a few standard errors 1/sqrt(K))."""
    K, S, q = 20000, 5, 4
    st = experiments.delay_statistics(inputs.delay_trace(K, S, q, seed=3), q)
    n = K * (S - 1) * 2
    assert np.all(np.abs(st["histogram"] / n - 1 / q) < 0.01)
    assert abs(st["mean"] - (q - 1) / 2) < 0.02
    assert abs(st["lag1_autocorrelation"]) < 4 / np.sqrt(K)


def test_delay_statistics_ignores_constant_sequences():
    """A side whose delay never changes has no defined correlation and is left
    out of the average."""
    tr = np.zeros((6, 2, 2), dtype=np.uint8)
    tr[:, 1, 0] = [0, 1, 0, 1, 0, 1]
    st = experiments.delay_statistics(tr, 2)
    x = np.array([-.5, .5, -.5, .5, -.5, .5])
    assert abs(st["lag1_autocorrelation"] - (x[1:] * x[:-1]).sum() / (x * x).sum()) < 1e-15
