"""Pins of the oracle's relative-binning likelihood: exact at the fiducial and with one
frequency per bin, second-order convergence of its error in the bin width."""
import numpy as np
import pytest

import oracle
import workloads
from oracle.events import make_event
from workloads import MC, Q, CHI1, TC


@pytest.fixture(scope="module")
def event():
    w = workloads.tiny()
    spec = w.events[0]
    ev, th, _ = make_event(w, spec)
    return w, ev, th


def edges_every(n_bins, width):
    e = list(range(0, n_bins, width))
    return np.array(e + [n_bins], dtype=np.int32)


def nearby(th, scale):
    p = np.tile(th, (4, 1))
    p[0, MC] *= 1 + 2e-3 * scale
    p[1, Q] *= 1 - 3e-2 * scale
    p[2, CHI1] += 0.05 * scale
    p[3, MC] *= 1 - 1e-3 * scale
    p[3, TC] += 2e-4 * scale
    return p


def test_exact_at_the_fiducial_and_with_one_frequency_per_bin(event):
    w, ev, th = event
    exact = oracle.loglike_batch(ev, nearby(th, 1.0))
    one = oracle.rb_loglike_batch(ev, th, edges_every(w.n_bins, 1), nearby(th, 1.0))
    assert np.allclose(one, exact, rtol=1e-11, atol=1e-9)
    at0 = oracle.rb_loglike_batch(ev, th, edges_every(w.n_bins, 64), th[None, :])
    assert at0[0] == pytest.approx(oracle.loglike(ev, th), rel=1e-11, abs=1e-9)


def test_error_falls_with_the_square_of_the_bin_width(event):
    """The chord of a smooth ratio deviates from it by O(width^2): halving the bins cuts the
    error of the overlap by ~4 (and the same offsets cost less close to the fiducial)."""
    w, ev, th = event
    pars = nearby(th, 1.0)
    exact = oracle.loglike_batch(ev, pars)
    err = {}
    for width in (64, 32, 16):
        err[width] = np.abs(oracle.rb_loglike_batch(ev, th, edges_every(w.n_bins, width), pars) - exact)
    for i in range(len(pars)):
        assert err[64][i] > 1e-7
        assert 2.5 < err[64][i] / err[32][i] < 6.0 and 2.5 < err[32][i] / err[16][i] < 6.0
    closer = np.abs(oracle.rb_loglike_batch(ev, th, edges_every(w.n_bins, 64), nearby(th, 0.5)) -
                    oracle.loglike_batch(ev, nearby(th, 0.5)))
    assert np.all(closer < err[64])
