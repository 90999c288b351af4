"""Pins of the oracle's bath correlation, G(t) and QUAPI coefficients (App. B.1)."""
import numpy as np
import pytest

from workloads import BathSpec
from oracle import bath

BATHS = [BathSpec(0.1, 4.0, 1.0), BathSpec(0.16, 4.0, 5.0), BathSpec(0.16, 4.0, 0.5),
         BathSpec(0.05, 3.0, 0.8), BathSpec(0.2, 2.0, 0.0)]


@pytest.mark.parametrize("b", BATHS)
@pytest.mark.parametrize("t", [0.05, 0.7, 2.5])
def test_G_closed_form_matches_quadrature(b, t):
    # G(t) = double time integral of C, written in frequency space and integrated adaptively.
    assert abs(bath.G_closed(b, t) - bath.G_quad(b, t)) < 1e-9


@pytest.mark.parametrize("b", BATHS[:4])
def test_G_second_derivative_is_C(b):
    # C(tau) (App. B.1, by quadrature of its definition) is the second derivative of G.
    h = 1e-3
    for tau in [0.3, 1.1]:
        d2 = (bath.G_closed(b, tau + h) - 2 * bath.G_closed(b, tau) + bath.G_closed(b, tau - h)) / h ** 2
        c = bath.correlation_quad(b, tau)
        assert abs(d2 - c) < 2e-5 * max(1.0, abs(c))


def test_G_at_zero_and_small_t():
    # G(0) = 0 and G(t) ~ C(0) t^2 / 2 for small t.
    b = BATHS[0]
    assert abs(bath.G_closed(b, 0.0)) < 1e-15
    t = 1e-4
    c0 = bath.correlation_quad(b, 0.0)
    assert abs(bath.G_closed(b, t) / (t * t / 2) - c0) < 1e-3 * abs(c0)


@pytest.mark.parametrize("b", BATHS)
def test_eta_sum_telescopes_to_G(b):
    # sum_{1<=k'<=k<=K} eta_{k-k'} = G(K dt): the identity that makes pure dephasing exact.
    dt, K = 0.1, 37
    eta = bath.eta_coefficients(b, dt, K)
    s = K * eta[0] + sum((K - D) * eta[D] for D in range(1, K))
    assert abs(s - bath.G_closed(b, K * dt)) < 1e-11 * max(1, abs(s))


def test_single_mode_G_matches_quadrature_of_its_C():
    g2, w0, T = 0.49, 1.3, 0.8
    import scipy.integrate as si
    coth = 1 / np.tanh(w0 / (2 * T))

    def C(u):
        return g2 * (coth * np.cos(w0 * u) - 1j * np.sin(w0 * u))

    t = 1.7
    re = si.dblquad(lambda u, s: C(u).real, 0, t, 0, lambda s: s)[0]
    im = si.dblquad(lambda u, s: C(u).imag, 0, t, 0, lambda s: s)[0]
    assert abs(bath.single_mode_G(g2, w0, T, t) - (re + 1j * im)) < 1e-10


def test_gaussian_cutoff_G_quad_is_consistent():
    # The Gaussian cutoff (the paper's own choice) has no closed form here; G by quadrature must
    # still satisfy G'' = C.
    b = BathSpec(0.32, 4.0, 1.6, "gaussian")
    h = 2e-3
    tau = 0.5
    d2 = (bath.G_quad(b, tau + h) - 2 * bath.G_quad(b, tau) + bath.G_quad(b, tau - h)) / h ** 2
    assert abs(d2 - bath.correlation_quad(b, tau)) < 1e-4 * abs(bath.correlation_quad(b, 0.0))
