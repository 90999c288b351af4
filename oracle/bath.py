"""Bath correlation function and QUAPI memory coefficients (oracle).

App. B.1 defines the bath auto-correlation
    C(tau) = int_0^inf J(w) [cos(w tau) coth(w / 2T) - i sin(w tau)] dw
for a Gaussian bosonic bath with spectral density J(w) (Eq. (bosonic-bath)). The paper gives no
discretisation; the oracle uses the quasi-adiabatic path-integral coefficients of the PT-TEMPO
literature it cites: with G(t) = int_0^t ds int_0^s du C(u),
    eta_0 = G(dt),   eta_D = G((D+1) dt) - 2 G(D dt) + G((D-1) dt)   (D >= 1),
so that sum_{1 <= k' <= k <= K} eta_{k-k'} = G(K dt) exactly.

For J(w) = 2 alpha w exp(-w/w_c) both integrals have closed forms (derived by expanding coth as a
geometric series and summing with the Gamma-function product formula):
    G(t) = 2 alpha [ln(1 + i w_c t) - i w_c t] + 2 alpha ln( Gamma(1+T/w_c)^2 / |Gamma(1+T/w_c+iTt)|^2 )
The tests pin this against adaptive quadrature of the defining integrals.
"""
from __future__ import annotations

import numpy as np
import scipy.integrate as si
from scipy.special import loggamma


def spectral_density(bath, w):
    w = np.asarray(w, dtype=float)
    if bath.cutoff == "exponential":
        return 2 * bath.alpha * w * np.exp(-w / bath.omega_c)
    if bath.cutoff == "gaussian":
        return 2 * bath.alpha * w * np.exp(-(w / bath.omega_c) ** 2)
    raise ValueError(bath.cutoff)


def _coth_weight(w, T):
    """coth(w / 2T), with the T -> 0 limit 1."""
    if T == 0:
        return np.ones_like(w)
    return 1.0 / np.tanh(w / (2 * T))


def correlation_quad(bath, tau, wmax_factor=60.0):
    """C(tau) by adaptive quadrature of its definition (App. B.1)."""
    wmax = wmax_factor * bath.omega_c

    def re(w):
        return spectral_density(bath, w) * np.cos(w * tau) * _coth_weight(w, bath.T)

    def im(w):
        return -spectral_density(bath, w) * np.sin(w * tau)

    lim = 2000
    a = si.quad(re, 0, wmax, limit=lim, epsabs=1e-13, epsrel=1e-12)[0]
    b = si.quad(im, 0, wmax, limit=lim, epsabs=1e-13, epsrel=1e-12)[0]
    return a + 1j * b


def G_quad(bath, t, wmax_factor=60.0):
    """G(t) = int_0^inf J(w)/w^2 [coth(w/2T)(1 - cos wt) - i (wt - sin wt)] dw, by quadrature.

    This is the double time integral of C written in frequency space (exchange of integrals)."""
    wmax = wmax_factor * bath.omega_c

    def re(w):
        return spectral_density(bath, w) / w ** 2 * _coth_weight(w, bath.T) * (1 - np.cos(w * t))

    def im(w):
        return -spectral_density(bath, w) / w ** 2 * (w * t - np.sin(w * t))

    lim = 4000
    a = si.quad(re, 1e-300, wmax, limit=lim, epsabs=1e-13, epsrel=1e-12)[0]
    b = si.quad(im, 1e-300, wmax, limit=lim, epsabs=1e-13, epsrel=1e-12)[0]
    return a + 1j * b


def G_closed(bath, t):
    """Closed form of G(t) for the exponential cutoff (see module docstring)."""
    if bath.cutoff != "exponential":
        raise ValueError("closed form only for the exponential cutoff")
    a, wc, T = bath.alpha, bath.omega_c, bath.T
    t = np.asarray(t, dtype=float)
    g = 2 * a * (np.log(1 + 1j * wc * t) - 1j * wc * t)
    if T > 0:
        x0 = 1.0 + T / wc
        g = g + 2 * a * (2 * loggamma(x0).real - 2 * loggamma(x0 + 1j * T * t).real)
    return g


def G_function(bath, t):
    if bath.cutoff == "exponential":
        return G_closed(bath, t)
    return np.array([G_quad(bath, float(x)) for x in np.atleast_1d(t)])


def eta_coefficients(bath, dt, n_memory):
    """eta_0 ... eta_{n_memory} (QUAPI memory coefficients, see module docstring)."""
    ts = np.arange(0, n_memory + 2) * dt
    G = G_function(bath, ts)
    eta = np.empty(n_memory + 1, dtype=complex)
    eta[0] = G[1]
    for D in range(1, n_memory + 1):
        eta[D] = G[D + 1] - 2 * G[D] + G[D - 1]
    return eta


def memory_steps(bath, dt, K, rel=1e-3):
    """Delta K: the number of steps after which |C(tau)| stays below rel * max|C| (App. B.1)."""
    taus = np.arange(0, K + 1) * dt
    c = np.array([abs(correlation_quad(bath, t)) for t in taus])
    above = np.nonzero(c >= rel * c.max())[0]
    return int(min(K, above.max() + 1)) if len(above) else 1


def single_mode_G(g2, w0, T, t):
    """G(t) for one harmonic mode, J(w) = g2 delta(w - w0) (used by the exact single-mode pin)."""
    coth = 1.0 if T == 0 else 1.0 / np.tanh(w0 / (2 * T))
    t = np.asarray(t, dtype=float)
    return g2 / w0 ** 2 * (coth * (1 - np.cos(w0 * t)) - 1j * (w0 * t - np.sin(w0 * t)))


def eta_from_G(G_of_t, dt, n_memory):
    ts = np.arange(0, n_memory + 2) * dt
    G = G_of_t(ts)
    eta = np.empty(n_memory + 1, dtype=complex)
    eta[0] = G[1]
    for D in range(1, n_memory + 1):
        eta[D] = G[D + 1] - 2 * G[D] + G[D - 1]
    return eta
