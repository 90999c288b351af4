"""Fluctuation and dissipation spectra of a steady-state two-time correlation (test infrastructure).

ORACLE: imported only by tests/, __graft_entry__.smoke() and bench.py's CPU baseline; never by the
product path.

Input: C(tau_k) = <A(tau_k) A(0)>_ss for tau_k = k dt, k = 0..n, A Hermitian, in a stationary state,
as obtained by branching the full augmented MPS at t_ss with the left super-operator A. and
propagating (App. B.2).
Stationarity gives <A(-tau) A(0)> = conj(C(tau)), so on (-tau_max, tau_max):
  anticommutator  (1/2)<{A(tau), A(0)}> = Re C(|tau|)                     (even in tau)
  commutator      <[A(tau), A(0)]>      = 2 i sign(tau) Im C(|tau|)        (odd in tau)
and, with the Fourier convention f(w) = int dtau e^{i w tau} f(tau) (Sec. III.A.2, Eqs. for the FDT
and the effective temperature):
  S(w)      = FT[(1/2)<{A(tau), A(0)}>](w)
  chi''(w)  = Im FT[i Theta(tau) <[A(tau), A(0)]>](w) = (1/2) FT[<[A(tau), A(0)]>](w)   (real)
  T(w)      = w / (2 artanh(chi''(w) / S(w)))
This module writes those definitions out as trapezoid-rule sums over the sampled interval,
evaluated at each requested frequency by a plain loop (no FFT), so that the product's FFT routine
can be checked against it; parity unpinned against the paper's own spectra (its figures are absent).
"""
from __future__ import annotations

import numpy as np


def _weights(n):
    """Trapezoid weights for tau_k, k = -n..n (end points half weight)."""
    w = np.ones(2 * n + 1)
    w[0] = w[-1] = 0.5
    return w


def symmetric_samples(C):
    """tau index k = -n..n and the anticommutator / commutator samples on it."""
    C = np.asarray(C, dtype=complex)
    n = len(C) - 1
    k = np.arange(-n, n + 1)
    Cabs = C[np.abs(k)]
    anti = Cabs.real
    comm = 2j * np.sign(k) * Cabs.imag
    return k, anti, comm


def spectra(C, dt, omegas):
    """(S(w), chi''(w), T(w)) at the given frequencies, by direct trapezoid sums."""
    k, anti, comm = symmetric_samples(C)
    wts = _weights((len(k) - 1) // 2)
    tau = k * dt
    S = np.zeros(len(omegas))
    chi2 = np.zeros(len(omegas))
    for i, w in enumerate(omegas):
        ph = np.exp(1j * w * tau)
        S[i] = (dt * np.sum(wts * ph * anti)).real
        chi2[i] = (0.5 * dt * np.sum(wts * ph * comm)).real
    with np.errstate(divide="ignore", invalid="ignore"):
        T = np.asarray(omegas) / (2.0 * np.arctanh(chi2 / S))
    return S, chi2, T
