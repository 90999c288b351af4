"""Branching two-time correlations and the fluctuation / dissipation spectra of a steady state.

The procedure of App. B.2: evolve the full augmented MPS (chain and environment correlations) to
t_ss, branch it, apply the left super-operator A. (or the right one .A) to the branch on one
site, and propagate the branch; the raw readout of B on the branch is
    C(tau) = Tr[B e^{L tau}(A rho(t_ss))] = <B(t_ss + tau) A(t_ss)>   (left)
    C(tau) = Tr[B e^{L tau}(rho(t_ss) A)] = <A(t_ss) B(t_ss + tau)>   (right),
never divided by the trace (two-time correlations are not trace-normalised). The branch is a clone
of the engine on the device (pt_tebd_clone), so the original continues undisturbed.

The spectra follow Sec. III.A.2: with A = B Hermitian and stationarity, C(-tau) = conj(C(tau)), so
the anticommutator (1/2)<{A(tau), A(0)}> = Re C(|tau|) and the commutator
<[A(tau), A(0)]> = 2i sign(tau) Im C(|tau|) are known on (-tau_max, tau_max). With
f(w) = int dtau e^{i w tau} f(tau) (trapezoid rule on the samples, zero padded, one FFT):
    S(w) = FT[anticommutator],  chi''(w) = (1/2) FT[commutator],  T(w) = w / (2 artanh(chi''/S)).
This is host-side analysis of the recorded correlation, not part of the time step.
"""
import numpy as np

__all__ = ["branch_correlation", "fdt_spectra"]


def branch_correlation(engine, chain, site_a, A, site_b, B, n_steps, side="left"):
    """C(tau_k) for tau_k = k dt, k = 0..n_steps, branched at the engine's current step.

    engine: a paper_2201_05529_gb300._capi.Engine whose max_steps covers n_steps more steps.
    A, B: 2x2 operators (row-major); site_a, site_b: 0-based sites of chain `chain`.
    Returns a complex array of n_steps + 1 values; the engine itself is not changed.
    """
    k0 = engine.steps_done()
    br = engine.clone()
    try:
        br.apply_local(chain, site_a, A, side)
        br.set_observables([B])            # records tau = 0 (the current step) first
        br.step(n_steps)
        obs, _ = br.read_history(k0, n_steps + 1)
    finally:
        br.destroy()
    return obs[:, chain, site_b, 0].copy()


def fdt_spectra(C, dt, n_fft=None):
    """(w, S(w), chi''(w), T(w)) from C(tau_k) = <A(tau_k) A(0)>_ss, k = 0..n, sorted by w.

    n_fft: transform length (>= 2n + 1; default the next power of two of 4n), which sets the
    frequency spacing 2 pi / (n_fft dt). T(w) is NaN where |chi''/S| >= 1 or w = 0.
    """
    C = np.asarray(C, dtype=np.complex128)
    n = C.shape[0] - 1
    M = int(n_fft) if n_fft is not None else 1 << int(np.ceil(np.log2(max(4 * n, 2))))
    if M < 2 * n + 1:
        raise ValueError("n_fft must be at least 2 len(C) - 1")
    w = np.ones(2 * n + 1)
    w[0] = w[-1] = 0.5                      # trapezoid end points at tau = -+ tau_max
    k = np.arange(-n, n + 1)
    Cabs = C[np.abs(k)]
    anti = np.zeros(M, dtype=np.complex128)
    comm = np.zeros(M, dtype=np.complex128)
    anti[k % M] = w * Cabs.real
    comm[k % M] = w * 2j * np.sign(k) * Cabs.imag
    # sum_k x_k e^{i w_m tau_k} dt with w_m = 2 pi m / (M dt): M dt ifft
    S = (M * dt * np.fft.ifft(anti)).real
    chi2 = (0.5 * M * dt * np.fft.ifft(comm)).real
    om = 2.0 * np.pi * np.fft.fftfreq(M, d=dt)
    order = np.argsort(om, kind="stable")
    om, S, chi2 = om[order], S[order], chi2[order]
    with np.errstate(divide="ignore", invalid="ignore"):
        T = om / (2.0 * np.arctanh(chi2 / S))
    T[~np.isfinite(T)] = np.nan
    return om, S, chi2, T
