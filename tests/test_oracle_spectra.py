"""Pins of the branching two-time correlation and of the spectra (test infrastructure, CPU)."""
import numpy as np

from oracle import exact, model, problem, spectra
from workloads.configs import ChainSpec, Workload


def _closed_chain(N, eps, init):
    return ChainSpec(N=N, eps=tuple(eps), J=((1.3, 0.7, 1.2),) * (N - 1), init=init, baths=(None,) * N)


def test_branching_at_a_later_step_matches_full_trotter_product():
    # App. B.2: the super-operator is applied to the evolved state (here after step 6), and the
    # readout continues from there; against the exact 4^N Trotter product with the same insertion
    ch = _closed_chain(4, [0.5, 0, 0, 0], "udud")
    w = Workload("t", (ch,), dt=0.05, K=14, chi_max=256, eps=1e-14, kappa_max=1)
    ci = problem.build_inputs(w)[0]
    for side in ("left", "right"):
        ins = (1, model.SZ, side)
        r = problem.simulate_chain(ci, w, [model.SZ, model.SX], insert=ins, insert_at=6)
        ft = exact.full_trotter_run(4, ci.rho0, ci.gates_q, ci.gates_h, w.K, [model.SZ, model.SX],
                                    insert=ins, insert_at=6)
        assert np.max(np.abs(r.obs - ft)) < 1e-12
        plain = exact.full_trotter_run(4, ci.rho0, ci.gates_q, ci.gates_h, w.K, [model.SZ, model.SX])
        assert np.max(np.abs(ft[:6] - plain[:6])) == 0.0          # nothing changes before the branch
        assert np.max(np.abs(ft[6:] - plain[6:])) > 1e-3


def _lorentz_disc(nu, g, dt):
    # sum_k dt e^{-g |k| dt} e^{i nu k dt} over all integers k (a geometric series)
    return dt * np.sinh(g * dt) / (np.cosh(g * dt) - np.cos(nu * dt))


def _damped_correlation(a, b, g, w0, dt, n):
    tau = np.arange(n + 1) * dt
    return np.exp(-g * tau) * (a * np.exp(-1j * w0 * tau) + b * np.exp(1j * w0 * tau))


def test_spectra_of_damped_oscillation_closed_form():
    # C(tau) = e^{-g tau} (a e^{-i w0 tau} + b e^{i w0 tau}): the trapezoid sums of the definitions
    # equal the discrete Lorentzians exactly (the tail beyond tau_max is below 1e-14), and approach
    # the continuous ones at O(dt^2)
    a, b, g, w0, dt, n = 1.4, 0.4, 0.5, 2.0, 0.01, 7000
    C = _damped_correlation(a, b, g, w0, dt, n)
    om = np.linspace(-6, 6, 61)
    S, chi2, T = spectra.spectra(C, dt, om)
    Sd = 0.5 * (a + b) * (_lorentz_disc(om + w0, g, dt) + _lorentz_disc(om - w0, g, dt))
    Cd = 0.5 * (a - b) * (_lorentz_disc(om - w0, g, dt) - _lorentz_disc(om + w0, g, dt))
    assert np.max(np.abs(S - Sd)) < 1e-10 * np.max(np.abs(Sd))
    assert np.max(np.abs(chi2 - Cd)) < 1e-10 * np.max(np.abs(Cd))
    lor = lambda nu: g / (g * g + nu * nu)
    Sc = (a + b) * (lor(om - w0) + lor(om + w0))
    Cc = (a - b) * (lor(om - w0) - lor(om + w0))
    assert np.max(np.abs(S - Sc)) < 1e-3 * np.max(Sc)
    assert np.max(np.abs(chi2 - Cc)) < 1e-3 * np.max(Cc)
    # S is even and chi'' odd in w; with a = n + 1, b = n the ratio at the peak is coth(w0 / 2T)
    assert np.max(np.abs(S - S[::-1])) < 1e-12 * np.max(S)
    assert np.max(np.abs(chi2 + chi2[::-1])) < 1e-12 * np.max(np.abs(chi2))


def test_effective_temperature_of_a_thermal_two_level_correlation():
    # a = n + 1, b = n with n = 1 / (e^{w0/T} - 1): at the peak w = w0 (narrow line) T(w0) -> T
    T0, w0, g, dt, n = 0.7, 2.0, 0.02, 0.02, 60000
    nb = 1.0 / np.expm1(w0 / T0)
    C = _damped_correlation(nb + 1, nb, g, w0, dt, n)
    S, chi2, T = spectra.spectra(C, dt, np.array([w0]))
    assert abs(T[0] - T0) < 2e-3


def test_product_fft_spectra_equal_the_definition():
    # the library's FFT route (paper_2201_05529_gb300.correlations) against the oracle's direct
    # trapezoid sums, on the oracle's frequency grid points
    from paper_2201_05529_gb300.correlations import fdt_spectra
    rng = np.random.default_rng(5)
    n, dt = 300, 0.05
    C = _damped_correlation(1.3, 0.45, 0.3, 1.7, dt, n) + 1e-3 * (rng.normal(size=n + 1)
                                                                   + 1j * rng.normal(size=n + 1))
    C[0] = C[0].real                       # <A A> is real at tau = 0
    om, S, chi2, T = fdt_spectra(C, dt)
    sel = np.arange(0, len(om), 37)
    So, Co, To = spectra.spectra(C, dt, om[sel])
    assert np.max(np.abs(S[sel] - So)) < 1e-10 * np.max(np.abs(So))
    assert np.max(np.abs(chi2[sel] - Co)) < 1e-10 * np.max(np.abs(Co))
    # T(w) where chi''/S is resolved (at w = 0 and the Nyquist frequency both vanish)
    ok = np.isfinite(To) & (np.abs(Co / So) > 1e-6)
    assert ok.sum() > 10
    assert np.allclose(T[sel][ok], To[ok], rtol=1e-8, atol=0)


def test_thermalised_chain_satisfies_the_fdt_at_the_bath_temperature():
    # Sec. III.A.2: a chain thermalised by one bath obeys S / chi'' = coth(w / 2T), i.e. a flat
    # effective temperature T(w) = T. Two-site XYZ chain, bath (alpha = 0.32, wc = 4, T = 1.6) on
    # site 1, branched at t_ss = 10 (App. B.2) and propagated to tau_max = 10; the finite tau_max
    # leaves a ripple, so the band average is held to 5 % and every point to 25 %
    from workloads.configs import BathSpec
    b = BathSpec(alpha=0.32, omega_c=4.0, T=1.6)
    ch = ChainSpec(N=2, eps=(0.5, 0.0), J=((1.3, 0.7, 1.2),), init="ud", baths=(b, None))
    dt, kss, ntau = 0.1, 100, 100
    w = Workload("t", (ch,), dt=dt, K=kss + ntau, chi_max=64, eps=1e-10, kappa_max=32, eps_tempo=1e-7)
    ci = problem.build_inputs(w)[0]
    r = problem.simulate_chain(ci, w, [model.SZ], insert=(1, model.SZ, "left"), insert_at=kss)
    C = r.obs[kss:, 1, 0]
    om = np.linspace(0.4, 1.6, 7)
    S, chi2, T = spectra.spectra(C, dt, om)
    assert np.all(S > 0) and np.all(chi2 > 0)
    assert abs(np.mean(T) - b.T) < 0.05 * b.T
    assert np.max(np.abs(T - b.T)) < 0.25 * b.T
