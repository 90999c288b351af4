"""The five PT-TEBD workloads, as plain parameters and seeded draws.

Physics (Sec. III, Eq. (xyz-spin-chain); Sec. IV, Eq. (xy-spin-chain); bath Eq. (bosonic-bath)):
  H = sum_n eps_n s^z_n + sum_n sum_g J^g_n s^g_n s^g_{n+1} + sum_n H^E_n,   s = sigma/2,
  H^E_n couples the bath to s^z_n (eigenvalues +1/2 for up, -1/2 for down),
  J(w) = 2 alpha w exp(-w/w_c) (exponential cutoff; the paper's own runs use exp(-w^2/w_c^2)).

Readings where the workload text is silent (each listed in the design notes):
  * "hz=0.5 on site 1" means eps_1 = 0.5 as the coefficient of s^z (not sigma^z).
  * "coupled via sigma z" means the bath operator is s^z = sigma^z / 2.
  * the five-site chain starts in |up down up down up>; the ensemble starts in Neel states with
    no field; the 21-site chain has no field (hz = 0).
  * eps (relative SVD threshold) is 1e-10 where the text says "no binding truncation", 1e-6 for
    the 21-site chain (the paper's typical value, App. A.2), and 1e-8 elsewhere.

Nothing here computes a propagator, an influence functional or a contraction.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional, Tuple

import numpy as np

BASE_SEED = 220105529


@dataclass(frozen=True)
class BathSpec:
    """Gaussian bosonic bath coupled to s^z of one site (Eq. (bosonic-bath))."""
    alpha: float
    omega_c: float
    T: float
    cutoff: str = "exponential"     # "exponential": exp(-w/wc); "gaussian": exp(-w^2/wc^2)


@dataclass(frozen=True)
class DriveSpec:
    """Two-spin thermal driving of sites 0 and 1 (the comparison network of Sec. III.A.3): a
    time-local generator that relaxes the pair to the Gibbs state of its own two-spin Hamiltonian
    at temperature T, with jump rates of scale `rate`."""
    T: float
    rate: float


@dataclass(frozen=True)
class ChainSpec:
    """One spin-1/2 chain: on-site fields, bond couplings, product initial state, baths, and
    optional time-local dissipation (App. A.1's GKSL terms of the system Liouvillians)."""
    N: int
    eps: Tuple[float, ...]                         # coefficient of s^z on each site
    J: Tuple[Tuple[float, float, float], ...]      # (Jx, Jy, Jz) per bond, len N-1
    init: str                                      # 'u' / 'd' per site
    baths: Tuple[Optional[BathSpec], ...]          # per site, None = no bath
    gksl: Tuple[Tuple[int, str, float], ...] = ()  # (site, 'minus'|'plus'|'z', rate): L = sqrt(rate) op
    drive: Optional[DriveSpec] = None              # two-spin thermal driving of sites 0, 1

    def __post_init__(self):
        assert len(self.eps) == self.N and len(self.J) == self.N - 1
        assert len(self.init) == self.N and len(self.baths) == self.N
        assert all(0 <= g[0] < self.N and g[1] in ("minus", "plus", "z") and g[2] >= 0 for g in self.gksl)
        assert self.drive is None or self.N >= 2


@dataclass
class Workload:
    name: str
    chains: Tuple[ChainSpec, ...]
    dt: float
    K: int                          # number of time steps
    chi_max: int
    eps: float                      # relative singular-value threshold (App. A.2)
    kappa_max: int                  # PT-MPO bond cap
    eps_tempo: float = 1e-7         # PT-MPO relative SVD threshold
    multiplet_tol: float = 1e-12    # a cut may not split singular values closer than this x s_max
    memory_steps: int = 0           # Delta K_max; 0 = every step of the run (no memory cut)
    two_time: Optional[Tuple[int, str]] = None   # (site, 'x'|'y'|'z') for <s(t) s(0)> at that site
    random_state: Optional[dict] = None          # stress workload: explicit tensors
    notes: str = ""

    @property
    def site_steps(self) -> int:
        return sum(c.N for c in self.chains) * self.K


XYZ_J = (1.3, 0.7, 1.2)


def _xyz_chain(N, baths, init, hz_site0=0.5, J=XYZ_J):
    eps = tuple([hz_site0] + [0.0] * (N - 1))
    return ChainSpec(N=N, eps=eps, J=tuple([tuple(J)] * (N - 1)), init=init, baths=tuple(baths))


def _config1():
    b = BathSpec(alpha=0.1, omega_c=4.0, T=1.0)
    ch = _xyz_chain(3, [b, None, None], "udu")
    return Workload("xyz3_onebath", (ch,), dt=0.1, K=20, chi_max=64, eps=1e-10, kappa_max=16,
                    notes="N=3 XYZ, one Ohmic bath on site 1, 20 steps")


def _config2():
    hot = BathSpec(alpha=0.16, omega_c=4.0, T=5.0)
    cold = BathSpec(alpha=0.16, omega_c=4.0, T=0.5)
    ch = _xyz_chain(5, [hot, None, None, None, cold], "ududu")
    return Workload("xyz5_twobaths", (ch,), dt=0.05, K=200, chi_max=64, eps=1e-8, kappa_max=32,
                    two_time=(2, "x"),
                    notes="N=5 XYZ between a hot (T=5) and a cold (T=0.5) bath, 200 steps")


def _config3():
    b = BathSpec(alpha=0.05, omega_c=3.0, T=0.8)
    N = 21
    init = "".join("u" if n == N // 2 else "d" for n in range(N))
    ch = ChainSpec(N=N, eps=tuple([0.0] * N), J=tuple([(1.0, 1.0, 0.0)] * (N - 1)), init=init,
                   baths=tuple([b] * N))
    # multiplet tolerance 1e-9: the U(1)-symmetric chain's exact multiplets (gaps ~1e-16) are kept whole
    # by any SVD accurate to well below 1e-9 of s_max, the tensor-core fast path included
    return Workload("xy21_allbaths", (ch,), dt=0.1, K=100, chi_max=128, eps=1e-6, kappa_max=16,
                    multiplet_tol=1e-9,
                    notes="N=21 isotropic XY, a bath on every site, one central excitation")


def _config4(n_chains=64):
    chains = []
    for c in range(n_chains):
        rng = np.random.default_rng([BASE_SEED, 4, c])
        N = int(rng.integers(4, 17))
        J = tuple(float(x) for x in rng.uniform(0.5, 1.5, size=3))
        bl = BathSpec(alpha=float(rng.uniform(0.05, 0.2)), omega_c=4.0, T=float(rng.uniform(0.5, 5.0)))
        br = BathSpec(alpha=float(rng.uniform(0.05, 0.2)), omega_c=4.0, T=float(rng.uniform(0.5, 5.0)))
        init = "".join("u" if n % 2 == 0 else "d" for n in range(N))
        baths = [bl] + [None] * (N - 2) + [br]
        chains.append(ChainSpec(N=N, eps=tuple([0.0] * N), J=tuple([J] * (N - 1)), init=init,
                                baths=tuple(baths)))
    return Workload("xyz_ensemble64", tuple(chains), dt=0.05, K=100, chi_max=64, eps=1e-8,
                    kappa_max=16, notes="64 independent XYZ chains, N in [4,16], baths on the ends")


def random_state_draws(N=32, chi=96, kappa=16, K=20, seed=(BASE_SEED, 5)):
    """Seeded random tensors for the stress workload (no physics, no method arithmetic).

    Returns Gaussian site tensors Gamma_n[chi_l][4][kappa][chi_r] (chi_l = 1 at the left end,
    chi_r = 1 at the right end), bond weights lambda_i ~ exp(-i/16) (unnormalised), Gaussian PT
    tensors P^(k)[kappa][4][4][kappa] for k = 1..K (shared by every site), and one Haar-random
    4x4 two-site unitary per bond and per gate length (dt/4, dt/2).
    """
    rng = np.random.default_rng(list(seed))

    def cgauss(*shape):
        return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)

    def haar(n):
        z = cgauss(n, n)
        q, r = np.linalg.qr(z)
        ph = np.diag(r) / np.abs(np.diag(r))
        return q * ph[None, :]

    chis = [1] + [chi] * (N - 1) + [1]
    gam = [cgauss(chis[n], 4, kappa, chis[n + 1]) for n in range(N)]
    lam = [np.ones(1)] + [np.exp(-np.arange(chi) / 16.0) for _ in range(N - 1)] + [np.ones(1)]
    pts = [cgauss(kappa, 4, 4, kappa) for _ in range(K)]
    u_q = [haar(4) for _ in range(N - 1)]
    u_h = [haar(4) for _ in range(N - 1)]
    return dict(gamma=gam, lam=lam, pt=pts, u_q=u_q, u_h=u_h, kappa=kappa, chi=chi)


def _config5(N=32, chi=96, kappa=16, K=20):
    ch = ChainSpec(N=N, eps=tuple([0.0] * N), J=tuple([(0.0, 0.0, 0.0)] * (N - 1)),
                   init="u" * N, baths=tuple([None] * N))
    rs = dict(N=N, chi=chi, kappa=kappa, K=K)
    return Workload("random32_stress", (ch,), dt=0.1, K=K, chi_max=chi, eps=1e-8,
                    kappa_max=kappa, random_state=rs,
                    notes="random Gaussian augmented MPS, random PT tensors and unitary gates")


def _config_gksl():
    # the five-site XYZ chain with on-site GKSL terms next to a bath: decay on site 1, dephasing on
    # site 3, pumping on site 5 (which also carries the hot bath)
    hot = BathSpec(alpha=0.16, omega_c=4.0, T=5.0)
    ch = _xyz_chain(5, [None, None, None, None, hot], "ududu")
    ch = replace(ch, gksl=((0, "minus", 0.2), (2, "z", 0.1), (4, "plus", 0.05)))
    return Workload("xyz5_gksl", (ch,), dt=0.05, K=40, chi_max=64, eps=1e-10, kappa_max=16,
                    notes="N=5 XYZ with on-site decay, dephasing and pumping, one bath")


def _config_drive():
    # Sec. III.A.3: two extra spins on the left of the five-site chain, driven towards the Gibbs
    # state of their own Hamiltonian (T = 1.6, the single-bath temperature of Sec. III.A); no PT-MPO
    ch = _xyz_chain(7, [None] * 7, "ududud" + "u", hz_site0=0.0)
    ch = replace(ch, drive=DriveSpec(T=1.6, rate=1.0))
    return Workload("xyz7_twospin_drive", (ch,), dt=0.05, K=40, chi_max=64, eps=1e-8, kappa_max=1,
                    notes="two-spin GKSL driving of a five-site XYZ chain (comparison network)")


_BUILDERS = {
    "xyz3_onebath": _config1,
    "xyz5_twobaths": _config2,
    "xy21_allbaths": _config3,
    "xyz_ensemble64": _config4,
    "random32_stress": _config5,
    "xyz5_gksl": _config_gksl,
    "xyz7_twospin_drive": _config_drive,
}
WORKLOAD_NAMES = tuple(_BUILDERS)


def workload(name: str, **overrides) -> Workload:
    """Return a workload by name; keyword overrides replace fields (e.g. K=10 for a short run)."""
    w = _BUILDERS[name]()
    if overrides:
        w = replace(w, **overrides)
    return w
