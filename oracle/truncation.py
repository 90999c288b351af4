"""Relative singular-value truncation rule (App. A.2), oracle version.

Given singular values s (descending) of an exact SVD, keep the smallest chi such that the 2-norm
of the discarded values is below eps * max(s) (strict "<"), then cap at chi_max. Reading of the
paper's silence: exact zeros are always dropped and chi >= 1; a cut that would split a multiplet
(relative gap below ``multiplet_tol``) is moved so the multiplet is kept whole when that fits
under chi_max, and dropped whole otherwise, so the kept subspace does not depend on the
arbitrary basis an SVD picks inside a degenerate subspace.
"""
from __future__ import annotations

import numpy as np

MULTIPLET_TOL = 1e-12


def truncation_rank(s, eps, chi_max, multiplet_tol=MULTIPLET_TOL):
    s = np.asarray(s, dtype=float)
    n = len(s)
    if n == 0 or s[0] <= 0.0:
        return 1
    smax = s[0]
    # tail[c] = sqrt(sum_{i >= c} s_i^2)
    tail = np.sqrt(np.concatenate([np.cumsum((s ** 2)[::-1])[::-1], [0.0]]))
    chi = n
    for c in range(1, n + 1):
        if tail[c] < eps * smax:
            chi = c
            break
    nz = int(np.count_nonzero(s > 0.0))
    chi = max(1, min(chi, nz))

    def splits(c):
        return 0 < c < n and (s[c - 1] - s[c]) <= multiplet_tol * smax

    if chi <= chi_max:
        while splits(chi) and chi < chi_max and s[chi] > 0.0:
            chi += 1
        if not splits(chi):
            return chi
    chi = min(chi, chi_max)
    while chi > 1 and splits(chi):
        chi -= 1
    return chi
