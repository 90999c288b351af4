"""FP64 CPU oracle for the PT-TEBD time step -- TEST INFRASTRUCTURE ONLY.

Plain NumPy/SciPy in complex128, written from the paper (arXiv:2201.05529) for a reader
to check against it by eye: Liouville-space conventions (Sec. II.A, App. A.1), the
second-order Trotter schedule (Eq. (propagator-env), App. A.1), the bath correlation
function (App. B.1), the discretised influence functional and its PT-MPO compression
(App. B.1, following the PT-TEMPO literature the paper cites), the augmented-MPS bond
update (App. A.2), the PT-MPO site contraction (App. A.2), cap
tensors (App. A.3) and readout, including two-time correlations (App. A.4).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg of
``bench.py`` may import this package. It shares no code with the CUDA path and imports
nothing from it; the only shared module is ``workloads`` (parameters and seeded draws).

Pins (tests/test_oracle_*.py): exact 4^N Liouvillian exponentiation and the exact
product of the same Trotter gates (alpha = 0), the pure-dephasing closed form, a
brute-force influence-functional path sum, an exact single-mode bath simulation,
closed forms of C(tau) and G(t) against quadrature, and trace / hermiticity invariants.
"""
