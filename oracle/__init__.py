"""FP64 CPU oracle for the low-Mach variable-density pseudospectral substage.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The product path (``paper_2206_09878_gb300``) never imports it and
shares no code with it: the oracle has its own B-spline basis (plain
Cox-de Boor recursion), and uses two library primitives: LAPACK's banded
Gaussian elimination with partial pivoting (``scipy.linalg.solve_banded``) for
the y-systems and ``scipy.fft`` (pocketfft) for the transforms.

Modules
-------
bspline     knots, Greville abscissae, collocation matrices, the exact
            derivative map D* between the two spline spaces (Appendix C).
banded      banded y-solves through LAPACK (scipy.linalg.solve_banded), one
            factorisation per distinct wavenumber magnitude.
transforms  3/2-padded Fourier transforms in x and z (Eq. disc_f, Sec. 4.4).
lmvd        the substage of Algorithm 2 written step by step (Sec. 4).
ode_e1      Algorithm 1 on the scalar test system of Sec. 3.3.1.

Every function is plain FP64 and follows the paper's steps in order. Readings
of points the paper leaves open are stated where they are used.
Parity status: every function here is pinned by a ``-m "not gpu"`` test
against closed forms, invariants, brute force, library routines or values
the paper prints. The convective right-hand side, the advection term of R_z,
f'(z), rho_t and the tail of L are pinned by exact solutions of the
continuous equations (tests/test_oracle_closed_forms.py). The composed
multi-step Rayleigh-Taylor run has no printed values ("parity unpinned" for
that sequence; its ingredients are pinned individually and by invariants).
"""
