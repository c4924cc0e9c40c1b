"""FP64 CPU oracle for the low-Mach variable-density pseudospectral substage.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The product path (``paper_2206_09878_gb300``) never imports it and
shares no code with it: the oracle has its own B-spline basis (plain
Cox-de Boor recursion), its own banded Gaussian elimination with partial
pivoting, and uses ``scipy.fft`` (pocketfft) as the transform primitive.

Modules
-------
bspline     knots, Greville abscissae, collocation matrices, the exact
            derivative map D* between the two spline spaces (Appendix C).
banded      batched banded Gaussian elimination with partial pivoting.
transforms  3/2-padded Fourier transforms in x and z (Eq. disc_f, Sec. 4.4).
lmvd        the substage of Algorithm 2 written step by step (Sec. 4).
ode_e1      Algorithm 1 on the scalar test system of Sec. 3.3.1.

Every function is plain FP64 and follows the paper's steps in order. Readings
of points the paper leaves open are stated where they are used.
Parity status: every function here is pinned by a ``-m "not gpu"`` test,
except the full Rayleigh-Taylor substage sequence, whose output the paper
prints no value for ("parity unpinned" for the composed multi-step RT run;
its ingredients are pinned individually and by invariants).
"""
