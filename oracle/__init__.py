"""Plain FP64 CPU oracle for the space-time waveform-relaxation multigrid method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It
shares no code with the CUDA path.

The oracle writes the method out the slow, obvious way:

* ``basis``     -- 1D Lagrange bases, Gauss-Legendre rules, right-Radau
                   (Radau IIA) temporal nodes and the DG(q) time matrices
                   (Def. "Temporal discretisation", Eq. dgintime).
* ``fem``       -- Taylor-Hood Q_{k+1}^2/Q_k on a uniform n x n quad mesh,
                   the space-time residual F(U) and Jacobian J(W) of
                   Eq. nsfem assembled into global sparse matrices.
* ``patches``   -- Vanka+star space-time patches (Sec. 3, NS relaxation)
                   and the waveform patch solve of Eq. waveform_patch_solve.
* ``transfer``  -- P = I (x) blockdiag(P_u, P_phi), R = P^T (Sec. 3).
* ``solver``    -- coarse direct solve, Chebyshev(2) relaxation weights,
                   the 10-step eigen-estimate, V(2,2) (Algorithm Vcycle),
                   FGMRES and inexact Newton with Eisenstat-Walker terms.

Parity status of every function is stated in its docstring; the pins that
check each one against what the paper and mathematics fix live in
``tests/test_oracle_*.py``.
"""
