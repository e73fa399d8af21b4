"""FP64 CPU oracle for the WaveHoltz domain-decomposition Helmholtz method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` use it.  It shares no code with
the CUDA library (``paper_2606_21695_gb300``); the only module both sides use
is ``workloads`` (seeded input generators, none of the method's arithmetic).

Plain, slow, obviously-correct NumPy/SciPy restatement of the paper
"Efficient Domain Decomposition for the Helmholtz Equation on GPUs":

* ``sem``   -- GLL nodes/weights, the Lagrange differentiation matrix, the
               structured quad mesh, and the element-by-element matrix-free
               stiffness apply (Sec. 4, eq. (discrete-helmholtz); Sec. 6.1
               describes the gradient-at-quadrature-point form used here).
* ``dd``    -- subdomains, the WaveHoltz subdomain solver (Sec. 5,
               eq. (WaveHoltz), modified leapfrog), the DDM cycle
               (Algorithm 1) with the transmission update (eq.
               (lambda-iteration), sign read as -2ik), plain and GMRES outer
               iterations (Sec. 3, Krylov acceleration), the global operator,
               residual, direct solve and FP64 refinement (Sec. 7, DD as a
               preconditioner: defect correction or flexible GMRES).
* ``krylov``-- plain restarted GMRES and flexible GMRES (minimal-residual
               definitions, least squares on the Hessenberg matrix).

Parity status of each function is listed in its docstring.  The WaveHoltz
and outer-iteration *convergence rates* are "parity unpinned": they are
reported, and matched iterate-by-iterate against the CUDA path, but no
closed form fixes them.
"""

from . import sem, krylov, dd  # noqa: F401
