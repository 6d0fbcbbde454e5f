"""Plain fp64 CPU oracle for the vielbein lattice Boltzmann RK3 stage.

This package is test infrastructure.  Only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the product path never
does.  It shares no code with the CUDA library: quadrature tables are rebuilt
here from their definitions in high-precision decimal arithmetic, and every
stage step is written out in the paper's order and notation:

* ``quadrature``  -- full- and half-range Gauss-Hermite rules (Sec. IV.B).
* ``lbmodel``     -- force kernels K, K~ (Sec. IV.C, App. D) and the truncated
                     equilibrium (Sec. IV.D).
* ``weno``        -- epsilon-free WENO-5 interface values (Sec. III.C, Table IV).
* ``couette``     -- the chi-formulation circular Couette stage operator L[F],
                     diffuse-reflection walls and TVD-RK3 (Secs. III, VI.A).
* ``channel``     -- the gradually expanding channel stage (Sec. VII.A-B).
* ``analytic``    -- closed-form Couette profiles used as pins (Sec. VI.B-D).
"""
