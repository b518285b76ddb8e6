"""Plain complex128 CPU oracle for the FFT-accelerated macromodel solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may use it.  It shares no code with the CUDA path.

Every function follows the paper (Patel, Triverio, Hum, "A Fast Macromodeling
Approach to Efficiently Simulate Inhomogeneous Electromagnetic Surfaces")
step by step, in plain NumPy/SciPy, without blocking, fusion or FFTs:

* ``quadrature``  -- triangle quadrature and closed-form potential integrals
                     used for singularity extraction (the paper is silent on
                     quadrature: 7-point Radon rule plus closed-form 1/R and
                     grad 1/R parts over the source triangle).
* ``mesh``        -- box surface S_eq and patch meshes, RWG bases (Sec. II-A,
                     Eqs. Hdiscretebox/Ediscretebox).
* ``operators``   -- Galerkin L and K blocks (Eqs. SIE_LOperator1,
                     SIE_KOperator1, blockZo), plane-wave excitation V
                     (Eq. out) and far field (Sec. III-D, last paragraph).
* ``lattice``     -- offset tables, the overlap map U_o (Sec. III-D, rule 1),
                     the direct (FFT-free) product U_o^T[Z_eq+Z_o]U_o x
                     (Eq. MVP) and dense assembly of Eq. final.
* ``macromodel``  -- per-cell macromodels by Schur complement (Eq. Zmacromodel).
* ``solve``       -- dense LU and plain restarted GMRES for Eq. final.
* ``precond``     -- the cell-grouped near-field preconditioner (Sec. IV-A,
                     Eq. final_precond) as restricted additive Schwarz with
                     dense complex128 subdomain solves.

Parity status of each function is stated in its module header.
"""
