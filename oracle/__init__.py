"""Plain complex128 CPU oracle for the one-way vector Helmholtz propagator.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may call it.  It shares no code with the CUDA path: the two
meet only in the seeded input generators of
``paper_2410_17446_gb300.workloads`` (which hold none of the method's
arithmetic) and in pole tables that ``oracle.make_tables`` writes.

Modules
  operators   -- wavenumbers, the operator matrix Z (Eq. Z_bar_eq), its
                 free-space part (Eq. Z_bar_fs_def), the FFT and the dense
                 Sylvester forms of the free-space solve (Eqs. freespace_prob,
                 fs_sylvester), dense matrices for small grids.
  aaa_lawson  -- the AAA-Lawson rational fit of exp(iK(-1+sqrt(1+zeta)))
                 (Sec. 3.1) and its partial fractions (Eq. pf_expan_eq).
  gmres       -- right-preconditioned GMRES with a Householder-orthogonalised
                 Krylov basis (Sec. 4.2).
  propagator  -- one z-step, Eqs. (W_k_def) and (approx_prop), by GMRES or by
                 dense LU; the exact angular-spectrum step (Eq.
                 exp_prop_planewave); runs with a medium schedule.

Every function is a direct statement of the passage it cites, in float64 /
complex128, with no blocking, fusion or reordering beyond it.
"""
