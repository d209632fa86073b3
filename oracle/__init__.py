"""Plain FP64 CPU oracle for the one-step ADER-WENO update on 3-D periodic meshes.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  The CUDA path in
``paper_1006_2146_gb300`` shares no code, tables or constant generators with
it; the two meet only through the seeded input generators of
``paper_1006_2146_gb300.inputs`` (which hold none of the method's arithmetic).

Source: Balsara, Meyer, Dumbser, Du & Xu, "Efficient implementation of ADER
schemes for Euler and magnetohydrodynamical flows on structured meshes"
(arXiv:1006.2146).  Every function cites the section / equation it follows.

Design of the oracle
--------------------
* Arrays are FP64 numpy, vectorised over zones: a per-zone quantity has shape
  ``(nvar, nz, ny, nx)`` (or ``(..., nz, ny, nx)``).  The arithmetic is written
  once per zone, in the paper's order, and numpy applies it to all zones.
* Where the method reaches a result that has a plain definition, the oracle
  writes the definition out instead of the paper's optimised formula:
    - values of the space-time polynomial at nodes (the "transcriptions" of
      Eqs. 32, 38-39, 47-48, A.5, B.4, C.4, D.3, D.8, D.13) are direct
      evaluations of the basis expansion, Eqs. 10-16;
    - face and edge averages (Eqs. 54-55, 57, 58-66, D.5, D.10, D.15) are exact
      integrals of the basis functions;
    - the source-free predictor update (Eqs. 30, 36, 45 and A.4, B.3, C.3) is
      "du/dtau = -div(flux polynomial)" matched mode by mode in the basis;
    - the nodal scheme's flux polynomial (Appendices A-C) is the Lagrange
      interpolant through its nodes (one node per mode).
* Where the method is a rule with no more basic definition (the modal
  flux-mode extraction of Eqs. 33, 40-42, 49-51, the facial extraction of
  Eqs. D.4, D.9, D.14, the WENO weights, the Riemann solvers) the oracle takes
  the paper's steps literally.  Readings of silent or garbled passages are the
  module-level constants of ``oracle.weno``, ``oracle.riemann`` and
  ``oracle.scheme``.
"""
