"""Plain FP64 CPU oracle for the PM-FEM effective-field path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import anything from here.
The product (the C-ABI library and its Python binding) never imports, links or
runs this package, and this package never imports the product.

Two tiers, both written from the paper (Ai, Duan, Lomakin, "Periodic micromagnetic
finite element method"):

* O1 (``direct``): the definition.  Point charges at the mesh nodes interact
  through the periodic Green's function G^p of Eq. 15 (lattice sums evaluated by
  Ewald-type splitting), plus the exact near-element correction of Eq. 14c; the
  field follows from the periodized gradient, Eq. 14d.  O(N'^2).
* O2 (``paim``): the four BAIM steps of Sec. 3.2 (project, FFT-convolve with the
  PGF on the grid of Eq. 16, interpolate, precorrect), with the same near sets.

Modules: ``topology`` (periodic pairing and LCA, Sec. 2.2; fold, Eq. 18),
``operators`` (local sparse operators, Eqs. 7-12 and 14a/14d), ``pgf`` (Eq. 15),
``integrals`` (exact potential integrals over triangles and tetrahedra),
``nearfield`` (Eq. 14c near-element matrix), ``direct`` (O1), ``paim`` (O2),
``llg`` (Eq. 2 with classical RK4), ``problem`` (ties them together).

Parity status of each function is stated in its docstring; functions whose values
no test pins against an independent fact say "parity unpinned".
"""
