"""Plain FP64 CPU oracle for the HSMA pair-sum path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package.
The product path (the CUDA library and its Python binding) never calls it,
shares no code with it and must fail loudly when its extension is missing.

Contents
--------
``ewald``      Ewald summation ground truth: 3D tin-foil (Sec. 2.1, Eq. 3) and
               the 2D-periodic image-layer series of a dielectric slab
               (Sec. 2.1, Eq. 4), each layer by a Parry-type 2D Ewald sum.
``harmonics``  Real orthonormal spherical harmonics, regular solid harmonics
               and their z-derivative (the basis of Eq. 5's truncated series).
``hsma``       CPU HSMA3D / HSMA2D step by step in the paper's order
               (Sec. 2.2): near set in the sphere B, least-squares fit of the
               harmonic coefficients, mapping onto Fibonacci surface charges,
               final near + far sums, energy and forces.

Every function works in FP64 with sums in fixed index order, so the oracle is
deterministic.  Nothing here is blocked, fused or reordered beyond what the
definitions state.
"""
