"""FP64 CPU oracle for the per-tile sCOLA particle-mesh evolution.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite (``tests/``),
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
anything from this package.  The CUDA library never calls into it and shares
no code, tables or constants with it; the only thing both sides consume is the
seeded synthetic input produced by ``synth_inputs``.

The oracle is a plain, slow, double-precision restatement of the method of
Leclercq et al., "Perfectly parallel cosmological simulations using spatial
comoving Lagrangian acceleration" (arXiv:2003.04925).  Each function cites the
section, equation or table of the paper it follows.  Equation numbers follow
the paper's numbering of displayed equations (Eq. 1 is x = q + Psi).

Modules
-------
cosmology   background, growth factors D1/D2, COLA time coefficients (App. A, B)
ics         white-noise colouring with a BBKS power spectrum (Sec. 3.1, A.1)
lpt         Lagrangian potentials phi1, phi2 and displacements Psi1, Psi2 (Sec. 2.1, A.2, C.2)
tiling      tiles, buffers, sCOLA boxes, r and p (Sec. 3.2, B.1, B.2; Eqs. 20-21)
boundary    Dirichlet boundary potential on the padded PM grid (Sec. 3.3 C.3, Eq. 23)
pm          B^sCOLA deposit, Dirichlet DST-I Poisson solve, FDA gradient and
            interpolation (Sec. 3.4, App. C)
scola       the KDK driver for sCOLA boxes and the untiling (App. B, Sec. 3.2)
tcola       periodic full-box tCOLA reference and the approximation-study runs of
            Sec. 4.3 (sCOLA boxes fed tCOLA's true density and/or potential)
fda         FDA stencils of order 2, 4, 6 and their symbols (Sec. 3.1, App. C)
adjoint     the reverse-mode gradient of a final-density loss (FP64 reference of the
            library's hand-written adjoint)
stats       final periodic CIC density and the P(k) estimator (Sec. 4.1-4.2, Eq. 24)
rng         restatement of the library's device white-noise generator (Philox4x32-10,
            Box-Muller) from the published definitions

Parity status of each part (what pins it) is listed in each module header.
"""
