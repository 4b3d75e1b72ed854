"""Plain, slow FP64 CPU oracle for the grid potential-flow method of
Beckers & Eldredge, "Planar potential flow on Cartesian grids" (arXiv 2102.11910).

This package is TEST INFRASTRUCTURE. Only the test-suite, the smoke check of the
package entry module and the CPU-baseline leg of the benchmark may import it.
The product path (the CUDA library and its Python binding) never imports,
links or calls anything here, and nothing here imports the product.

Every routine follows a passage of the paper (section / equation cited in its
docstring) in the paper's order and notation, in numpy float64, with no
blocking, fusion or reordering beyond what the definition states.

Modules
-------
lgf      lattice Green's function of the 5-point Laplacian (Sec. 2.1) by
         one-dimensional quadrature of its Fourier definition.
kernels  the M4' (vortex) and smoothed three-point (surface) discrete deltas.
vic      regularization R_v (Eq. vortexregularization), the unbounded inverse
         Laplacian by direct summation, node velocity and interpolation E_v.
body     surface operators R_s/E_s, Schur complement S (Eq. vsheet), f0, Gamma0,
         circulation removal, Kutta projection and the constrained sheet solves
         of Sec. 2.3-2.4 (Eqs. circsystem, kuttasystem, kuttasystem2,
         kuttasystem3/twovortex), the generalized edge condition (Sec. 2.5)
         and several bodies sharing one S (Sec. 2.7, Eq. kuttasystem4).
step     vortex shedding placement and the Euler / RK2 time step (Sec. 2.4.2),
         with one body or several.
diagnostics  linear and angular impulse of the fluid (Sec. 2.6.2, Eqs.
         linimpxd, linimpyd, angimpd).
pressure the jump in scalar potential of the sheet, the surface pressure
         jump of the immersed-boundary Bernoulli equation and the cell-centre
         pressure field (Sec. 2.6.1).
"""
