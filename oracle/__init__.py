"""CPU FP64 oracle for exchange-correlation integration in a Gaussian basis.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything from this package.  The
library path never calls it and shares no code with it.

The oracle is written from the paper (Williams-Young, de Jong, van Dam, Yang,
"On the Efficient Evaluation of the Exchange Correlation Potential on Graphics
Processing Unit Clusters"), section by section:

* ``quadrature``  -- atomic product grids (Sec. 2.2, Eq. num_int): Mura-Knowles
  radial rule and a Gauss-Legendre(theta) x trapezoid(phi) angular rule.
* ``partition``   -- atomic partition functions p_A (Sec. 2.2, Eq.
  atomic_partition): Becke and Stratmann-Scuseria-Frisch (SSF).
* ``planner``     -- screening radius (Eq. rcut), cuboid subdivision into
  batches (Sec. 2.2 and the grid-partition figure), cuboid-sphere screening
  (Algorithm 1), merging batches with equal shell lists and the work estimate
  (Algorithm 3, Eq. batch_work).
* ``collocation`` -- contracted Cartesian Gaussians and their gradients
  (Eq. gau_cart).
* ``functionals`` -- Slater exchange and PBE exchange-correlation with
  hand-derived first derivatives.
* ``integrate``   -- E_xc, V_xc and N_el in two modes: definitional (every grid
  point, every function: Eqs. exc_vvar, vxc_exact, zvec_r) and
  method-equivalent (batch by batch over S_j: Eqs. x_mat, eval_local_den,
  eval_local_den_grad, exc_batch, vxc_inc, vxc_batch, eval_xc_batch, z_mat).

Every function is plain NumPy in float64; the only library primitives used are
elementwise arithmetic, ``math``/``numpy`` elementary functions and matrix
products.

Parity pins: each module's tests live in ``tests/test_oracle_*.py``; the functional
constants are pinned by closed forms and design conditions in
``tests/test_oracle_pins_physics.py`` (the reduced gradient from its definition, PBE's
cancellation of the second-order gradient terms, which fixes mu = beta pi^2/3 and the s and t
normalisations, PW92's high-density coefficient against Gell-Mann-Brueckner's (1 - ln 2)/pi^2,
the hydrogen atom's closed-form LSD exchange and exact exchange -5/16, which MVS reproduces,
PW92's high-density expansion for all three parameter sets: A, the constant c1 and no
r_s^(1/2) term, which fix beta_1 and beta_2; and PBE's beta against Ma and Brueckner's
gradient coefficient through the small-t limit of H).
Still "parity unpinned", because nothing in reach fixes them beyond those relations:
PW92's alpha_1, beta_3 and beta_4 (published values are used
verbatim; PBE's tabulated hydrogen values are checked to three decimals only), MVS's e1 and c1
(they do not enter at alpha = 0), and the Mura-Knowles radial scale alpha = 5.0.
"""
