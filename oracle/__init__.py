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

Parity pins: each module's tests live in ``tests/test_oracle_*.py``.  Two
constants are "parity unpinned" because nothing outside the chosen convention
fixes them: the absolute PW92/PBE correlation parameters (published values are
used verbatim) and the Mura-Knowles radial scale alpha = 5.0.
"""
