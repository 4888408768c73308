"""Seeded synthetic inputs for the P4D DFN linear solves.

This module only draws random numbers and lays out meshes, coefficient
fields and linearization states.  It contains none of the method's
arithmetic (no residual, Jacobian, reaction kinetics or solver): the FP64
oracle and the CUDA path each compute those from these arrays with their
own code.  Both sides consume exactly the arrays returned here.

Conventions
-----------
* Structured tensor-product hex mesh: ``nx*ny*nz`` elements with per-axis
  spacings ``hx[nx]``, ``hy[ny]``, ``hz[nz]``.  Element ``(i, j, k)`` has
  index ``i + nx*(j + ny*k)``; node ``(i, j, k)`` has index
  ``i + (nx+1)*(j + (ny+1)*k)`` (x fastest).
* ``region`` per element: 0 anode (negative electrode), 1 separator,
  2 cathode (positive electrode), 3 void (electrolyte only).  The anode
  sits at ``z = 0`` (grounded face Gamma_n), the cathode at ``z = Lz``
  (applied-current face Gamma_p).
* Per-node particle data ``Rs``/``Ds`` are only read at electrode nodes.
* Concentrations in the particle ``cs_node[nnode, nc]`` are given for every
  node; consumers keep the rows of electrode nodes only.
"""
from .generators import (  # noqa: F401
    PARAMS_DEFAULT, make_case, make_box_case, make_tiny_case, make_slab_case, theoretical_iapp,
    ocp_linear_secants, CASES, make_gyroid_cell, make_gyroid_batch, radial_grid, make_tpms_cell,
)
from .partition import owned_plane_bounds, slab_cases, slab_node_rows  # noqa: F401
