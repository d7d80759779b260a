"""Plain FP64 CPU oracle for the sparse-grid time-DG streamline-diffusion method.

TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may import,
call or execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` do.  It shares
no code with the CUDA library (no common helpers, tables or generators); the
only shared module is ``sgdg_workloads`` which holds inputs, not arithmetic.

The oracle follows the paper step by step, slowly and obviously:

* ``mesh``      nested uniform refinement, P1 spaces and embeddings E (Sect. 2, Sect. 4.2)
* ``assembly``  finest-level FE factor matrices and their Galerkin projection (Sect. 4.2)
* ``operator``  time matrices, the Kronecker block formula and the blockwise
                apply with its ordering rule (Sect. 4.2)
* ``solver``    GMRES, the combination-technique preconditioner (Algorithm 1),
                component solves with the (T+dC+G) x M x M preconditioner, strip driver
* ``tensor``    tensor-product Q_r elements on box meshes of squares (Sect. 5.1, Table 1's d = 2 meshes)
* ``brute``     literal full-grid 2d-dimensional assembly of the weak form
                (Sect. 2, Eq. 5) for tiny levels - the pin for the block formula

Every function is pinned by the ``-m "not gpu"`` tests; see the module headers.
"""
