"""Plain, slow, FP64 CPU oracle for the segregated implicit Bidomain step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call this
package: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  It shares no code with the CUDA library.

It follows Huynh, Pavarino and Scacchi, "Parallel Newton-Krylov BDDC and
FETI-DP deluxe solvers for implicit time discretizations of the cardiac
Bidomain equations" (arXiv 2101.02959):

* ``mesh``     Section 4.1: structured Q1 grid, subdomains, the sets N_x and
               the face / edge / vertex equivalence classes, primal sets;
               Section 6: the truncated-ellipsoid map.
* ``fem``      Section 3a: fibre field, conductivity tensors D_{i,e},
               Q1 stiffness A_{i,e} and the lumped mass M, on box elements
               and on isoparametric (ellipsoid) elements.
* ``ionic``    Section 2: Rogers-McCulloch I_ion and R; Section 3b Step 1.
* ``bidomain`` Section 3b Step 2 (F, G), Section 3c (Jacobian, Newton),
               direct sparse solve of the Jacobian system.
* ``dd``       Sections 4.1-4.4: local matrices, Schur complements, deluxe
               and rho scaling, BDDC and FETI-DP operators, and the option of
               a lagged BDDC preconditioner.
* ``krylov``   PCG, GMRES and the Lanczos condition-number estimate.
* ``mlp``      FP64 forward / backward of the initial-guess network.

Every function states the passage it follows.  Parity status of each part is
listed in the module docstrings ("pinned by ..." or "parity unpinned").
"""
