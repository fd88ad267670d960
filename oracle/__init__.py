"""Plain, slow, FP64 CPU oracle for periodic thermal-microstructure design.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call, link
or execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, tables or helpers with the CUDA implementation under
``paper_2405_19991_gb300/``; the two meet only through the seeded input
generators in ``workloads/``.

Every routine follows the paper (Quan, Zhai, Fu, "OpenTM", arXiv 2405.19991)
and cites the section or equation it restates:

* ``fem``    -- element matrix, periodic assembly, macro load, CG solve,
               homogenized tensor (Sec. 2.2 Eq. homo and its discrete form,
               Sec. 2.4 enforceMacroLoad / FEM), Galerkin coarse operators
               (Alg. 3).
* ``design`` -- density filter (Sec. 2.3), SIMP (Sec. 2.2), objective
               (Eq. mse, fracmse, l1), sensitivity (Eq. sens, Sec. 2.3),
               OC update (Sec. 3.3 OCOptimizer) and the adaptive volume bound
               (Alg. 1), assembled into one design iteration (Alg. 2 and the
               optimisation loop of Sec. 3.4).
* ``mma``    -- the Method of Moving Asymptotes with one constraint
               (Svanberg's standard form, dual route), for model 2
               (Eq. model2, MMAOptimizer of Sec. 3.3).
* ``unet``   -- plain-loop periodic 3-D conv U-Net forward/backward used to
               check the learned warm-start kernels' gradients.

Parity status of each function is listed in its docstring; all of ``fem``,
``design`` and ``mma`` are pinned by tests in ``tests/test_oracle_*.py`` against closed
forms, bounds, invariants, finite differences and brute force.
"""
