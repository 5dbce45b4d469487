"""FP64 CPU oracle for the projection-tree reduced-order model (arXiv 2103.01983).

TEST INFRASTRUCTURE ONLY.  This package is the independent reference the CUDA
path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it; the
product library (``paper_2103_01983_gb300``) never does, and the oracle never
imports the product library (it shares only the seeded input generators in
``paper_2103_01983_gb300.workloads``, which hold no arithmetic of the method).

Modules:
  direct  -- ctypes front end of ``bs_direct.c`` (plain FP64 double loops:
             velocity, self blocks, J v, J^T w, (df/dGamma)^T w, J Phi).
  kernel  -- dense NumPy formulations: f = K gamma (Eq. 4-6) and the full
             Jacobian d f / d x assembled block by block.
  fom     -- implicit trapezoid rule (Eq. linKstep) solved by Newton with a
             dense, block-diagonal or Jacobian-free (GMRES) linear solve.
  qoi     -- Hamiltonian, AE_H, MAE_D and the linear/angular impulses (Sec. 6.1).
  rom     -- POD, quadtree, ClusterPOD (Alg. 2/3), greedy sampling (Alg. 1),
             LSPG/GNAT and the online PTROM Gauss-Newton (Alg. 4/5).
"""
