"""The oracle: plain FP64 CPU implementation of the per-step cloth solve.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import it.  It shares no code
with the CUDA library (paper_2403_19272_gb300); both read their inputs from
the ``workloads`` module.

  pd.py       PD stepper (Sec. 3 Eqs. var/z/local/global, Sec. 4 Eq. exp,
              Sec. 5.1, Alg. 1 / Sec. 7) with an exact sparse global solve.
  collide.c   brute-force broad phase, exact CCD, partial CCD (Sec. 4.1),
              closest points, triangle-triangle intersection.
  subspace.py dense reference of the subspace-reuse correction (Sec. 5,
              Eqs. subspace_global / subspace_collision / uu).
"""
