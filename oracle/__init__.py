"""CPU FP64 oracle for the even-odd preconditioned twisted-mass clover solver path.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import this package.  The library (include/tm.h and the
CUDA kernels behind it) never imports, links or calls anything here, and this
package imports nothing from the library: the two share no code.  The one
common module is ``synth`` (seeded input fields), which holds none of the
method's arithmetic.

Paper: "Twisted mass ensemble generation on GPU machines" (arXiv 2212.06635).
  dirac.py    operators of Sec. 2: Q_pm (unnumbered eqs. above eq:hQpm), the
              asymmetric even-odd Schur operator Q_hat_pm (eq:hQpm), the
              mass-preconditioned W_hat_pm (eq:hWpm) and the heavy doublet
              Q_hat_h (eq:hQh)
  solvers.py  CG, multishift CG (Sec. 4.2), power iteration, dense solves
  ptc.py      gauge-equivariant parallel-transport network preconditioner
              (not in the paper; parity of its training trajectory unpinned)
  force.py    fermion-force outer products of the hopping term on every link
              (the rational-approximation force step of Sec. 4.3)
  rational.py Zolotarev's rational approximation of A^-1/2, its application in
              partial fractions, and the binomial series of the correction
              term (Sec. 4.2, Fig. 4's heatbath and acceptance)
  multigrid.py aggregation-based two-level multigrid preconditioner for GCR on
              the full operator (Sec. 4.1's MG-preconditioned light solves)
"""
