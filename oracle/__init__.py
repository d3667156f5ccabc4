"""FP64 CPU oracle for the parallel-Newton hot path.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` use it. It shares no code with
the CUDA library (no kernels, headers, tables or pre/post-processing); both
sides receive their inputs from ``synth`` only.

Contents (each function cites the passage of the paper it follows):

* ``dynamics``  - the recurrences f_t (Brusselator-Euler, mass-action
  Euler/RK4, GRU, linear; the mean-field RNN, two-well Langevin,
  Lorenz-96 with Dormand-Prince steps and the word-problem permutation
  of the thesis's second workloads), their Jacobians and parameter
  derivatives, written as plain per-reaction / per-gate loops.
* ``newton``    - the sequential rollout (the plain definition of the
  answer, Sec. 2.1), the residual (Eq. r_def), the generalised
  quasi-Newton step in correction form (Eq. qdeer_lds, forward
  substitution), the iteration loop of Algorithm alg:deer, and the
  brute-force dense residual Jacobian (Eq. big_j) for tiny problems.
* ``elk``       - Levenberg-Marquardt by dense solve (Eq. lagrangian), the
  Kalman filter of Sec. 4.3 (predict/update with process noise I and
  emission variance 1/lambda) and an RTS smoother for the LM = smoother pin.
* ``adjoint``   - the loss sum_t ||s_t - y_t||^2, its gradient by the
  reverse recursion of Eq. bptt / bptt_lds, by forward sensitivities and by
  central finite differences.
* ``lle``       - the largest Lyapunov exponent along a trajectory by the
  renormalised tangent recursion of Algorithm alg:LLE_estimate.
* ``rng``       - the iid N(0, 1) initial guess of Sec. 3.3.3 from a counter-based
  generator (SplitMix64 outputs through the Box-Muller transform).

Every function runs in float64. Parity unpinned: the iteration counts of the
synthetic workloads (the paper reports none for them).
"""
