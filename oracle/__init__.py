"""Plain, slow FP64 CPU oracle for the LF-LTS / MLMC hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never calls it, and it shares no code with the CUDA library: the only
inputs both sides receive come from the seeded generators in ``workload/``.

Modules
  fem   P1 element geometry, lumped mass, stiffness assembly, coefficient
        (Sec. 3.1, Eq. (3.1)-(3.2) and the paragraph defining M, K, F)
  lts   leapfrog (Eq. LF2scheme) and stabilised LF-LTS (Alg. 2) in the
        paper's symmetric z-form, per-sample solves and the QoI
  mlmc  MLMC estimator, variance, optimal sample numbers, bias test and
        the adaptive driver (Sec. 2.2, Eqs. MLMCestimator, Vell_est,
        optimal_Nl, bias_est, Alg. 1)
  adjoint  discrete adjoint of the u-form LF-LTS solve with full history
        and central finite differences (gradient of Q with respect to xi)
  field_qoi  the L2(D)-valued QoI u(., T) (Sec. 4): interpolation between
        level meshes, the consistent mass matrix, V-norm level sums, mean and
        variance (Eqs. MLMCestimator, Vell_est, bias_est in V = L2(D))
"""
