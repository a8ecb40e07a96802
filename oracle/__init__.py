"""Plain FP64 CPU oracle of the improved Yau--Yau filter's online stage.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import or run anything in this package; the product path never
does.  The oracle shares no code with the CUDA path: it reads only the seeded inputs from
``synth`` and follows the paper's definitions step by step in float64.

Modules (each cites the passage it follows):
    coeffs   multi-scale kernel coefficients, generalised Vandermonde system
             ("High-Order Kernel Construction")
    sobol    Sobol points (Gray code, Appendix A) and the affine scramble
    model    drift, divergence and sensor of the two workload models; complex-step
             divergence ("Numerical Divergence Calculation")
    filter   one filter step: kernel prediction ("Solving Kolmogorov Equations ...",
             "Log-Domain Computation"), Ito-corrected update
             ("Procedure for the Improved Yau-Yau Algorithm"), log-domain normalisation,
             estimate, ESS, restart ("Local Resampling-Restart Mechanism")
    kalman   exact discrete Kalman filter for the Euler-discretised linear model
    metrics  RMSE and ME ("Numerical Experiments", error metrics)
    mlp      FP64 reference of the restart-proposal MLP (forward, backward, Adam)

Pins: every function is checked by ``tests/test_oracle_*.py`` against closed forms,
brute force, invariants or printed values; see the test files for which pin covers which
function.
"""
