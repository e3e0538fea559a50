"""Plain, slow FP64 CPU oracle for THC-driven matrix-free CP-ALS.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference arm may import this package. The library path never calls it,
and it shares no code with the CUDA path (only the seeded input generators in
thc_inputs/ serve both).

Modules:
  thc_cpd  - explicit tensors, matrix-free MTTKRP, factor-form loss, CP-ALS.
  mlp      - FP64 forward/backward of the extrapolation MLP.
  exchange - the CPD+THC LT-MP2 exchange energy (single, double, robust).
  corefit  - the THC core least-squares fit f(Z) from a density-fitting tensor.
  df_cpd   - DF-driven CP-ALS (the prior-work O(N^3 R) MTTKRP from the DF tensor).
  nd       - THC-driven CP-ALS of order-d THC-like tensors (two grid-index groups).
"""
