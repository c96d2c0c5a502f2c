"""CPU oracle: plain FP64 restatement of the paper's method.

TEST INFRASTRUCTURE ONLY.  Imported by tests/, by __graft_entry__.smoke() and by
bench.py's CPU-baseline leg; never by the GPU library (paper_2010_12056_gb300),
which shares no code with it.

Parity status of each function:
  cp_oracle.mttkrp / mttkrp_bruteforce / dt_updates / msdt_updates  pinned
  cp_oracle.solve_normal, residual_formula, residual_direct           pinned
  cp_oracle.cp_als (naive / dt / msdt)                                pinned
  cp_oracle.pp_operators, pp_mttkrp, pp_cp_als                        pinned
  mlp_oracle.grad, adam_step                                          pinned
  the learned PP policy's outcome                                     parity unpinned
"""
