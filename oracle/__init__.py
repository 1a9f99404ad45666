"""FP64 CPU oracle of the split PFC Vlasov--Poisson step.

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
the CPU-baseline leg of bench.py, never by the package.  See vp_oracle.py.
"""
