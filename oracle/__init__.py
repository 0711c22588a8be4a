"""FP64 CPU oracle for batched beta-CROWN bound propagation.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the tests, the smoke check of ``__graft_entry__`` and the CPU-baseline
leg of ``bench.py`` may use it.  It shares no code with the CUDA path; the
only module both sides read is the seeded input generator
(``paper_2103_06624_gb300.workloads``), which holds none of the method's
arithmetic.

Parity status of each function is stated in ``oracle.bcrown_oracle``'s header.
"""
