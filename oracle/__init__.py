"""FP64 CPU oracle for the EFE residual-ChFSI path -- test infrastructure only.

Only the tests, the smoke check and the CPU-baseline leg of the benchmark use
this package.  It shares no code with the CUDA path and imports nothing from
the product package.
"""
