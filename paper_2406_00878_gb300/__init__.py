"""GB300-native all-at-once BDF1 Newton solver (parallel-in-time direct inverse).

The compute path is the CUDA library ``libpit.so`` (C ABI declared in
``include/pit.h``); ``paper_2406_00878_gb300.pit`` is its thin ctypes binding and
``paper_2406_00878_gb300.workloads`` builds seeded synthetic inputs.  Importing
this package loads nothing; the binding loads the library on first use and
raises if it is missing.
"""
__all__ = ["pit", "workloads", "build"]
