"""GB300-native ABIP: ADMM-based interior-point method for LP (arXiv 1805.12344).

The solver lives in the CUDA library ``libabip.so`` (C ABI declared in include/abip.h);
``paper_1805_12344_gb300.abip`` is the thin Python binding and
``paper_1805_12344_gb300.workloads`` the seeded synthetic-LP generators.
"""
