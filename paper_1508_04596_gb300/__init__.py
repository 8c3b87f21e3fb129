"""GB300-native stabilised Q1-Q1 natural-convection solver (Alexandersen, Sigmund, Aage).

The compute path lives in the C-ABI library ``libnc.so`` built from ``csrc/``;
``paper_1508_04596_gb300.nc`` is its Python binding.  ``synth`` holds the seeded
workload generators.  Importing this package loads nothing.
"""
