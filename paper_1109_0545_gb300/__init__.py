"""GB300-native hot path of the multithreaded DD/QD polynomial homotopy path tracker
(Verschelde & Yoffe, "Quality Up in Polynomial Homotopy Continuation by Multithreaded
Path Tracking", 2011).

The compute path is the C-ABI CUDA library ``libhc.so`` built from ``csrc/``; the binding
in :mod:`paper_1109_0545_gb300.hc` marshals arguments to it and nothing else.  Importing
this package does not load the library; :func:`paper_1109_0545_gb300.hc.load` does, and
it raises if the library is missing -- there is no CPU fallback.
"""
