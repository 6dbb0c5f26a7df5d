"""GB300-native B-spline registration objective (arXiv 1806.09907, AIRLab).

The compute path is the C-ABI library ``libairgb.so`` (hand-written CUDA for
sm_103a); :mod:`paper_1806_09907_gb300.airgb` is its thin ctypes binding and
:mod:`paper_1806_09907_gb300.synth` draws seeded synthetic inputs. Importing
the package loads nothing; the binding loads the library on first use and
raises if it is missing.
"""
