"""Multifaceted 4D feature segmentation (Sauer & Ma, arXiv 1903.12294) on GB300.

The compute path is the CUDA library ``libmsf.so`` built from ``csrc/`` for sm_103a; the
binding in ``msf.py`` is argument marshalling over its C ABI (``include/msf.h``). ``synth``
holds the seeded synthetic workloads.
"""
