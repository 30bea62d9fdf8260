"""Spectral sum-of-Gaussians (SOG) quasi-2D Coulomb summation on one GB300.

The compute path is the C-ABI library ``libsog.so`` (hand-written sm_103a
CUDA, declared in ``include/sog.h``); ``binding`` marshals PyTorch tensors
into it.  ``workloads`` holds the seeded synthetic inputs.
"""
