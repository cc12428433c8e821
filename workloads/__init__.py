"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This package holds no arithmetic of the lensing method itself: it draws
particle positions, random density fields and galaxy catalogues, and turns
cosmological parameters into the plane distances and source scalings that
both the CUDA library and the oracle receive as plain inputs.  The paper's
N-body light cones (Carmen, Lb2600; Table 1) are not available, so these
generators stand in for them.
"""
