"""GB300-native iterative cone-beam CT: interpolated projector, voxel-driven
backprojector, TV step and SIRT / OS-SART / CGLS drivers behind a C ABI.

Importing the package loads nothing native; ``paper_1905_03748_gb300.tigre``
loads the CUDA library (and raises if it has not been built).
"""
