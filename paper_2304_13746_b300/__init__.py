"""B300-native (sm_103a) ideal-MHD RK2 stage: PLM + HLLD + E^c constrained transport.

Importing the package loads nothing native; ``paper_2304_13746_b300.idx`` binds
the CUDA library (libidx.so) and ``paper_2304_13746_b300.inputs`` generates the
seeded initial conditions.
"""
