"""GB300-native pass-efficient randomized low-rank SVD (Bjarkason 2018).

The compute path is liblowrank.so (CUDA for sm_103a, C ABI in
include/lowrank.h); `api` is its thin torch binding, `synth` the seeded input
generators.  Importing the package does not load the library; the first API
call does, and raises if it has not been built.
"""
