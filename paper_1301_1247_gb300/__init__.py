"""GB300-native fast direct solver for quasi-periodic scattering (HBS + periodizing scheme).

The compute path is the CUDA library libhbsqp.so (C ABI in include/hbsqp.h); `hbs`
is its ctypes binding.  `inputs` holds the seeded synthetic obstacle and angle
generators shared by the tests and the benchmark.
"""
