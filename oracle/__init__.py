"""Oracle: plain, slow, obviously correct CPU implementations of what the CUDA
path computes, written from the paper (FP64).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
baseline leg of the benchmark may import or run anything in this package.  It
shares no code with the CUDA library; the two sides only receive the same seeded
inputs.
"""
