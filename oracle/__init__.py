"""FP64 CPU oracle of the core-excitation BSE hot path.

TEST INFRASTRUCTURE ONLY: imported by the test-suite, by the smoke check in
the package entry file and by the benchmark's CPU-baseline leg, never by the
product path.  It shares no code with the CUDA library.
"""
