"""FP64 CPU oracle: TEST INFRASTRUCTURE ONLY.

Imported by the test suite, the package smoke check and the benchmark's
CPU-baseline leg; the library never imports it.  See ``nrx_oracle``.
"""
