"""Plain, slow FP64 CPU oracle for the spaQR hot path (test infrastructure).

This package is test infrastructure: only the tests, the smoke check and the
benchmark's CPU-baseline / reference arm may import it.  It shares no code with
the CUDA library and imports nothing from it.
"""
