"""Plain FP64 CPU oracle for the deterministic NQS hot path (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg may import this
package. It shares no code with the CUDA library.
"""
