"""CPU oracle for the multiple-precision GEMM / LU path (test infrastructure only)."""
