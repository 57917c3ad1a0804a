"""FP64 CPU oracle for the Wilson-Dirac CG path (test infrastructure only)."""
