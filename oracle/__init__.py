"""CPU oracle for NN-sort (test infrastructure only; see oracle.c's header)."""
