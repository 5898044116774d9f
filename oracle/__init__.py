"""CPU FP64 oracle for FA steepest-descent Landau gauge fixing (test infrastructure only)."""
