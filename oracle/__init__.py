"""CPU FP64 oracle of Progressive Material Caching (test infrastructure only)."""
