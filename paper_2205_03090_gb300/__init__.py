"""GB300-native batched isothermal two-phase flash (arXiv 2205.03090)."""
