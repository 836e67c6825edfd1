"""GB300-native batched alignment DP for MuSAlS (arXiv 2601.15458)."""
