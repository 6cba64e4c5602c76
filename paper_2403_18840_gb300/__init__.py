"""GB300-native batched self-energy integrand evaluation (arXiv 2403.18840 hot path)."""
