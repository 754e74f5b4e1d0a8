"""GB300-native high-order kinetic relaxation Poisson solver (placeholder;
the C-ABI binding lands with the CUDA library)."""
