"""GB300-native pseudospectral Navier-Stokes hot path (placeholder; the
binding is added with the CUDA library)."""
