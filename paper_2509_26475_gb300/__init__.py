"""GB300-native phi-combination solver (placeholder; the binding is added with the CUDA library)."""
