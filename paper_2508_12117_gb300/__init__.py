"""GB300-native SPIDER sampling step (placeholder; the binding lands with the library)."""
