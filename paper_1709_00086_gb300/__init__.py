"""GB300-native anisotropic 3PCF (placeholder; the binding is added below)."""
