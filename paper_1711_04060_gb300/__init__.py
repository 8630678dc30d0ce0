"""GB300-native Poisson-Fermi solver (placeholder; the binding is added with the library)."""
