"""GB300-native DDHF hot path (placeholder; the binding is added with the library)."""
