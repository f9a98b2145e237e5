"""GB300-native feature-field Gaussian rasterizer (package placeholder)."""
