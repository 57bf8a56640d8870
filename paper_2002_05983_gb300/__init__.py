"""GB300-native repeated star-stencil sweeps (placeholder, filled below)."""
