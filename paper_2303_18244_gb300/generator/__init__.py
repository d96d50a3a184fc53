"""Process generator: diagrams, exact colour algebra, straight-line CUDA emission."""
