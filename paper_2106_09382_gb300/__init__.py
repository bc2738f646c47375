"""CONCORD-PCD on GB300 (package root; the CUDA library loads lazily)."""
