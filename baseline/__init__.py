"""Baselines the GPU library is reported against (not part of its path)."""
