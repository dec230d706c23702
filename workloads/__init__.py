"""Seeded synthetic workloads (initial data, grids, time steps) shared by the
tests, the benchmark and the smoke check.  Kept outside the product package:
the CUDA library and its binding never import it."""
