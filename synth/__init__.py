"""Seeded synthetic workloads (inputs only; no part of the factorisation)."""
