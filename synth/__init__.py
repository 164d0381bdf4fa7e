"""Seeded synthetic inputs (no SPH arithmetic here)."""
