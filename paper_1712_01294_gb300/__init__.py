"""GB300-native MFM hydrodynamics hot path (placeholder; binding added below)."""
