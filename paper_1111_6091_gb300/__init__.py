"""GB300-native multigrid CP-ALS (placeholder; filled in with the binding)."""
