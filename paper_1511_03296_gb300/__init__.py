"""GB300-native Fast Bilateral Solver (hot path on sm_103a)."""
