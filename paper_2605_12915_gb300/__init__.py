"""GB300-native RB-TAI Active Flux step (placeholder; binding added below)."""
