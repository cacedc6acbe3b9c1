"""Independent exact computations used to pin the oracle (brute force, closed forms, ED)."""
