"""CPU oracle for the EA spin-glass engine (test infrastructure only)."""
