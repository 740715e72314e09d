"""CPU oracle for GAME (test infrastructure only; never imported by the product path)."""
