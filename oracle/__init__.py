"""CPU oracle of the NGP-RT render path: test infrastructure only."""
