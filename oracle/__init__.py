"""CPU oracle (test infrastructure): see hub_oracle.py."""
