"""CPU oracle (test infrastructure only; see ``lmfao_oracle``)."""
