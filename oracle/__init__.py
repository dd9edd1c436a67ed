"""CPU oracle (test infrastructure only; see mfipm_oracle's header)."""
