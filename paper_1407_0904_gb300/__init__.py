"""GB300 finite-element local assembly (COFFEE, arXiv:1407.0904)."""
