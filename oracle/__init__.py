"""FP64 CPU oracle of the dOpInf hot path: test infrastructure, never the product path."""
