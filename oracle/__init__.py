"""FP64 CPU oracle (test infrastructure; the CUDA library never imports it)."""
