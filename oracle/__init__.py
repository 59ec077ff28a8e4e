"""FP64 CPU oracle of the CPM charge update (test infrastructure only)."""
