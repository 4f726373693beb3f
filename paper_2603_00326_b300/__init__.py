"""B300 (sm_103a) split search for sparse oblique forests.

The hot path -- projection, min/max, equal-width histograms or exact sort,
Gini scan with double re-score, stable partition, breadth-first tree growth --
runs in the CUDA library lib/libsoforest.so behind the C ABI of
include/soforest.h; `soforest` is its thin Python binding and `datagen` makes
seeded synthetic inputs.
"""
__all__ = ["soforest", "datagen", "build"]
