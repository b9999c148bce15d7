"""GB300-native multi-scale local-criterion community growth (LFK criterion).

``mscd`` is the Python binding of the CUDA library declared in
include/mscd.h; ``synth`` generates the seeded synthetic input graphs.
"""
