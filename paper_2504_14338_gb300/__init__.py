"""GB300-native dOpInf hot path: C-ABI CUDA library plus a thin Python binding.

Importing the package loads nothing; ``paper_2504_14338_gb300.dopinf`` loads the compiled
library and raises if it is missing.
"""
