"""GB300-native randomized POD (Alg. 1 of arXiv 2504.15350) and its LSTM.

The compute path is librpod.so (hand-written CUDA for sm_103a behind the C ABI
in include/rpod.h).  `paper_2504_15350_gb300.rpod` holds the ctypes binding
(argument marshalling only) and `paper_2504_15350_gb300.build` the nvcc build.
Nothing here computes on the CPU: a missing library raises on first use.
"""
__all__ = ["rpod", "build"]
