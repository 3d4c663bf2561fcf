"""GB300-native batched evaluator for the cuROB benchmark functions
(Ding & Tan, "A CUDA-Based Real Parameter Optimization Benchmark").

The compute lives in ``libcurob.so`` (hand-written sm_103a CUDA behind a C ABI,
declared in ``include/curob.h``); ``binding`` marshals arguments to it.
"""
