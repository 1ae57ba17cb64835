"""GB300-native batched steady-state PSR solver (libpsr) and its Python binding.

`psr` wraps the C ABI of include/psr.h; `synth` draws seeded synthetic mechanisms and
inlet batches. The CUDA library is built in-tree by `_build.build()`.
"""
