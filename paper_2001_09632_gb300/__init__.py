"""GB300-native adaptive block compressive sensing (ABCS) hot path.

The compute lives in the CUDA library libabcs.so (C ABI declared in
include/abcs.h); `paper_2001_09632_gb300.abcs` is the thin ctypes binding
with the same entry-point names.  `synth` holds the seeded input recipe.
Nothing is imported eagerly, so `import paper_2001_09632_gb300.synth` works
on machines without the built library.
"""
__all__ = ["synth", "abcs"]
