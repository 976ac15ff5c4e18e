"""GB300-native HDC classification hot path (ApproxHDC knobs).

Submodules:
  hdc    -- Python binding of the C-ABI library libhdc.so (needs a CUDA GPU)
  build  -- nvcc build of libhdc.so for sm_103a
  synth  -- seeded synthetic workloads (no method arithmetic)
"""
