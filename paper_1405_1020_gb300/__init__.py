"""GB300 (sm_103a) histogram oil-paint filter (section 4 of arXiv 1405.1020).

Modules:
  binding  -- ctypes binding of include/oilpaint.h, same names as the C ABI
  filter   -- torch-facing wrappers (OilPaint, Batch)
  synth    -- seeded synthetic inputs (no filter arithmetic)
  autotune -- launch-configuration search per (radius, levels)
  serve    -- continuous-batching request loop over the persistent kernel

Nothing is imported eagerly, so importing the package never needs a GPU.
"""
