// learned refinement predictor kernels (filled in later)
