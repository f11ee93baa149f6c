"""GB300-native TA-SC-IVR power spectra (Herman-Kluk, time-averaged, Kaledin-Miller form).

Submodules:
  scivr      -- ctypes binding of the C-ABI library ``libscivr.so`` (CUDA, sm_103a)
  workloads  -- seeded synthetic inputs (potential descriptors, reference states, grids)

Importing this package loads nothing; ``paper_1312_4698_gb300.scivr`` loads the
CUDA library and raises if it has not been built.
"""
__version__ = "0.1.0"
