"""GB300-native multigrid solve of the coupled pressure-temperature system.

Saade, Lohse & Fuster, Sec. 3 (Eqs. 27-34): per cell a 2x2 local block plus
face-weighted Laplacians (1/rho for p, k for T), solved by multigrid on one GPU.

Submodules:
  inputs   seeded synthetic inputs (no solver arithmetic)
  binding  ctypes binding of the C-ABI library libcoupledmg.so (loaded lazily)
  serve    continuous-batching request loop over the C-ABI
"""
__all__ = ["inputs", "binding"]
