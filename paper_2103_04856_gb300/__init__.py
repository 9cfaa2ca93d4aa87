"""GB300-native phase-field curvature energies (Song, arXiv 2103.04856).

Hot path: the energy F_eps(u) of eq. Feps and its exact discrete gradient on a
periodic 3-D voxel grid, iterated by mass-projected gradient descent, as
hand-written CUDA for sm_103a behind the C ABI of ``include/pfc.h``.

Importing this package loads nothing; the CUDA library is loaded on the first
call into ``paper_2103_04856_gb300.pfc`` and raises if it was not built.
"""
__all__ = ["inputs", "pfc"]
