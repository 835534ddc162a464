"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This package prepares *inputs only*: a radial library of off-axis coronagraph
PSFs (``lyot``), exozodiacal ring scenes with point planets (``scenes``) and the
named workloads built from them (``workloads``).  It holds none of the
interpolation, rotation or contraction arithmetic of the method (Sec. 2-3 of
the paper); the paper's own PSF cubes (Sec. 2, Sec. 4.1) and ZODIPIC scenes
(Sec. 2) are not available, so these generators stand in for them with the
same shapes and the same kind of structure.
"""
