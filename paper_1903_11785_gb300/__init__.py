"""GB300 (sm_103a) coarse-to-fine visual-hull reconstruction: the hot path of
"A Fast Free-viewpoint Video Synthesis Algorithm for Sports Scenes"
(arXiv 1903.11785) as a C-ABI CUDA library (libfvv.so, include/fvv.h) with a
thin ctypes binding (paper_1903_11785_gb300.fvv).

Build the library with paper_1903_11785_gb300.build.build(); importing
paper_1903_11785_gb300.fvv fails loudly if it is missing.
"""
