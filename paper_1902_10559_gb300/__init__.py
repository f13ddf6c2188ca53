"""GB300 (sm_103a) symmetric-split SART.

Reconstruction of a symmetric tomographic slice by the split of
arXiv:1902.10559.

- ``splitsart``: the Python binding of the C ABI (include/splitsart.h). It
  loads ``libsplitsart.so`` lazily and raises if the library is missing.
- ``synthetic``: seeded synthetic inputs (phantoms, noise draws, presets).
- ``build``: compiles the CUDA library in-tree.

Importing the package loads nothing, so the input generators stay usable on a
machine without the built library.
"""
