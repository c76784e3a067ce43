"""Matrix-free Neo-Hookean Jacobian and p-multigrid for B300 (sm_103a).

* ``nh``: ctypes binding of the C ABI in ``include/nh.h`` (``libnh.so``); every
  arithmetic step runs in the library's CUDA kernels, and importing ``nh`` fails
  when the library has not been built.
* ``build``: compiles ``libnh.so`` in-tree with nvcc for sm_103a.
* ``inputs``: seeded synthetic meshes, fields, masks and material layouts (no
  finite-element arithmetic).
* ``learned``: training driver of the learned coarse correction.
"""
