"""GB300-native direct-sum Hermite N-body force engine.

Submodules (import them explicitly):

* ``paper_0709_4552_gb300.nbody``  -- thin ctypes binding to the CUDA C-ABI
  library ``libnbody.so`` built from ``csrc/`` for sm_103a;
* ``paper_0709_4552_gb300.inputs`` -- seeded synthetic inputs (no method
  arithmetic, no GPU library needed);
* ``paper_0709_4552_gb300.build``  -- compiles ``libnbody.so`` with nvcc.
"""
