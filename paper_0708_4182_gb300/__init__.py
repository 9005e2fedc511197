"""GB300-native D2Q9 Shan-Chen electrowetting lattice Boltzmann library.

The hot path (one fused collide+stream CUDA kernel per time step, with the
pseudopotential, wall, electric and body forces) lives in ``csrc/`` and is
reached through the C ABI declared in ``include/lbm_ewod.h``. Submodules:

* ``paper_0708_4182_gb300.lbm`` -- thin ctypes binding with the C entry-point
  names (loads the compiled library; fails loudly when it is missing);
* ``paper_0708_4182_gb300.workloads`` -- seeded synthetic inputs.

Importing the package itself loads nothing.
"""
