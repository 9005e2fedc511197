"""GB300-native D2Q9 Shan-Chen electrowetting lattice Boltzmann library.

The hot path (one fused collide+stream CUDA kernel per time step, with the
pseudopotential, wall, electric and body forces) lives in ``csrc/`` and is
reached through the C ABI declared in ``include/lbm_ewod.h``. Submodules:

* ``paper_0708_4182_gb300.lbm`` -- thin ctypes binding with the C entry-point
  names, single domains and batched sweeps (loads the compiled library;
  fails loudly when it is missing);
* ``paper_0708_4182_gb300.surrogate`` -- the warm-start U-Net (BF16 kernels of
  ``include/unet_bf16.h``), its training on steady states and warm-started
  batched runs;
* ``paper_0708_4182_gb300.replicas`` -- rank partition and reductions of
  multi-GPU runs;
* ``paper_0708_4182_gb300.workloads`` -- seeded synthetic inputs.

Importing the package itself loads nothing.
"""
