"""FP64 CPU oracle of the MUSER imaging hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct NumPy implementations of what the GPU library
computes, written from the paper (Mei et al., "GPU-Based High-Performance Imaging
for Mingantu Spectral RadioHeliograph") and the textbook definitions it relies on.
Every function cites the passage it follows.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and its
Python binding) never imports, calls or links it, and this package never imports
the product.  The two share no code; only the seeded input generator (``synth``)
feeds both.

Modules
  geometry   -- (u, v, w), pixel-size rule, per-visibility grid records    (Sec. 3.2)
  pswf       -- prolate spheroidal kernel, its table and grid correction (Sec. 3.2.3)
  imaging    -- gridding, inverse FFT, dirty map / dirty beam, direct DFT (Sec. 3.2.3, Alg. 1)
  gmm        -- histogram + Gaussian mixture: sky and disk brightness      (Sec. 4.1)
  clean      -- Hogbom CLEAN with the sky-brightness stopping rule          (Sec. 4.3, Alg. 1)
  restore    -- clean beam fit and restored image                          (Alg. 1)
  centering  -- solar-disk centring and phase correction                   (Sec. 4.2, Alg. 1)
  operator   -- degridding forward operator, adjoint, chi-square gradient
  steer      -- Steer clean in major cycles                                (Sec. 3.2, Alg. 1)
  wproj      -- w-projection: w-kernel tables, gridding, direct transform with w (Sec. 6.1, Alg. 1)
  pipeline   -- one instance end to end

Parity status: every function is pinned by the ``-m "not gpu"`` tests except where
its docstring says "parity unpinned".
"""
