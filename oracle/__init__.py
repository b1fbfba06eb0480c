"""Oracle for the Holstein HMC hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct CPU implementations of what the GPU library
computes, written from the paper (Cohen-Stead et al., "Fast and scalable
quantum Monte Carlo simulations of electron-phonon models"):

* ``oracle.dense``   -- FP64 NumPy, forms every matrix densely (n = N*Ltau up
  to a few thousand); the definitions written out.
* ``oracle.matfree`` -- plain C (FP64, OpenMP) matrix-free operator, textbook
  CG and the force, for sizes the dense oracle cannot hold; it is also the
  timed CPU baseline.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import anything here. The oracle
shares no code with the CUDA path; both take their inputs from
``holstein_inputs``.
"""
