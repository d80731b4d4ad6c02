"""CPU oracle for averaged RQA -- TEST INFRASTRUCTURE, not part of the product.

A plain, slow, obviously correct restatement of what the method computes,
used only by ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
and ``--impl reference`` legs of ``bench.py`` to check and time the CUDA path.
It shares no code with the CUDA library and never imports it; the product
path never calls anything in here.

* ``rqa_oracle`` -- NumPy: explicit distances, sort-based thresholds,
  run-length scans, DET and its average (Eq. 1-4, Eq. avgDET).
* ``c_oracle``   -- the same definitions as plain C for series too long to
  materialise (streaming counts and diagonal scans), loaded via ctypes.
* ``mlp_oracle`` -- FP64 NumPy forward/backward of the bracket network and its
  quantile loss, plus the distance sketch it reads.
"""
