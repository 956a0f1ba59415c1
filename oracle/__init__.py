"""CPU oracle of the ST-HOSVD + bit-plane quantization path (TEST INFRASTRUCTURE).

This package is test infrastructure.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` may import it.  It shares
no code, header, table or helper with the CUDA library under
``paper_2107_01384_gb300/``; the only thing both sides consume is the seeded
input data from ``synth``.

* ``oracle.sthosvd`` -- FP64 NumPy restatement of Algorithm 1 with the error
  control of Section 4.1.3 (Gram + ``numpy.linalg.eigh`` as the SVD step).
* ``oracle.quant``   -- ctypes front of ``quant.c``: exact-integer bit-plane
  tracker, breakpoint, run-length + rANS block encoder and decoder
  (Sections 3.3, 4.2, 4.3, supplement S.6).
* ``oracle.pipeline`` -- the whole compressor / decompressor stream built from
  the two above.
"""
from .build import build_oracle  # noqa: F401
