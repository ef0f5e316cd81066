"""Plain, slow CPU oracle for RNS-CKKS evaluation of neural-network graphs
(arXiv 2110.13638).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke()
and the cpu_baseline / --impl reference legs of bench.py may import it.  The
CUDA library (paper_2110_13638_gb300) never imports it and shares no code,
header, table or constant generator with it.

Layout:
  ckks_oracle.c  -- C core: exact modular arithmetic ('%' on 128-bit products),
                    textbook negacyclic NTT + schoolbook product, SplitMix64
                    samplers, binary128 canonical-embedding encode/decode
  core.py        -- ctypes wrappers of the C core
  params.py      -- Alg. autoHE / autoHE_discover / parameterise, primes,
                    primitive roots, Gaussian table (decimal, 80 digits)
  ckks.py        -- keys, encrypt/decrypt, tensor, key switching, rescale,
                    the dense / square / degree-3 blocks, Alg. firing, and the
                    FP64 plaintext forward pass

Parity pins: every function here is checked by tests/test_oracle_*.py against
closed forms, brute force on tiny inputs, big-integer arithmetic and the
coefficients the paper prints (Eq. sigmoid_approximate).  No function is
"parity unpinned".
"""
from . import core, params, ckks  # noqa: F401
