"""CPU oracle for the RNS-CKKS CinS conv2d + bootstrapping path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, independent
re-statement of the paper's method used to check the CUDA library
(paper_2312_04356_gb300).  It shares no code with it.  Only tests/,
__graft_entry__.smoke() and the cpu_baseline / reference legs of bench.py may
import it; the library itself never does.

Modules
  ckks_ref.c   integer primitives (NTT, base conversion, rescale, samplers), gcc + OpenMP
  _clib.py     ctypes loader / numpy wrappers for ckks_ref.c
  params.py    primes, roots, canonical scale ladder, named parameter sets
  encoding.py  FP64 encodings, special DFT factors, real CinS, conv kernels
  scheme.py    keys, encryption, key switching, rotations, BSGS, Chebyshev evaluation
  boot.py      Alg. 1 block: fused conv, ModRaise, CtoS, EvalMod, mask, StoC1
  plain.py     the same steps without the key-switch restructurings (a ModDown per
               rotation, separate rescales, term-by-term Chebyshev series), to pin them

Parity status: every function is pinned by tests/test_oracle_*.py against a
value or identity the paper or the mathematics fixes (see the test docstrings).
"""
