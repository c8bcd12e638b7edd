"""CPU oracle of the homomorphic WiSARD hot path.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.  It shares no code
with the CUDA library (see oracle.c for the representation and the readings
of the paper it implements).

Parity pins (tests/test_oracle_*.py):
* transform vs schoolbook negacyclic product on tiny rings;
* Philox4x64-10 vs numpy's independent implementation;
* gadget recomposition, encryption/decryption round trips and noise-free
  exactness of the external product, CMUX, blind rotation, CDEMUX, IVP, VP;
* decrypted trained counters == Integer WiSARD counts (Algorithm 4);
* PD-act labels == plaintext WiSARD labels, brute force on tiny inputs;
* the paper's worked examples (Fig. 1, Fig. 2, the T_4 examples).
"""
from ._lib import build, lib  # noqa: F401
from .hom import Oracle  # noqa: F401
from .params import derive  # noqa: F401
from . import wisard  # noqa: F401
