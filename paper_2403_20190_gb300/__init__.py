"""GB300 (sm_103a) homomorphic WiSARD hot path.

Encrypted training (Algorithm 6) and inference (Algorithm 7, PD-act) of an
Integer WiSARD over RLWE/RGSW ciphertexts, implemented in CUDA behind the C
ABI of include/hwisard.h (libhwisard.so).  ``binding`` exposes the C calls
under their own names; ``session`` wraps them with torch-allocated device
buffers for a whole workload.
"""
from . import binding  # noqa: F401
from .binding import (HwError, hw_create, hw_decrypt, hw_encode, hw_encrypt_sample,  # noqa: F401
                      hw_export_rgsw, hw_get_ram_slots, hw_get_sizes, hw_infer,
                      hw_infer_scratch_words, hw_keygen, hw_launch_count, hw_ntt_forward,
                      hw_ntt_inverse, hw_pdact, hw_train_accumulate, hw_train_scratch_words)
