// k_ext_misc.cu -- external-product geometries instantiated for N = 128, 256, 512 and 2048 (default geometry only).
#include "hw_ext.cuh"

HW_EXT_TABLE(7, HW_EXT_VARIANT(7, 3, 2, 0))
HW_EXT_TABLE(8, HW_EXT_VARIANT(8, 3, 2, 0))
HW_EXT_TABLE(9, HW_EXT_VARIANT(9, 3, 2, 0))
HW_EXT_TABLE(11, HW_EXT_VARIANT(11, 3, 2, 0))
