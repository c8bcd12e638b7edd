// k_ext_l13.cu -- external-product geometries instantiated for N = 8192.
#include "hw_ext.cuh"

HW_EXT_TABLE(13, HW_EXT_VARIANT(13, 3, 1, 0) HW_EXT_VARIANT(13, 4, 1, 0) HW_EXT_VARIANT(13, 4, 1, 2) HW_EXT_VARIANT(13, 3, 1, 2) HW_EXT_VARIANT(13, 3, 1, 3) HW_EXT_VARIANT(13, 4, 1, 3))
