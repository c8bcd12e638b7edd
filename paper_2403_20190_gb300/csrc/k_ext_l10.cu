// k_ext_l10.cu -- external-product geometries instantiated for N = 1024.
#include "hw_ext.cuh"

HW_EXT_TABLE(10, HW_EXT_VARIANT(10, 3, 1, 0) HW_EXT_VARIANT(10, 3, 2, 0) HW_EXT_VARIANT(10, 4, 1, 0) HW_EXT_VARIANT(10, 4, 2, 0) HW_EXT_VARIANT(10, 3, 1, 1) HW_EXT_VARIANT(10, 3, 2, 1) HW_EXT_VARIANT(10, 2, 1, 0) HW_EXT_VARIANT(10, 2, 2, 0) HW_EXT_VARIANT(10, 2, 2, 1))
