// k_ext_l6.cu -- external-product geometries instantiated for N = 64 (test rings).
#include "hw_ext.cuh"

HW_EXT_TABLE(6, HW_EXT_VARIANT(6, 3, 1, 0) HW_EXT_VARIANT(6, 3, 2, 0) HW_EXT_VARIANT(6, 4, 1, 0) HW_EXT_VARIANT(6, 4, 2, 0) HW_EXT_VARIANT(6, 3, 1, 1) HW_EXT_VARIANT(6, 3, 2, 1) HW_EXT_VARIANT(6, 4, 1, 2) HW_EXT_VARIANT(6, 2, 1, 0) HW_EXT_VARIANT(6, 2, 2, 0) HW_EXT_VARIANT(6, 2, 2, 1) HW_EXT_VARIANT(6, 3, 2, 2) HW_EXT_VARIANT(6, 3, 1, 2))
