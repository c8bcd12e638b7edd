// k_ext_l6b.cu -- external-product geometries instantiated for N = 64 (test
// rings), second part.
#include "hw_ext.cuh"

HW_EXT_TABLE_PART(6, 1, HW_EXT_VARIANT(6, 4, 1, 2) HW_EXT_VARIANT(6, 2, 1, 0) HW_EXT_VARIANT(6, 2, 2, 0) HW_EXT_VARIANT(6, 2, 2, 1) HW_EXT_VARIANT(6, 3, 2, 2) HW_EXT_VARIANT(6, 3, 1, 2) HW_EXT_VARIANT(6, 3, 2, 3))
