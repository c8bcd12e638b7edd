// k_ext_l12b.cu -- external-product geometries instantiated for N = 4096,
// second part.
#include "hw_ext.cuh"

HW_EXT_TABLE_PART(12, 1, HW_EXT_VARIANT(12, 4, 1, 2) HW_EXT_VARIANT(12, 2, 1, 0) HW_EXT_VARIANT(12, 2, 2, 0) HW_EXT_VARIANT(12, 2, 2, 1) HW_EXT_VARIANT(12, 2, 1, 1) HW_EXT_VARIANT(12, 3, 2, 2) HW_EXT_VARIANT(12, 3, 2, 3))
