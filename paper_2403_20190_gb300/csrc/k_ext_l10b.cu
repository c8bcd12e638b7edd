// k_ext_l10b.cu -- external-product geometries instantiated for N = 1024,
// second part.
#include "hw_ext.cuh"

HW_EXT_TABLE_PART(10, 1, HW_EXT_VARIANT(10, 3, 2, 1) HW_EXT_VARIANT(10, 2, 1, 0) HW_EXT_VARIANT(10, 2, 2, 0) HW_EXT_VARIANT(10, 2, 2, 1))
