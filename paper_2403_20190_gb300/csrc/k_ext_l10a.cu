// k_ext_l10a.cu -- external-product geometries instantiated for N = 1024,
// first part (the default first); k_ext_l10b.cu holds the rest.
#include "hw_ext.cuh"

HW_EXT_TABLE_PART(10, 0, HW_EXT_VARIANT(10, 3, 2, 0) HW_EXT_VARIANT(10, 3, 1, 0) HW_EXT_VARIANT(10, 4, 1, 0) HW_EXT_VARIANT(10, 4, 2, 0) HW_EXT_VARIANT(10, 3, 1, 1))
