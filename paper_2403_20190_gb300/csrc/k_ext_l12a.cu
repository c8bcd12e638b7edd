// k_ext_l12a.cu -- external-product geometries instantiated for N = 4096,
// first part (the default first); k_ext_l12b.cu holds the rest.
#include "hw_ext.cuh"

HW_EXT_TABLE_PART(12, 0, HW_EXT_VARIANT(12, 3, 2, 0) HW_EXT_VARIANT(12, 3, 1, 0) HW_EXT_VARIANT(12, 4, 1, 0) HW_EXT_VARIANT(12, 4, 2, 0) HW_EXT_VARIANT(12, 3, 1, 1) HW_EXT_VARIANT(12, 3, 2, 1))
