// k_ext_l6a.cu -- external-product geometries instantiated for N = 64 (test
// rings), first part (the default first); k_ext_l6b.cu holds the rest.
#include "hw_ext.cuh"

HW_EXT_TABLE_PART(6, 0, HW_EXT_VARIANT(6, 3, 2, 0) HW_EXT_VARIANT(6, 3, 1, 0) HW_EXT_VARIANT(6, 4, 1, 0) HW_EXT_VARIANT(6, 4, 2, 0) HW_EXT_VARIANT(6, 3, 1, 1) HW_EXT_VARIANT(6, 3, 2, 1))
