"""GB300-native sparse correlation match (automated crystal orientation
mapping, arXiv 2111.00171): a CUDA library for sm_103a behind a C ABI
(include/acom.h) with a thin ctypes binding."""

from .acom import (ACOM_PREC_BF16, ACOM_PREC_FP32, AcomError, CrystalSpec, Plan,  # noqa: F401
                   au_crystal, cubic_triangle, hexagonal_triangle, library_path,
                   load_library, mg_crystal)
