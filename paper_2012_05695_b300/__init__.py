"""B300 (sm_103a) DDM structure function through a Fourier transform in time.

Implements the WITH_FT scheme of Norouzisadeh, Cerchiari, Croccolo (arXiv 2012.05695):
per wave vector, D(q, m) from running sums of |F|^2 and the autocorrelation of the
zero-padded time sequence, behind the C ABI of include/ddm.h.  This package is the thin
Python binding; all arithmetic runs in the CUDA library built from csrc/.
"""
from ._binding import (DDM_IN_F32, DDM_IN_U16, DDM_PREC_FP32, DDM_PREC_FP32_FP64FIX, DDM_PREC_FP64,  # noqa: F401
                       DDM_PREC_TC_TF32X3,
                       DDMError, LIB_PATH, MLP, Plan, header_functions, lib, selftest_bounded_wait,
                       spectrum_index_map, status_string)
