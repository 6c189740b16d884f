// Orders 6..8 (generic root and power chain) of the fused beamforming kernel.
#include "pa_bf_kernel.cuh"

PA_DEFINE_ORDER(6)
PA_DEFINE_ORDER(7)
PA_DEFINE_ORDER(8)
