// Order-2 instantiations of the fused beamforming kernel.
#include "pa_bf_kernel.cuh"

PA_DEFINE_ORDER(2)
