// Pass kernels with check-to-bit messages stored as __nv_bfloat16.
#include "ldpc_pass_kernels.cuh"

LDPC_INSTANTIATE_PASS_KERNELS(__nv_bfloat16)
