// Pass kernels with check-to-bit messages stored as __half.
#include "ldpc_pass_kernels.cuh"

LDPC_INSTANTIATE_PASS_KERNELS(__half)
