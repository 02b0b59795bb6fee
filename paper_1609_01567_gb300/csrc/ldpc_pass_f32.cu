// Pass kernels with check-to-bit messages stored as float.
#include "ldpc_pass_kernels.cuh"

LDPC_INSTANTIATE_PASS_KERNELS(float)
