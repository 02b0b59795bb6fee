// Pass kernels with check-to-bit messages stored as int8 (step 20/127).
#include "ldpc_pass_kernels.cuh"

LDPC_INSTANTIATE_PASS_KERNELS(int8_t)
