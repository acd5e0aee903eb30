// batch_c16bf.cu -- the persistent batched beamforming kernel for BF16 IQ.
#include "batch_impl.cuh"

rca_status launch_batch_c16bf(rca_handle* h, rca_batch* b) { return batch_maxr<__nv_bfloat162>(h, b); }
