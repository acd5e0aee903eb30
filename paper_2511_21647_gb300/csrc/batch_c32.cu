// batch_c32.cu -- the persistent batched beamforming kernel for FP32 IQ.
#include "batch_impl.cuh"

rca_status launch_batch_c32(rca_handle* h, rca_batch* b) { return batch_maxr<float2>(h, b); }
