// batch_c16f.cu -- the persistent batched beamforming kernel for FP16 IQ.
#include "batch_impl.cuh"

rca_status launch_batch_c16f(rca_handle* h, rca_batch* b) { return batch_maxr<__half2>(h, b); }
