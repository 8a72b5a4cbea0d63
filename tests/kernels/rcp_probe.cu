// Test probe: evaluates the library's rcp_refined over an array of inputs.
// Built by tests/test_rcp_gpu.py (not part of the library).
#include "tslb_internal.cuh"

__global__ void rcp_probe_kernel(const float* r, float* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = tslb::rcp_refined(r[i]);
}

extern "C" int rcp_probe(const float* r, float* out, int n) {
    rcp_probe_kernel<<<(n + 255) / 256, 256>>>(r, out, n);
    return (int)cudaDeviceSynchronize();
}
