// Dispatch of the sum-factorised step to the per-storage-type instances
// (tslb_step_factored_{f32,bf16,bf16sr,f16,f16sr}.cu; kernels in tslb_step_factored.cuh).
#include "tslb_internal.cuh"

namespace tslb {

cudaError_t launch_factored_CodecF32(const tslb_s*, const void*, void*, const Physics&, int, int);
cudaError_t launch_factored_CodecBF16(const tslb_s*, const void*, void*, const Physics&, int, int);
cudaError_t launch_factored_CodecBF16SR(const tslb_s*, const void*, void*, const Physics&, int, int);
cudaError_t launch_factored_CodecF16(const tslb_s*, const void*, void*, const Physics&, int, int);
cudaError_t launch_factored_CodecF16SR(const tslb_s*, const void*, void*, const Physics&, int, int);

bool factored_supports(const tslb_s* h) {
    // node offsets inside a field are unsigned 32-bit (n = col + plane * z, and
    // every byte offset is formed in 64 bits from it): up to 2^32 - 1 nodes,
    // which covers FP32 storage up to the device's memory (80 bytes per node
    // for the two buffers) and 16-bit storage up to 4.29 G nodes
    return (long long)h->g.plane * h->g.nz < (1LL << 32);
}

cudaError_t launch_step_factored_range(const tslb_s* h, const void* src, void* dst, const Physics& p, int zlo,
                                       int zhi) {
    if (zhi <= zlo) return cudaSuccess;
    switch (h->precision) {
        case TSLB_FP32: return launch_factored_CodecF32(h, src, dst, p, zlo, zhi);
        case TSLB_BF16:
            return h->rounding == TSLB_ROUND_STOCHASTIC ? launch_factored_CodecBF16SR(h, src, dst, p, zlo, zhi)
                                                        : launch_factored_CodecBF16(h, src, dst, p, zlo, zhi);
        default:
            return h->rounding == TSLB_ROUND_STOCHASTIC ? launch_factored_CodecF16SR(h, src, dst, p, zlo, zhi)
                                                        : launch_factored_CodecF16(h, src, dst, p, zlo, zhi);
    }
}

cudaError_t launch_step_factored(const tslb_s* h, const void* src, void* dst, const Physics& p) {
    return launch_step_factored_range(h, src, dst, p, 0, h->g.nz);
}

}  // namespace tslb
