// Moment codecs (host FP64 or FP32 <-> stored FP32 / BF16 / FP16 deviations)
// and the FP64 diagnostics reductions of the TSLB library.
#include "tslb_internal.cuh"

namespace tslb {
namespace {

// Full-lattice arrays -> interior storage (layout and 16-bit scaling in
// NodeIO): rho - 1, u and Pi^neq.  H = double (rho given) or float (DEV: the
// deviation rho - 1 given, as stored).
template <class Codec, class H = double, bool DEV = false>
__global__ void encode_kernel(const H* __restrict__ rho, const H* __restrict__ u, const H* __restrict__ pi,
                              typename Codec::T* __restrict__ dst, Geometry g, long long fnx, long long fny,
                              long long fN, Physics p) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.plane * g.nz) return;
    const long long xi = n % g.nx, yi = (n / g.nx) % g.ny, zi = n / g.plane;
    const long long node = (xi + g.lo[0]) + fnx * ((yi + g.lo[1]) + fny * (zi + g.lo[2]));
    float v[NFIELDS];
    v[F_DRHO] = DEV ? (float)rho[node] : (float)(rho[node] - 1.0);
    for (int a = 0; a < 3; ++a) v[F_UX + a] = (float)u[a * fN + node];
    for (int k = 0; k < 6; ++k) v[F_PXX + k] = pi ? (float)pi[k * fN + node] : 0.0f;
    NodeIO<Codec>::store(dst, g.fstride, n, p, v);
}

// Interior storage -> full-lattice arrays (FP64 rho, or with DEV FP32 rho - 1);
// boundary-layer nodes get the rest state.
template <class Codec, class H = double, bool DEV = false>
__global__ void decode_kernel(const typename Codec::T* __restrict__ src, H* __restrict__ rho, H* __restrict__ u,
                              H* __restrict__ pi, Geometry g, long long fnx, long long fny, long long fnz, Physics p) {
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long fN = fnx * fny * fnz;
    if (node >= fN) return;
    const long long xi = node % fnx - g.lo[0], yi = (node / fnx) % fny - g.lo[1], zi = node / (fnx * fny) - g.lo[2];
    const bool inside = xi >= 0 && xi < g.nx && yi >= 0 && yi < g.ny && zi >= 0 && zi < g.nz;
    float v[NFIELDS];
    if (inside) {
        const long long n = xi + g.nx * yi + g.plane * zi;
        NodeIO<Codec>::load(src, g.fstride, n, p, v);
    } else {
        for (int f = 0; f < NFIELDS; ++f) v[f] = 0.0f;
    }
    if (rho) rho[node] = DEV ? (H)v[F_DRHO] : (H)(1.0 + (double)v[F_DRHO]);
    if (u)
        for (int a = 0; a < 3; ++a) u[a * fN + node] = (H)v[F_UX + a];
    if (pi)
        for (int k = 0; k < 6; ++k) pi[k * fN + node] = (H)v[F_PXX + k];
}

// FP64 block reduction of [mass, jx, jy, jz, ke, shear_sum, max_speed, nonfinite].
constexpr int NDIAG = 8;

template <class Codec>
__global__ void __launch_bounds__(256) diag_partial_kernel(const typename Codec::T* __restrict__ src, Geometry g,
                                                           Physics p, double shear_scale,
                                                           double* __restrict__ part) {
    double acc[NDIAG] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long total = g.plane * g.nz;
    const bool ywalls = g.bc[2] == TSLB_BC_BOUNCEBACK || g.bc[2] == TSLB_BC_NEE_WALL;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < total;
         n += (long long)gridDim.x * blockDim.x) {
        float v[NFIELDS];
        NodeIO<Codec>::load(src, g.fstride, n, p, v);
        bool finite = true;
        for (int f = 0; f < NFIELDS; ++f) finite = finite && isfinite(v[f]);
        if (!finite) {
            acc[7] += 1.0;
            continue;
        }
        const double rho = 1.0 + (double)v[F_DRHO];
        const double ux = v[F_UX], uy = v[F_UY], uz = v[F_UZ];
        acc[0] += rho;
        acc[1] += rho * ux;
        acc[2] += rho * uy;
        acc[3] += rho * uz;
        const double u2 = ux * ux + uy * uy + uz * uz;
        acc[4] += 0.5 * rho * u2;
        acc[6] = fmax(acc[6], sqrt(u2));
        if (ywalls) {
            const long long yi = (n / g.nx) % g.ny;
            if (yi == 0) acc[5] += -shear_scale * (double)v[F_PXY];
            if (yi == g.ny - 1) acc[5] += shear_scale * (double)v[F_PXY];
        }
    }
    __shared__ double red[NDIAG][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < NDIAG; ++k) {
        double x = acc[k];
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_xor_sync(0xffffffffu, x, o);
            x = (k == 6) ? fmax(x, y) : x + y;
        }
        if (lane == 0) red[k][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < NDIAG) {
        const int k = threadIdx.x;
        double x = red[k][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) x = (k == 6) ? fmax(x, red[k][w]) : x + red[k][w];
        part[(long long)blockIdx.x * NDIAG + k] = x;
    }
}

__global__ void diag_final_kernel(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
    const int k = threadIdx.x;
    if (k >= NDIAG) return;
    double x = 0.0;
    for (int b = 0; b < nblocks; ++b) x = (k == 6) ? fmax(x, part[b * NDIAG + k]) : x + part[b * NDIAG + k];
    out[k] = x;
}

}  // namespace

cudaError_t launch_encode(const tslb_s* h, const double* rho, const double* u, const double* pi, void* dst,
                          const Physics& p) {
    if (h->lattice == TSLB_D2Q9) return launch_encode2d(h, rho, u, pi, dst);
    const long long total = h->g.plane * h->g.nz;
    const int threads = 256;
    const unsigned blocks = (unsigned)((total + threads - 1) / threads);
    const long long fN = h->dims[0] * h->dims[1] * h->dims[2];
    switch (h->precision) {
        case TSLB_FP32:
            encode_kernel<CodecF32><<<blocks, threads, 0, h->stream>>>(rho, u, pi, (float*)dst, h->g, h->dims[0],
                                                                       h->dims[1], fN, p);
            break;
        case TSLB_BF16:
            encode_kernel<CodecBF16><<<blocks, threads, 0, h->stream>>>(rho, u, pi, (__nv_bfloat16*)dst, h->g,
                                                                        h->dims[0], h->dims[1], fN, p);
            break;
        default:
            encode_kernel<CodecF16><<<blocks, threads, 0, h->stream>>>(rho, u, pi, (__half*)dst, h->g, h->dims[0],
                                                                       h->dims[1], fN, p);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_decode(const tslb_s* h, const void* src, double* rho, double* u, double* pi, const Physics& p) {
    if (h->lattice == TSLB_D2Q9) return launch_decode2d(h, src, rho, u, pi);
    const long long fN = h->dims[0] * h->dims[1] * h->dims[2];
    const int threads = 256;
    const unsigned blocks = (unsigned)((fN + threads - 1) / threads);
    switch (h->precision) {
        case TSLB_FP32:
            decode_kernel<CodecF32><<<blocks, threads, 0, h->stream>>>((const float*)src, rho, u, pi, h->g,
                                                                       h->dims[0], h->dims[1], h->dims[2], p);
            break;
        case TSLB_BF16:
            decode_kernel<CodecBF16><<<blocks, threads, 0, h->stream>>>((const __nv_bfloat16*)src, rho, u, pi,
                                                                        h->g, h->dims[0], h->dims[1], h->dims[2], p);
            break;
        default:
            decode_kernel<CodecF16><<<blocks, threads, 0, h->stream>>>((const __half*)src, rho, u, pi, h->g,
                                                                       h->dims[0], h->dims[1], h->dims[2], p);
            break;
    }
    return cudaGetLastError();
}

// FP32 host interface (D3Q27): drho = rho - 1, u and Pi^neq as FP32 full-lattice arrays.
cudaError_t launch_encode_f32(const tslb_s* h, const float* drho, const float* u, const float* pi, void* dst,
                              const Physics& p) {
    const long long total = h->g.plane * h->g.nz;
    const int threads = 256;
    const unsigned blocks = (unsigned)((total + threads - 1) / threads);
    const long long fN = h->dims[0] * h->dims[1] * h->dims[2];
    switch (h->precision) {
        case TSLB_FP32:
            encode_kernel<CodecF32, float, true><<<blocks, threads, 0, h->stream>>>(drho, u, pi, (float*)dst, h->g,
                                                                                   h->dims[0], h->dims[1], fN, p);
            break;
        case TSLB_BF16:
            encode_kernel<CodecBF16, float, true><<<blocks, threads, 0, h->stream>>>(
                drho, u, pi, (__nv_bfloat16*)dst, h->g, h->dims[0], h->dims[1], fN, p);
            break;
        default:
            encode_kernel<CodecF16, float, true><<<blocks, threads, 0, h->stream>>>(drho, u, pi, (__half*)dst, h->g,
                                                                                   h->dims[0], h->dims[1], fN, p);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_decode_f32(const tslb_s* h, const void* src, float* drho, float* u, float* pi, const Physics& p) {
    const long long fN = h->dims[0] * h->dims[1] * h->dims[2];
    const int threads = 256;
    const unsigned blocks = (unsigned)((fN + threads - 1) / threads);
    switch (h->precision) {
        case TSLB_FP32:
            decode_kernel<CodecF32, float, true><<<blocks, threads, 0, h->stream>>>(
                (const float*)src, drho, u, pi, h->g, h->dims[0], h->dims[1], h->dims[2], p);
            break;
        case TSLB_BF16:
            decode_kernel<CodecBF16, float, true><<<blocks, threads, 0, h->stream>>>(
                (const __nv_bfloat16*)src, drho, u, pi, h->g, h->dims[0], h->dims[1], h->dims[2], p);
            break;
        default:
            decode_kernel<CodecF16, float, true><<<blocks, threads, 0, h->stream>>>(
                (const __half*)src, drho, u, pi, h->g, h->dims[0], h->dims[1], h->dims[2], p);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_diag(const tslb_s* h, const void* src, const Physics& p, double* out_dev) {
    if (h->lattice == TSLB_D2Q9) return launch_diag2d(h, src, out_dev);
    const int threads = 256;
    const double shear_scale = 1.0 - 0.5 * h->omega;
    switch (h->precision) {
        case TSLB_FP32:
            diag_partial_kernel<CodecF32><<<h->diag_blocks, threads, 0, h->stream>>>((const float*)src, h->g, p,
                                                                                     shear_scale, h->diag_part);
            break;
        case TSLB_BF16:
            diag_partial_kernel<CodecBF16><<<h->diag_blocks, threads, 0, h->stream>>>(
                (const __nv_bfloat16*)src, h->g, p, shear_scale, h->diag_part);
            break;
        default:
            diag_partial_kernel<CodecF16><<<h->diag_blocks, threads, 0, h->stream>>>((const __half*)src, h->g, p,
                                                                                     shear_scale, h->diag_part);
            break;
    }
    diag_final_kernel<<<1, 32, 0, h->stream>>>(h->diag_part, h->diag_blocks, out_dev);
    return cudaGetLastError();
}

namespace {
__global__ void pack_force_kernel(const float* __restrict__ planar, float4* __restrict__ packed, long long fs,
                                  long long total) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= total) return;
    packed[n] = make_float4(planar[n], planar[fs + n], planar[2 * fs + n], 0.0f);
}
}  // namespace

cudaError_t launch_pack_force(const tslb_s* h, const float* planar, float* packed) {
    const long long total = h->g.plane * h->g.nz;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    pack_force_kernel<<<blocks, 256, 0, h->stream>>>(planar, reinterpret_cast<float4*>(packed), h->g.fstride, total);
    return cudaGetLastError();
}

}  // namespace tslb
