// Direct TSLB step: one thread per interior node, 27 pull-gathers.
//
// For every arriving direction c_i the thread locates the upstream node
// x - c_i (periodic wrap, halfway bounce-back, specular free-slip reflection,
// inflow / outflow ghost layers), rebuilds that node's post-collision
// population f_i from its stored moments with the third-order Hermite
// reconstruction (Eq. eqts + (1 - omega) Eq. noneqts + Luo force, Sec. 2.2 and
// Sec. 3.1) and adds it to the new moments (Sec. 2.1).  This is Eq. pushLB in
// pull form.  It recomputes the 17 mode coefficients of every neighbour, so it
// is ALU-heavy; it is the simple cross-check path for the sum-factorised
// kernel and the fallback for configurations that kernel does not cover.
#include "tslb_internal.cuh"

namespace tslb {
namespace {

template <class Codec>
__device__ __forceinline__ void load_node(const typename Codec::T* __restrict__ src, const Geometry& g,
                                          const Physics& p, long long idx, float m[NFIELDS]) {
    NodeIO<Codec>::load(src, g.fstride, idx, p, m);
}

template <class Codec>
__device__ __forceinline__ void node_modes(const typename Codec::T* __restrict__ src, const Geometry& g,
                                           const Physics& p, long long idx, int zfull, float A[NMODES]) {
    float m[NFIELDS];
    if (!TSLB_IN_RANGE(idx, g.plane * g.nz, p.err)) {
#pragma unroll
        for (int k = 0; k < NMODES; ++k) A[k] = 0.0f;
        return;
    }
    load_node<Codec>(src, g, p, idx, m);
    float F0 = p.F[0], F1 = p.F[1], F2 = p.F[2];
    if (p.force) {
        const float4 f = reinterpret_cast<const float4*>(p.force)[idx];
        F0 = f.x;
        F1 = f.y;
        F2 = f.z;
    }
    post_modes(m[F_DRHO], m[F_UX], m[F_UY], m[F_UZ], m[F_UX], m[F_UY], m[F_UZ], &m[F_PXX], F0, F1, F2,
               omega1_at(p, zfull), A, p.guo != 0);
}

template <class Codec>
__global__ void __launch_bounds__(256) step_direct_kernel(const typename Codec::T* __restrict__ src,
                                                          typename Codec::T* __restrict__ dst, Geometry g,
                                                          Physics p) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = g.plane * g.nz;
    if (n >= total) return;
    const int own[3] = {(int)(n % g.nx), (int)((n / g.nx) % g.ny), (int)(n / g.plane)};
    const int ext[3] = {g.nx, g.ny, g.nz};

    float D0 = 0.f, J[3] = {0.f, 0.f, 0.f}, S[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float Aown[NMODES];
    node_modes<Codec>(src, g, p, n, own[2] + g.lo[2], Aown);

    for (int cz = -1; cz <= 1; ++cz)
        for (int cy = -1; cy <= 1; ++cy)
            for (int cx = -1; cx <= 1; ++cx) {
                int s[3] = {own[0] - cx, own[1] - cy, own[2] - cz};
                int c[3] = {cx, cy, cz};
                bool bounce = false;
                int ghost = 0;  // 1 inflow layer, 2 outflow layer, 3 NEE wall layer
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (s[a] >= 0 && s[a] < ext[a]) continue;
                    const int face = g.bc[2 * a + (s[a] >= ext[a] ? 1 : 0)];
                    if (face == TSLB_BC_PERIODIC) {
                        s[a] = (s[a] + ext[a]) % ext[a];
                    } else if (face == TSLB_BC_BOUNCEBACK) {
                        bounce = true;
                    } else if (face == TSLB_BC_FREESLIP) {
                        s[a] = own[a];
                        c[a] = -c[a];
                    } else if (face == TSLB_BC_NEE_WALL) {
                        ghost = 3;
                        s[a] = s[a] < 0 ? 0 : ext[a] - 1;  // x_F: the adjacent interior node
                    } else if (face == TSLB_BC_INFLOW) {
                        ghost = 1;
                        s[a] = 0;
                    } else {
                        ghost = 2;
                        s[a] = ext[a] - 1;
                    }
                }
                float gi;
                if (bounce) {
                    gi = pop_dev216(Aown, -cx, -cy, -cz);
                } else if (ghost == 3) {
                    // the wall node emits f^eq(rho_F, 0) + (1 - omega) f^neq(Pi_F, u_F) (Eq. neq_final)
                    const long long fidx = (long long)s[0] + (long long)g.nx * s[1] + g.plane * s[2];
                    float m[NFIELDS];
                    load_node<Codec>(src, g, p, fidx, m);
                    float A[NMODES];
                    post_modes(m[F_DRHO], 0.f, 0.f, 0.f, m[F_UX], m[F_UY], m[F_UZ], &m[F_PXX], 0.f, 0.f, 0.f,
                               omega1_at(p, s[2] + g.lo[2]), A);
                    gi = pop_dev216(A, c[0], c[1], c[2]);
                } else if (ghost == 1) {
                    const long long fidx = (long long)s[0] + (long long)g.nx * s[1];  // x_F: first interior layer
                    float m[NFIELDS];
                    load_node<Codec>(src, g, p, fidx, m);
                    const float uBz = inflow_uz(p, (long long)s[0] + g.lo[0], (long long)s[1] + g.lo[1]);
                    float A[NMODES];
                    post_modes(m[F_DRHO], 0.f, 0.f, uBz, m[F_UX], m[F_UY], m[F_UZ], &m[F_PXX], 0.f, 0.f, 0.f,
                               omega1_at(p, 0), A);
                    gi = pop_dev216(A, c[0], c[1], c[2]);
                } else {
                    const long long sidx = (long long)s[0] + (long long)g.nx * s[1] + g.plane * s[2];
                    float A[NMODES];
                    // an outflow ghost relaxes with the omega of its own layer
                    node_modes<Codec>(src, g, p, sidx, ghost == 2 ? ext[2] + g.lo[2] : s[2] + g.lo[2], A);
                    gi = pop_dev216(A, c[0], c[1], c[2]);
                }
                D0 += gi;
                J[0] = fmaf(gi, (float)cx, J[0]);
                J[1] = fmaf(gi, (float)cy, J[1]);
                J[2] = fmaf(gi, (float)cz, J[2]);
                S[0] = fmaf(gi, (float)(cx * cx), S[0]);
                S[1] = fmaf(gi, (float)(cy * cy), S[1]);
                S[2] = fmaf(gi, (float)(cz * cz), S[2]);
                S[3] = fmaf(gi, (float)(cx * cy), S[3]);
                S[4] = fmaf(gi, (float)(cx * cz), S[4]);
                S[5] = fmaf(gi, (float)(cy * cz), S[5]);
            }

    // New moments (Sec. 2.1) from the 216-scaled deviation sums.
    float out[NFIELDS];
    finish_moments(D0, J, S, out);
    if (p.guo) {
        float F0 = p.F[0], F1 = p.F[1], F2 = p.F[2];
        if (p.force) {
            const float4 f = reinterpret_cast<const float4*>(p.force)[n];
            F0 = f.x;
            F1 = f.y;
            F2 = f.z;
        }
        guo_finish(out, F0, F1, F2, 1.0f);
    }
    if (TSLB_IN_RANGE(n, g.plane * g.nz, p.err)) NodeIO<Codec>::store(dst, g.fstride, n, p, out);
}

}  // namespace

cudaError_t launch_step_direct(const tslb_s* h, const void* src, void* dst, const Physics& p) {
    const long long total = h->g.plane * h->g.nz;
    const int threads = 256;
    const unsigned blocks = (unsigned)((total + threads - 1) / threads);
    switch (h->precision) {
        case TSLB_FP32:
            step_direct_kernel<CodecF32><<<blocks, threads, 0, h->stream>>>((const float*)src, (float*)dst, h->g, p);
            break;
        case TSLB_BF16:
            if (h->rounding == TSLB_ROUND_STOCHASTIC)
                step_direct_kernel<CodecBF16SR><<<blocks, threads, 0, h->stream>>>(
                    (const __nv_bfloat16*)src, (__nv_bfloat16*)dst, h->g, p);
            else
                step_direct_kernel<CodecBF16><<<blocks, threads, 0, h->stream>>>(
                    (const __nv_bfloat16*)src, (__nv_bfloat16*)dst, h->g, p);
            break;
        default:
            if (h->rounding == TSLB_ROUND_STOCHASTIC)
                step_direct_kernel<CodecF16SR><<<blocks, threads, 0, h->stream>>>((const __half*)src, (__half*)dst,
                                                                                  h->g, p);
            else
                step_direct_kernel<CodecF16><<<blocks, threads, 0, h->stream>>>((const __half*)src, (__half*)dst,
                                                                                h->g, p);
            break;
    }
    return cudaGetLastError();
}

}  // namespace tslb
