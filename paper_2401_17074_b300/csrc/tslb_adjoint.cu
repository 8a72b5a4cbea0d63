// Discrete adjoint of the TSLB step with respect to a per-node body force.
//
// The forward step factors into three maps per node (Sec. 2.1-2.2):
//   A(y)  = modes(m(y), F(y))          local, nonlinear (Eq. eqts / Eq. noneqts / Luo force)
//   G(x)  = sum_i T_i A(x - c_i)        linear gather (streaming, Eq. pushLB, and moment sums)
//   m'(x) = finish(G(x))                local, nonlinear (rho, u, Pi^neq from the sums)
// so the adjoint of one step is
//   Gbar(x) = (d finish / d G)^T lambda'(x)           (kernel adj_finish)
//   Abar(y) = sum_i T_i^T Gbar(y + c_i)                (transpose gather, kernel adj_gather)
//   lambda(y) = (d modes / d m)^T Abar(y),  Fbar(y) += (d modes / d F)^T Abar(y).
// The objective is J = 1/2 sum rho |u|^2 at the final step; the control is a
// time-constant per-node acceleration field.  Segments between the forward
// checkpoints are recomputed with the forward kernel (bitwise identical
// states) and then swept backwards.  Periodic boxes only.
#include <vector>

#include "tslb_internal.cuh"

namespace tslb {
namespace {

template <class Codec>
__device__ __forceinline__ void load_m(const typename Codec::T* __restrict__ src, long long fs, long long idx,
                                       const Physics& p, float m[NFIELDS]) {
    NodeIO<Codec>::load(src, fs, idx, p, m);
}

// lambda at the final step: dJ/d(rho-1) = |u|^2 / 2, dJ/du = rho u, dJ/dPi = 0.
template <class Codec>
__global__ void adj_seed(const typename Codec::T* __restrict__ m_end, float* __restrict__ lam, Geometry g, Physics p) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.plane * g.nz) return;
    float m[NFIELDS];
    load_m<Codec>(m_end, g.fstride, n, p, m);
    const float rho = 1.0f + m[F_DRHO];
    lam[F_DRHO * g.fstride + n] = 0.5f * (m[F_UX] * m[F_UX] + m[F_UY] * m[F_UY] + m[F_UZ] * m[F_UZ]);
    lam[F_UX * g.fstride + n] = rho * m[F_UX];
    lam[F_UY * g.fstride + n] = rho * m[F_UY];
    lam[F_UZ * g.fstride + n] = rho * m[F_UZ];
    for (int k = 0; k < 6; ++k) lam[(F_PXX + k) * g.fstride + n] = 0.0f;
}

// Transpose of finish_moments: G = (D0, J, S) -> (drho', u', Pi') with
//   drho' = D0/216, u_a = J_a / r (r = 216 + D0),
//   Pi_aa = (S_aa - J_a^2 / r - D0/3)/216, Pi_ab = (S_ab - J_a J_b / r)/216.
// Gbar layout: [D0, Jx, Jy, Jz, Sxx, Syy, Szz, Sxy, Sxz, Syz].
template <class Codec>
__global__ void adj_finish(const float* __restrict__ lam, const typename Codec::T* __restrict__ m_next,
                           float* __restrict__ gbar, Geometry g, Physics p) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.plane * g.nz) return;
    float m[NFIELDS], l[NFIELDS];
    load_m<Codec>(m_next, g.fstride, n, p, m);
#pragma unroll
    for (int f = 0; f < NFIELDS; ++f) l[f] = lam[f * g.fstride + n];
    const float u[3] = {m[F_UX], m[F_UY], m[F_UZ]};
    const float inv_r = 1.0f / (216.0f * (1.0f + m[F_DRHO]));
    const float k = 1.0f / 216.0f;
    // lambda_Pi as a symmetric matrix
    const float L[3][3] = {{l[F_PXX], l[F_PXY], l[F_PXZ]}, {l[F_PXY], l[F_PYY], l[F_PYZ]}, {l[F_PXZ], l[F_PYZ], l[F_PZZ]}};
    float gD = l[F_DRHO] * k;
    float gJ[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        gD -= u[a] * l[F_UX + a] * inv_r;
        gD += (u[a] * u[a] - 1.0f / 3.0f) * L[a][a] * k;
        float s = 2.0f * u[a] * L[a][a];
#pragma unroll
        for (int b = 0; b < 3; ++b)
            if (b != a) s += u[b] * L[a][b];
        gJ[a] = l[F_UX + a] * inv_r - s * k;
    }
    gD += (u[0] * u[1] * L[0][1] + u[0] * u[2] * L[0][2] + u[1] * u[2] * L[1][2]) * k;
    gbar[0 * g.fstride + n] = gD;
    gbar[1 * g.fstride + n] = gJ[0];
    gbar[2 * g.fstride + n] = gJ[1];
    gbar[3 * g.fstride + n] = gJ[2];
    for (int c = 0; c < 6; ++c) gbar[(4 + c) * g.fstride + n] = l[F_PXX + c] * k;
}

// Transpose gather + transpose of post_modes at the source node y.
template <class Codec>
__global__ void __launch_bounds__(256) adj_gather(const float* __restrict__ gbar, const typename Codec::T* __restrict__ m_cur,
                                                  float* __restrict__ lam, float* __restrict__ fbar, Geometry g,
                                                  Physics p) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.plane * g.nz) return;
    const int y0 = (int)(n % g.nx), y1 = (int)((n / g.nx) % g.ny), y2 = (int)(n / g.plane);
    float Ab[NMODES];
#pragma unroll
    for (int k = 0; k < NMODES; ++k) Ab[k] = 0.0f;
    for (int cz = -1; cz <= 1; ++cz)
        for (int cy = -1; cy <= 1; ++cy)
            for (int cx = -1; cx <= 1; ++cx) {
                const int x0 = (y0 + cx + g.nx) % g.nx, x1 = (y1 + cy + g.ny) % g.ny, x2 = (y2 + cz + g.nz) % g.nz;
                const long long xi = (long long)x0 + (long long)g.nx * x1 + g.plane * x2;
                const float* G = gbar + xi;
                const long long fs = g.fstride;
                // adjoint population: psi(c) . Gbar(y + c)
                float gb = G[0];
                gb = fmaf((float)cx, G[1 * fs], gb);
                gb = fmaf((float)cy, G[2 * fs], gb);
                gb = fmaf((float)cz, G[3 * fs], gb);
                gb = fmaf((float)(cx * cx), G[4 * fs], gb);
                gb = fmaf((float)(cy * cy), G[5 * fs], gb);
                gb = fmaf((float)(cz * cz), G[6 * fs], gb);
                gb = fmaf((float)(cx * cy), G[7 * fs], gb);
                gb = fmaf((float)(cx * cz), G[8 * fs], gb);
                gb = fmaf((float)(cy * cz), G[9 * fs], gb);
                gb *= wgt(cx) * wgt(cy) * wgt(cz);
#pragma unroll
                for (int k = 0; k < NMODES; ++k) {
                    int k1, k2, k3;
                    mode_digits(k, k1, k2, k3);
                    Ab[k] = fmaf(gb, phi(k1, cx) * phi(k2, cy) * phi(k3, cz), Ab[k]);
                }
            }
    // transpose of post_modes (u = v, constant or per-node force)
    float m[NFIELDS];
    load_m<Codec>(m_cur, g.fstride, n, p, m);
    float F[3] = {p.F[0], p.F[1], p.F[2]};
    if (p.force) {
        F[0] = p.force[n];
        F[1] = p.force[g.fstride + n];
        F[2] = p.force[2 * g.fstride + n];
    }
    const float w1 = p.omega1;
    const float rho = 1.0f + m[F_DRHO];
    const float u[3] = {m[F_UX], m[F_UY], m[F_UZ]};
    // Pi as symmetric matrix (stored xx yy zz xy xz yz)
    const float P[3][3] = {{m[F_PXX], m[F_PXY], m[F_PXZ]}, {m[F_PXY], m[F_PYY], m[F_PYZ]}, {m[F_PXZ], m[F_PYZ], m[F_PZZ]}};
    float lr = Ab[M000];
    float lu[3] = {0.f, 0.f, 0.f};
    float lP[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float fb[3];
    // first order: A_a = 3 rho (u_a + F_a)
    const int m1[3] = {M100, M010, M001};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float ab = Ab[m1[a]];
        lr += 3.0f * (u[a] + F[a]) * ab;
        lu[a] += 3.0f * rho * ab;
        fb[a] = 3.0f * rho * ab;
    }
    // second order diagonal: A_aa = 1.5 (rho u_a^2 + w1 Pi_aa)
    const int m2d[3] = {M200, M020, M002};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float ab = Ab[m2d[a]];
        lr += 1.5f * u[a] * u[a] * ab;
        lu[a] += 3.0f * rho * u[a] * ab;
        lP[a][a] += 1.5f * w1 * ab;
    }
    // second order off-diagonal: A_ab = 9 (rho u_a u_b + w1 Pi_ab)
    const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
    const int m2o[3] = {M110, M101, M011};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int a = pa[q], b = pb[q];
        const float ab = Ab[m2o[q]];
        lr += 9.0f * u[a] * u[b] * ab;
        lu[a] += 9.0f * rho * u[b] * ab;
        lu[b] += 9.0f * rho * u[a] * ab;
        lP[a][b] += 9.0f * w1 * ab;
    }
    // third order A_aab = 4.5 (rho u_a^2 u_b + 2 u_a w1 Pi_ab + u_b w1 Pi_aa)
    const int ta[6] = {0, 0, 1, 1, 2, 2}, tb[6] = {1, 2, 0, 2, 0, 1};
    const int m3[6] = {M210, M201, M120, M021, M102, M012};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const int a = ta[q], b = tb[q];
        const float ab = 4.5f * Ab[m3[q]];
        lr += u[a] * u[a] * u[b] * ab;
        lu[a] += (2.0f * rho * u[a] * u[b] + 2.0f * w1 * P[a][b]) * ab;
        lu[b] += (rho * u[a] * u[a] + w1 * P[a][a]) * ab;
        if (a < b) lP[a][b] += 2.0f * u[a] * w1 * ab;
        else lP[b][a] += 2.0f * u[a] * w1 * ab;
        lP[a][a] += u[b] * w1 * ab;
    }
    // A_xyz = 27 (rho u_x u_y u_z + w1 (u_x Pi_yz + u_y Pi_xz + u_z Pi_xy))
    {
        const float ab = 27.0f * Ab[M111];
        lr += u[0] * u[1] * u[2] * ab;
        lu[0] += (rho * u[1] * u[2] + w1 * P[1][2]) * ab;
        lu[1] += (rho * u[0] * u[2] + w1 * P[0][2]) * ab;
        lu[2] += (rho * u[0] * u[1] + w1 * P[0][1]) * ab;
        lP[1][2] += w1 * u[0] * ab;
        lP[0][2] += w1 * u[1] * ab;
        lP[0][1] += w1 * u[2] * ab;
    }
    const long long fs = g.fstride;
    lam[F_DRHO * fs + n] = lr;
    lam[F_UX * fs + n] = lu[0];
    lam[F_UY * fs + n] = lu[1];
    lam[F_UZ * fs + n] = lu[2];
    lam[F_PXX * fs + n] = lP[0][0];
    lam[F_PYY * fs + n] = lP[1][1];
    lam[F_PZZ * fs + n] = lP[2][2];
    lam[F_PXY * fs + n] = lP[0][1];
    lam[F_PXZ * fs + n] = lP[0][2];
    lam[F_PYZ * fs + n] = lP[1][2];
    fbar[n] += fb[0];
    fbar[fs + n] += fb[1];
    fbar[2 * fs + n] += fb[2];
}

template <class Codec>
cudaError_t adj_launch_all(const tslb_s* h, int which, const void* a, const void* b, float* c, float* d,
                           const Physics& p) {
    const long long total = h->g.plane * h->g.nz;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    typedef typename Codec::T T;
    if (which == 0) adj_seed<Codec><<<blocks, 256, 0, h->stream>>>((const T*)a, c, h->g, p);
    else if (which == 1) adj_finish<Codec><<<blocks, 256, 0, h->stream>>>((const float*)b, (const T*)a, c, h->g, p);
    else adj_gather<Codec><<<blocks, 256, 0, h->stream>>>((const float*)b, (const T*)a, c, d, h->g, p);
    return cudaGetLastError();
}

cudaError_t adj_launch(const tslb_s* h, int which, const void* a, const void* b, float* c, float* d, const Physics& p) {
    switch (h->precision) {
        case TSLB_FP32: return adj_launch_all<CodecF32>(h, which, a, b, c, d, p);
        case TSLB_BF16: return adj_launch_all<CodecBF16>(h, which, a, b, c, d, p);
        default: return adj_launch_all<CodecF16>(h, which, a, b, c, d, p);
    }
}

}  // namespace

// Host driver of the adjoint; error text goes to *msg.  Returns a tslb_status.
int adjoint_force_gradient(tslb_s* h, int64_t nsteps, float* dJdF, int where, std::string* msg) {
    const Geometry& g = h->g;
    const int k = h->checkpoint_every;
    for (int f = 0; f < 6; ++f)
        if (h->bc[f] != TSLB_BC_PERIODIC) {
            *msg = "the adjoint supports periodic boxes only";
            return TSLB_ERR_UNSUPPORTED;
        }
    if (k <= 0) {
        *msg = "create the handle with options.checkpoint_every > 0";
        return TSLB_ERR_STATE;
    }
    if (nsteps <= 0 || nsteps > h->t || (h->t - nsteps) % k != 0) {
        *msg = "nsteps must be in (0, steps taken] with (steps taken - nsteps) a multiple of checkpoint_every";
        return TSLB_ERR_INVALID;
    }
    if ((int64_t)h->ckpts.size() * k < h->t) {
        *msg = "missing checkpoints";
        return TSLB_ERR_STATE;
    }
    const size_t fs = (size_t)g.fstride;
    const size_t state_bytes = (size_t)NFIELDS * fs * h->elem;
    float *lam = nullptr, *gbar = nullptr, *fbar = nullptr;
    char* seg = nullptr;
    cudaError_t e = cudaMalloc(&lam, sizeof(float) * NFIELDS * fs);
    if (e == cudaSuccess) e = cudaMalloc(&gbar, sizeof(float) * NFIELDS * fs);
    if (e == cudaSuccess) e = cudaMalloc(&fbar, sizeof(float) * 3 * fs);
    if (e == cudaSuccess) e = cudaMalloc(&seg, state_bytes * (size_t)(k + 1));
    auto cleanup = [&]() {
        cudaStreamSynchronize(h->stream);
        cudaFree(lam);
        cudaFree(gbar);
        cudaFree(fbar);
        cudaFree(seg);
    };
    if (e != cudaSuccess) {
        cleanup();
        *msg = "adjoint workspace allocation failed";
        return TSLB_ERR_ALLOC;
    }
    Physics p = make_physics(h);
    e = cudaMemsetAsync(fbar, 0, sizeof(float) * 3 * fs, h->stream);
    if (e == cudaSuccess) e = adj_launch(h, 0, h->buf[h->cur], nullptr, lam, nullptr, p);
    int64_t n_end = h->t;
    const int64_t n_stop = h->t - nsteps;
    while (e == cudaSuccess && n_end > n_stop) {
        const int64_t s = (n_end - 1) / k;
        const int64_t n_beg = s * k;
        const int64_t len = n_end - n_beg;
        e = cudaMemcpyAsync(seg, h->ckpts[s], state_bytes, cudaMemcpyDeviceToDevice, h->stream);
        for (int64_t j = 0; j < len && e == cudaSuccess; ++j) {
            Physics pj = p;
            pj.t = n_beg + j;
            pj.sr_key = sr_step_key(h->rounding_seed, pj.t);
            e = launch_step_any(h, seg + j * state_bytes, seg + (j + 1) * state_bytes, pj);
        }
        for (int64_t n = n_end - 1; n >= n_beg && e == cudaSuccess; --n) {
            const char* m_next = seg + (n + 1 - n_beg) * state_bytes;
            const char* m_cur = seg + (n - n_beg) * state_bytes;
            e = adj_launch(h, 1, m_next, lam, gbar, nullptr, p);
            if (e == cudaSuccess) e = adj_launch(h, 2, m_cur, gbar, lam, fbar, p);
        }
        n_end = n_beg;
    }
    // scatter the interior gradient into the full-lattice [3][N] output
    if (e == cudaSuccess) {
        const long long fnx = h->dims[0], fny = h->dims[1], fN = fnx * fny * h->dims[2];
        const cudaMemcpyKind kind = where == TSLB_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        for (int a = 0; a < 3 && e == cudaSuccess; ++a)
            e = cudaMemcpyAsync(dJdF + a * fN, fbar + a * fs, sizeof(float) * (size_t)fN, kind, h->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cleanup();
    if (e != cudaSuccess) {
        *msg = std::string("adjoint: ") + cudaGetErrorString(e);
        return TSLB_ERR_CUDA;
    }
    return TSLB_OK;
}

}  // namespace tslb
